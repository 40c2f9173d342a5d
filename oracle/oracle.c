/*
 * oracle.c -- FP64 CPU oracle for Armadillo-style expression trees.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Plain, slow, one operation at a time; every node materialises
 * a full matrix.  See oracle.h for the program format and the error-bound
 * model.
 *
 * Definitions followed (Bandicoot paper):
 *   Sec. 2  -- Armadillo-compatible function semantics: accu, sum/mean along a
 *             dimension, statistics such as variance, submatrix views.
 *   Sec. 3  -- Op (trans), eOp (element-wise unary incl. scalar forms),
 *             eGlue (element-wise binary: + - % /) and delayed evaluation:
 *             the fused result equals the eager one-op-at-a-time result up to
 *             rounding, which is what this walker computes.
 *   Sec. 4  -- column-major storage: element (i,j) at data[i + j*ld].
 * Readings where the paper is silent (documented with the design):
 *   - a scalar in a tree is converted to the element type (compute type for
 *     BF16/FP16 storage), as an Armadillo scalar of type eT is;
 *   - INT32 + - * wrap modulo 2^32; / truncates toward zero, a zero divisor
 *     gives 0 and raises the div_by_zero flag; reductions are exact int64
 *     (modulo 2^64); dot multiplies exactly in int64;
 *   - var uses N-1 (norm_type 0) or N (norm_type 1), two passes; N==1 gives 0;
 *   - norm of a vector is the 2-norm; matrices take the Frobenius norm only.
 *
 * Threads: the element-wise loops (every element computed on its own) carry
 * OpenMP pragmas.  Built with -fopenmp (liborc_omp.so) they run on all host
 * cores; without it (liborc.so) the pragmas are ignored.  Every reduction is
 * one sequential pass in either build, so the two builds give bit-identical
 * values and bounds.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads the element-wise loops of this build use */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* helpers                                                             */
/* ------------------------------------------------------------------ */

double orc_ulp(double x, int32_t dtype) {
  int e;
  int mant_bits, emin;
  x = fabs(x);
  switch (dtype) {
    case ORC_F32: mant_bits = 24; emin = -126; break;
    case ORC_F64: mant_bits = 53; emin = -1022; break;
    case ORC_BF16: mant_bits = 8; emin = -126; break;
    case ORC_F16: mant_bits = 11; emin = -14; break;
    default: return 0.0;
  }
  if (isnan(x) || isinf(x)) return 0.0;
  (void)frexp(x, &e); /* x = m * 2^e, m in [0.5, 1) -> x in [2^(e-1), 2^e) */
  if (x == 0.0 || e - 1 < emin) e = emin + 1;
  return ldexp(1.0, e - mant_bits);
}

double orc_sum_neumaier(const double* x, int64_t n) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = s + x[i];
    if (fabs(s) >= fabs(x[i]))
      c += (s - t) + x[i];
    else
      c += (x[i] - t) + s;
    s = t;
  }
  return s + c;
}

static double sum_plain(const double* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i];
  return s;
}

static int64_t wrap32(int64_t x) { return (int64_t)(int32_t)(uint32_t)(uint64_t)x; }

static double bf16_to_double(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

static double f16_to_double(uint16_t h) {
  int sign = (h >> 15) & 1;
  int e = (h >> 10) & 31;
  int m = h & 1023;
  double v;
  if (e == 0)
    v = ldexp((double)m, -24);
  else if (e == 31)
    v = (m == 0) ? INFINITY : NAN;
  else
    v = ldexp((double)(1024 + m), e - 25);
  return sign ? -v : v;
}

/* |d| * b, with 0 when b == 0 (so an exact input never turns inf*0 into NaN) */
static double mulb(double d, double b) { return b == 0.0 ? 0.0 : fabs(d) * b; }

/* ------------------------------------------------------------------ */
/* values on the evaluation stack                                      */
/* ------------------------------------------------------------------ */

enum { V_MAT = 0, V_SCALAR = 1 };

typedef struct {
  int kind;
  int64_t r, c;
  double* v;   /* FP values */
  double* b;   /* FP bounds */
  int64_t* iv; /* integer values */
  double k;    /* scalar (already converted to the element type) */
} val_t;

typedef struct {
  int is_int;
  int ct; /* compute dtype: ORC_F32, ORC_F64 or ORC_I32 */
  int div0;
  char* err;
} ctx_t;

static void val_free(val_t* x) {
  free(x->v);
  free(x->b);
  free(x->iv);
  x->v = x->b = NULL;
  x->iv = NULL;
}

static int val_alloc(ctx_t* cx, val_t* x, int64_t r, int64_t c) {
  size_t n = (size_t)(r * c);
  size_t nn = n ? n : 1;
  x->kind = V_MAT;
  x->r = r;
  x->c = c;
  x->v = x->b = NULL;
  x->iv = NULL;
  if (cx->is_int) {
    x->iv = (int64_t*)calloc(nn, sizeof(int64_t));
    if (!x->iv) return -1;
  } else {
    x->v = (double*)calloc(nn, sizeof(double));
    x->b = (double*)calloc(nn, sizeof(double));
    if (!x->v || !x->b) return -1;
  }
  return 0;
}

/* local rounding allowance of a node in the compute type, plus the
 * oracle's own FP64 rounding of the same node */
static double local(ctx_t* cx, double v, double c_dev, double c_orc) {
  if (!isfinite(v)) return 0.0;
  return c_dev * orc_ulp(v, cx->ct) + c_orc * orc_ulp(v, ORC_F64);
}

static double finite_or_zero_bound(double v, double b) { return isfinite(v) ? b : 0.0; }

/* Largest magnitude that still rounds to a finite value of the format (the
 * IEEE overflow threshold: max finite + half an ulp of max finite). */
static double overflow_threshold(int32_t dtype) {
  switch (dtype) {
    case ORC_F32: return ldexp(2.0 - ldexp(1.0, -24), 127);   /* (2 - 2^-24) 2^127 */
    case ORC_BF16: return ldexp(2.0 - ldexp(1.0, -8), 127);   /* (2 - 2^-8)  2^127 */
    case ORC_F16: return 65520.0;                              /* (2 - 2^-11) 2^15  */
    default: return INFINITY;
  }
}

/* A node result outside the compute type's range is what an IEEE device
 * returns for it: +-inf (exact, so its bound is 0). */
static void clamp_to_range(ctx_t* cx, double* v, double* b) {
  if (cx->ct == ORC_F32 && isfinite(*v) && fabs(*v) >= overflow_threshold(ORC_F32)) {
    *v = copysign(INFINITY, *v);
    *b = 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* leaves                                                              */
/* ------------------------------------------------------------------ */

static int load_leaf(ctx_t* cx, const orc_mat* m, val_t* out) {
  if (m->n_rows < 0 || m->n_cols < 0 || m->ld < m->n_rows) {
    snprintf(cx->err, 256, "leaf: bad shape");
    return -1;
  }
  if (val_alloc(cx, out, m->n_rows, m->n_cols)) {
    snprintf(cx->err, 256, "out of memory");
    return -1;
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t j = 0; j < m->n_cols; ++j)
    for (int64_t i = 0; i < m->n_rows; ++i) {
      int64_t s = i + j * m->ld, d = i + j * m->n_rows;
      switch (m->dtype) {
        case ORC_F32: out->v[d] = (double)((const float*)m->data)[s]; break;
        case ORC_F64: out->v[d] = ((const double*)m->data)[s]; break;
        case ORC_BF16: out->v[d] = bf16_to_double(((const uint16_t*)m->data)[s]); break;
        case ORC_F16: out->v[d] = f16_to_double(((const uint16_t*)m->data)[s]); break;
        case ORC_I32: out->iv[d] = (int64_t)((const int32_t*)m->data)[s]; break;
      }
    }
  return 0; /* stored values are exact: bounds stay 0 */
}

/* ------------------------------------------------------------------ */
/* element-wise operations                                             */
/* ------------------------------------------------------------------ */

enum { U_NEG, U_EXP, U_LOG, U_ABS, U_SQUARE, U_SQRT, U_TRANS };
enum { B_PLUS, B_MINUS, B_SCHUR, B_DIV, B_TIMES };

static int unary(ctx_t* cx, int op, val_t* x, val_t* out) {
  int64_t r = x->r, c = x->c, n = r * c;
  if (op == U_TRANS) {
    if (val_alloc(cx, out, c, r)) return -1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t j = 0; j < c; ++j)
      for (int64_t i = 0; i < r; ++i) {
        /* trans(X)(j,i) = X(i,j) */
        int64_t s = i + j * r, d = j + i * c;
        if (cx->is_int)
          out->iv[d] = x->iv[s];
        else {
          out->v[d] = x->v[s];
          out->b[d] = x->b[s];
        }
      }
    return 0;
  }
  if (val_alloc(cx, out, r, c)) return -1;
  if (cx->is_int) {
    if (op != U_NEG && op != U_ABS && op != U_SQUARE) {
      snprintf(cx->err, 256, "exp/log/sqrt are not defined for INT32 trees");
      return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) {
      int64_t a = x->iv[t];
      switch (op) {
        case U_NEG: out->iv[t] = wrap32(-a); break;
        case U_ABS: out->iv[t] = wrap32(a < 0 ? -a : a); break;
        default: out->iv[t] = wrap32((int64_t)((uint64_t)a * (uint64_t)a)); break; /* U_SQUARE */
      }
    }
    return 0;
  }
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < n; ++t) {
    double a = x->v[t], ba = x->b[t], v = 0.0, bv = 0.0;
    switch (op) {
      case U_NEG: v = -a; bv = ba; break;
      case U_ABS: v = fabs(a); bv = ba; break;
      case U_EXP:
        v = exp(a);
        bv = (ba == 0.0) ? 0.0 : v * expm1(ba);
        bv += local(cx, v, 4.0, 2.0);
        break;
      case U_LOG:
        v = log(a);
        if (ba == 0.0)
          bv = 0.0;
        else if (ba < fabs(a))
          bv = -log1p(-ba / fabs(a));
        else
          bv = INFINITY;
        bv += local(cx, v, 4.0, 2.0);
        break;
      case U_SQRT: {
        v = sqrt(a);
        if (ba == 0.0 || !(a >= 0.0))
          bv = 0.0;
        else {
          double up = ba / (sqrt(a + ba) + sqrt(a));
          double lo = (a - ba > 0.0) ? ba / (sqrt(a) + sqrt(a - ba)) : sqrt(a);
          bv = up > lo ? up : lo;
        }
        bv += local(cx, v, 4.0, 1.0);
        break;
      }
      case U_SQUARE:
        v = a * a;
        bv = mulb(2.0 * a, ba) + ba * ba + local(cx, v, 2.0, 1.0);
        break;
    }
    bv = finite_or_zero_bound(v, bv);
    clamp_to_range(cx, &v, &bv);
    out->v[t] = v;
    out->b[t] = bv;
  }
  return 0;
}

/* integer binary op with the INT32 tree semantics */
static int64_t ibin(int op, int64_t a, int64_t b, int* div0) {
  switch (op) {
    case B_PLUS: return wrap32(a + b);
    case B_MINUS: return wrap32(a - b);
    case B_SCHUR:
    case B_TIMES: return wrap32((int64_t)((uint64_t)a * (uint64_t)b));
    case B_DIV:
      if (b == 0) {
        *div0 = 1;
        return 0;
      }
      return wrap32(a / b); /* C99 division truncates toward zero */
  }
  return 0;
}

/* FP binary op: value and propagated bound */
static void fbin(ctx_t* cx, int op, double a, double ba, double b, double bb, double* v, double* bv) {
  double r = 0.0, e = 0.0;
  switch (op) {
    case B_PLUS:
      r = a + b;
      e = ba + bb;
      break;
    case B_MINUS:
      r = a - b;
      e = ba + bb;
      break;
    case B_SCHUR:
    case B_TIMES:
      r = a * b;
      e = mulb(a, bb) + mulb(b, ba) + ((ba == 0.0 || bb == 0.0) ? 0.0 : ba * bb);
      break;
    case B_DIV:
      r = a / b;
      if (ba == 0.0 && bb == 0.0)
        e = 0.0;
      else if (bb >= fabs(b))
        e = INFINITY;
      else
        e = (ba + mulb(r, bb)) / (fabs(b) - bb);
      break;
  }
  e += local(cx, r, 2.0, 1.0);
  e = finite_or_zero_bound(r, e);
  clamp_to_range(cx, &r, &e);
  *v = r;
  *bv = e;
}

static int binary(ctx_t* cx, int op, val_t* x, val_t* y, val_t* out) {
  int xs = x->kind == V_SCALAR, ys = y->kind == V_SCALAR;
  if (xs && ys) {
    snprintf(cx->err, 256, "operation between two scalars");
    return -1;
  }
  if (op == B_TIMES && !xs && !ys) {
    snprintf(cx->err, 256, "'*' of two matrices is matrix multiplication, not element-wise");
    return -1;
  }
  if (op == B_SCHUR && (xs || ys)) {
    snprintf(cx->err, 256, "'%%' needs two matrices");
    return -1;
  }
  if (!xs && !ys && (x->r != y->r || x->c != y->c)) {
    snprintf(cx->err, 256, "incompatible matrix dimensions: %lldx%lld and %lldx%lld", (long long)x->r,
             (long long)x->c, (long long)y->r, (long long)y->c);
    return -1;
  }
  val_t* m = xs ? y : x;
  if (val_alloc(cx, out, m->r, m->c)) return -1;
  int64_t n = m->r * m->c;
  int div0 = 0;
#pragma omp parallel for schedule(static) reduction(| : div0)
  for (int64_t t = 0; t < n; ++t) {
    if (cx->is_int) {
      int64_t a = xs ? (int64_t)x->k : x->iv[t];
      int64_t b = ys ? (int64_t)y->k : y->iv[t];
      out->iv[t] = ibin(op, a, b, &div0);
    } else {
      double a = xs ? x->k : x->v[t], ba = xs ? 0.0 : x->b[t];
      double b = ys ? y->k : y->v[t], bb = ys ? 0.0 : y->b[t];
      fbin(cx, op, a, ba, b, bb, &out->v[t], &out->b[t]);
    }
  }
  if (div0) cx->div0 = 1;
  return 0;
}

static int submat(ctx_t* cx, val_t* x, int64_t r0, int64_t c0, int64_t nr, int64_t nc, val_t* out) {
  if (x->kind != V_MAT || r0 < 0 || c0 < 0 || nr < 0 || nc < 0 || r0 + nr > x->r || c0 + nc > x->c) {
    snprintf(cx->err, 256, "submat: view out of bounds");
    return -1;
  }
  if (val_alloc(cx, out, nr, nc)) return -1;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t j = 0; j < nc; ++j)
    for (int64_t i = 0; i < nr; ++i) {
      /* submat(i,j) = X(r0+i, c0+j) */
      int64_t s = (r0 + i) + (c0 + j) * x->r, d = i + j * nr;
      if (cx->is_int)
        out->iv[d] = x->iv[s];
      else {
        out->v[d] = x->v[s];
        out->b[d] = x->b[s];
      }
    }
  return 0;
}

/* Matrix product x * y (Armadillo's operator* between matrices; Sec. 3 maps
 * trans(X)*Y onto one GEMM call with a transposed operand).  Each output is
 * the exact dot product rounded once to double (double-double sums of the
 * products, each product exact in double-double via fma).  Bound: the
 * operands' bounds propagated (sum of |x_ik| b(y_kj) + |y_kj| b(x_ik) + their
 * product) plus k u sum |x_ik y_kj|, u the compute type's unit roundoff --
 * the error bound of a k-term dot product in the compute type in any order of
 * additions, products rounded or exact.  Floating point only. */
static int matmul(ctx_t* cx, val_t* x, val_t* y, val_t* out) {
  if (x->kind != V_MAT || y->kind != V_MAT || x->c != y->r) {
    snprintf(cx->err, 256, "mm: incompatible matrix dimensions");
    return -1;
  }
  if (cx->is_int) {
    snprintf(cx->err, 256, "mm is not defined for INT32 trees here");
    return -1;
  }
  const int64_t m = x->r, k = x->c, n = y->c;
  if (val_alloc(cx, out, m, n)) return -1;
  const double u = (cx->ct == ORC_F64) ? ldexp(1.0, -53) : ldexp(1.0, -24);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      double sh = 0.0, sl = 0.0, asum = 0.0, bsum = 0.0;
      for (int64_t t = 0; t < k; ++t) {
        const double a = x->v[i + t * m], b = y->v[t + j * k];
        const double p = a * b, pe = fma(a, b, -p);
        const double s2 = sh + p, bp = s2 - sh;
        sl += (sh - (s2 - bp)) + (p - bp) + pe;
        sh = s2;
        asum += fabs(p);
        bsum += fabs(a) * y->b[t + j * k] + fabs(b) * x->b[i + t * m] + x->b[i + t * m] * y->b[t + j * k];
      }
      double v = sh + sl;
      double b = bsum + (double)k * u * asum + orc_ulp(v, ORC_F64);
      clamp_to_range(cx, &v, &b);
      out->v[i + j * m] = v;
      out->b[i + j * m] = finite_or_zero_bound(v, b);
    }
  return 0;
}

/* Broadcasting (Armadillo's each_col / each_row operands) and diagonal
 * views (X.diag(k)), Sec. 2: each element of the result is one element of x.
 *   each_col:n  x is r x 1, result r x n, result(i,j) = x(i,0)
 *   each_row:n  x is 1 x c, result n x c, result(i,j) = x(0,j)
 *   diag:k      result(i,0) = x(i + max(-k,0), i + max(k,0)), as many rows as
 *               the k-th diagonal has elements                              */
enum { G_EACH_COL, G_EACH_ROW, G_DIAG };

static int broadcast_or_diag(ctx_t* cx, int op, int64_t arg, val_t* x, val_t* out) {
  int64_t r = 0, c = 0;
  if (x->kind != V_MAT) {
    snprintf(cx->err, 256, "each_col/each_row/diag need a matrix");
    return -1;
  }
  if (op == G_EACH_COL) {
    if (x->c != 1 || arg < 0) {
      snprintf(cx->err, 256, "each_col repeats a column vector");
      return -1;
    }
    r = x->r;
    c = arg;
  } else if (op == G_EACH_ROW) {
    if (x->r != 1 || arg < 0) {
      snprintf(cx->err, 256, "each_row repeats a row vector");
      return -1;
    }
    r = arg;
    c = x->c;
  } else {
    if ((arg > 0 && arg >= x->c) || (arg < 0 && -arg >= x->r)) {
      snprintf(cx->err, 256, "diag: diagonal outside the matrix");
      return -1;
    }
    const int64_t len = (arg >= 0) ? (x->r < x->c - arg ? x->r : x->c - arg) : (x->r + arg < x->c ? x->r + arg : x->c);
    r = len > 0 ? len : 0;
    c = 1;
  }
  if (val_alloc(cx, out, r, c)) return -1;
  const int64_t kr = arg < 0 ? -arg : 0, kc = arg > 0 ? arg : 0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t j = 0; j < c; ++j)
    for (int64_t i = 0; i < r; ++i) {
      int64_t src;
      if (op == G_EACH_COL)
        src = i;
      else if (op == G_EACH_ROW)
        src = j * x->r;
      else
        src = (i + kr) + (i + kc) * x->r;
      const int64_t d = i + j * r;
      if (cx->is_int)
        out->iv[d] = x->iv[src];
      else {
        out->v[d] = x->v[src];
        out->b[d] = x->b[src];
      }
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* reductions                                                          */
/* ------------------------------------------------------------------ */

enum { R_ACCU, R_SUM0, R_SUM1, R_MEAN, R_MEAN0, R_MEAN1, R_DOT, R_NORM, R_NORMFRO, R_VAR0, R_VAR1 };

static int alloc_result(orc_result* res, int is_int, int64_t r, int64_t c) {
  size_t n = (size_t)(r * c);
  size_t nn = n ? n : 1;
  res->n_rows = r;
  res->n_cols = c;
  if (is_int) {
    res->iv = (int64_t*)calloc(nn, sizeof(int64_t));
    return res->iv ? 0 : -1;
  }
  res->v = (double*)calloc(nn, sizeof(double));
  res->b = (double*)calloc(nn, sizeof(double));
  return (res->v && res->b) ? 0 : -1;
}

/* sum of a strided selection: elements x[off + t*stride], t < n */
static void gather(const double* x, int64_t off, int64_t stride, int64_t n, double* buf) {
  for (int64_t t = 0; t < n; ++t) buf[t] = x[off + t * stride];
}

static int reduce(ctx_t* cx, int kind, val_t* x, val_t* y, orc_result* res) {
  int64_t r = x->r, c = x->c, n = r * c;
  if (cx->is_int && (kind == R_MEAN || kind == R_MEAN0 || kind == R_MEAN1 || kind == R_NORM ||
                     kind == R_NORMFRO || kind == R_VAR0 || kind == R_VAR1)) {
    snprintf(cx->err, 256, "mean/norm/var are not defined for INT32 trees");
    return -1;
  }
  if (kind == R_NORM && r != 1 && c != 1) {
    snprintf(cx->err, 256, "norm: the 2-norm is defined here for vectors only; use norm:fro");
    return -1;
  }
  res->is_reduction = 1;
  if (kind == R_SUM0 || kind == R_MEAN0 || kind == R_SUM1 || kind == R_MEAN1) {
    int by_col = (kind == R_SUM0 || kind == R_MEAN0);
    int64_t nout = by_col ? c : r, len = by_col ? r : c;
    if (alloc_result(res, cx->is_int, by_col ? 1 : r, by_col ? c : 1)) return -1;
    if (cx->is_int) {
      for (int64_t o = 0; o < nout; ++o) {
        uint64_t s = 0;
        for (int64_t t = 0; t < len; ++t) s += (uint64_t)x->iv[by_col ? (t + o * r) : (o + t * r)];
        res->iv[o] = (int64_t)s;
      }
      return 0;
    }
    double* buf = (double*)malloc((size_t)(len ? len : 1) * sizeof(double));
    double* bbuf = (double*)malloc((size_t)(len ? len : 1) * sizeof(double));
    if (!buf || !bbuf) return -1;
    for (int64_t o = 0; o < nout; ++o) {
      gather(x->v, by_col ? o * r : o, by_col ? 1 : r, len, buf);
      gather(x->b, by_col ? o * r : o, by_col ? 1 : r, len, bbuf);
      double s = orc_sum_neumaier(buf, len), e = sum_plain(bbuf, len);
      if (kind == R_MEAN0 || kind == R_MEAN1) {
        s = s / (double)len;
        e = e / (double)len;
      }
      res->v[o] = s;
      res->b[o] = finite_or_zero_bound(s, e);
    }
    free(buf);
    free(bbuf);
    return 0;
  }
  if (alloc_result(res, cx->is_int, 1, 1)) return -1;
  if (cx->is_int) {
    uint64_t s = 0;
    if (kind == R_DOT) {
      for (int64_t t = 0; t < n; ++t) s += (uint64_t)(x->iv[t] * y->iv[t]);
    } else {
      for (int64_t t = 0; t < n; ++t) s += (uint64_t)x->iv[t];
    }
    res->iv[0] = (int64_t)s;
    return 0;
  }
  double* buf = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
  double* bbuf = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
  if (!buf || !bbuf) return -1;
  double s = 0.0, e = 0.0;
  switch (kind) {
    case R_ACCU:
    case R_MEAN:
      s = orc_sum_neumaier(x->v, n);
      e = sum_plain(x->b, n);
      if (kind == R_MEAN) {
        s /= (double)n; /* empty: 0/0 = NaN */
        e /= (double)n;
      }
      break;
    case R_DOT:
      for (int64_t t = 0; t < n; ++t) {
        buf[t] = x->v[t] * y->v[t];
        bbuf[t] = mulb(x->v[t], y->b[t]) + mulb(y->v[t], x->b[t]);
      }
      s = orc_sum_neumaier(buf, n);
      e = sum_plain(bbuf, n);
      break;
    case R_NORM:
    case R_NORMFRO: {
      for (int64_t t = 0; t < n; ++t) {
        buf[t] = x->v[t] * x->v[t];
        bbuf[t] = mulb(2.0 * x->v[t], x->b[t]);
      }
      double ss = orc_sum_neumaier(buf, n), es = sum_plain(bbuf, n);
      s = sqrt(ss);
      e = (es == 0.0) ? 0.0 : (s > 0.0 ? es / (2.0 * s) : sqrt(es));
      break;
    }
    case R_VAR0:
    case R_VAR1: {
      if (n == 0) {
        s = NAN;
        break;
      }
      if (n == 1) {
        s = 0.0;
        break;
      }
      /* pass 1: mean; pass 2: centred sum of squares */
      double mu = orc_sum_neumaier(x->v, n) / (double)n;
      for (int64_t t = 0; t < n; ++t) {
        double d = x->v[t] - mu;
        buf[t] = d * d;
        bbuf[t] = mulb(2.0 * d, x->b[t]);
      }
      double den = (kind == R_VAR0) ? (double)(n - 1) : (double)n;
      s = orc_sum_neumaier(buf, n) / den;
      e = sum_plain(bbuf, n) / den;
      break;
    }
  }
  free(buf);
  free(bbuf);
  res->v[0] = s;
  res->b[0] = finite_or_zero_bound(s, e);
  return 0;
}

/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* cumsum: prefix sums along a dimension (Armadillo's cumsum, Sec. 2)  */
/* ------------------------------------------------------------------ */
/*
 * dim 0 runs down each column, dim 1 along each row; dim -1 is Armadillo's
 * default: along the vector for a row or column vector, else dim 0.  The
 * value is the exact prefix sum (double-double running sum, rounded once to
 * double).  Bound of output k of a line: the sum of the element bounds plus
 * (k-1) u |y_1| + ... + |y_k| with u the compute type's unit roundoff -- the
 * error bound of a sum of k terms in the compute type in any order of
 * additions -- so that an FP32 prefix sum computed any way passes.  An
 * FP32 prefix beyond the format's range is +-inf.  INT32 trees wrap modulo
 * 2^32 like every INT32 node.
 */
static int cumsum(ctx_t* cx, int dim, val_t* x, val_t* out) {
  const int64_t r = x->r, c = x->c;
  if (dim < 0) dim = (r == 1) ? 1 : 0; /* a row vector runs along dim 1 */
  if (val_alloc(cx, out, r, c)) return -1;
  const int64_t nline = (dim == 0) ? c : r, len = (dim == 0) ? r : c;
  const double u = (cx->ct == ORC_F64) ? ldexp(1.0, -53) : ldexp(1.0, -24);
  for (int64_t o = 0; o < nline; ++o) {
    double sh = 0.0, sl = 0.0, plain = 0.0, asum = 0.0, bsum = 0.0;
    int64_t isum = 0;
    int special = 0;
    for (int64_t t = 0; t < len; ++t) {
      const int64_t q = (dim == 0) ? t + o * r : o + t * r;
      if (cx->is_int) {
        isum = (int64_t)((uint64_t)isum + (uint64_t)x->iv[q]);
        out->iv[q] = wrap32(isum);
        continue;
      }
      const double y = x->v[q];
      plain += y;
      if (!isfinite(y)) special = 1;
      /* TwoSum of the running high part and y, error into the low part */
      const double s2 = sh + y;
      const double bp = s2 - sh;
      const double e = (sh - (s2 - bp)) + (y - bp);
      sh = s2;
      sl += e;
      asum += fabs(y);
      bsum += x->b[q];
      double v = special ? plain : sh + sl;
      double b = special ? 0.0 : bsum + (double)t * u * asum + orc_ulp(v, ORC_F64);
      clamp_to_range(cx, &v, &b);
      out->v[q] = v;
      out->b[q] = finite_or_zero_bound(v, b);
    }
  }
  return 0;
}

/* statistics along a dimension: min, max, index_min, index_max, prod, */
/* var, stddev (Armadillo's statistics functions, Sec. 2)               */
/* ------------------------------------------------------------------ */
/*
 * dim -1 reduces all elements (index outputs are column-major linear
 * indices), dim 0 each column (index outputs are row indices), dim 1 each
 * row (index outputs are column indices).  Readings: NaN elements are passed
 * over by min/max and their indices; ties give the first occurrence; an empty
 * set gives NaN (0 for INT32 trees) and index -1.  prod is the exact product
 * rounded once to the result type (double-double significands with the
 * exponent carried apart, error ~ n u^2 before that rounding; an empty
 * product is 1); INT32 trees multiply modulo 2^64.  var/stddev are the
 * two-pass definitions of the all-element form.
 */
enum { S_MIN, S_MAX, S_IMIN, S_IMAX, S_PROD, S_VAR, S_STD };

static int reduce_stat(ctx_t* cx, int op, int dim, int norm, val_t* x, orc_result* res) {
  const int64_t r = x->r, c = x->c;
  const int64_t nout = (dim == -1) ? 1 : (dim == 0 ? c : r);
  const int64_t len = (dim == -1) ? r * c : (dim == 0 ? r : c);
  const int idx_out = (op == S_IMIN || op == S_IMAX);
  if (cx->is_int && (op == S_VAR || op == S_STD)) {
    snprintf(cx->err, 256, "var/stddev are not defined for INT32 trees");
    return -1;
  }
  const int out_int = cx->is_int || idx_out;
  res->is_reduction = 1;
  if (alloc_result(res, out_int, dim == 1 ? r : 1, dim == 0 ? c : 1)) return -1;
  res->is_int = out_int;
  double* buf = (double*)malloc((size_t)(len ? len : 1) * sizeof(double));
  if (!buf) return -1;
  for (int64_t o = 0; o < nout; ++o) {
    /* element t of output o sits at column-major position q(t) */
#define QPOS(t) ((dim == -1) ? (t) : (dim == 0 ? (t) + o * r : o + (t) * r))
    if (op == S_MIN || op == S_MAX || op == S_IMIN || op == S_IMAX) {
      const int want_min = (op == S_MIN || op == S_IMIN);
      int64_t best = -1;
      double bv = 0.0, bmax = 0.0;
      int64_t biv = 0;
      for (int64_t t = 0; t < len; ++t) {
        const int64_t q = QPOS(t);
        if (cx->is_int) {
          const int64_t v = x->iv[q];
          if (best < 0 || (want_min ? v < biv : v > biv)) {
            best = t;
            biv = v;
          }
        } else {
          const double v = x->v[q];
          if (isnan(v)) continue;
          if (x->b[q] > bmax) bmax = x->b[q];
          if (best < 0 || (want_min ? v < bv : v > bv)) {
            best = t;
            bv = v;
          }
        }
      }
      if (idx_out) {
        res->iv[o] = (best < 0) ? -1 : ((dim == -1) ? QPOS(best) : best);
      } else if (cx->is_int) {
        res->iv[o] = (best < 0) ? 0 : biv;
      } else {
        res->v[o] = (best < 0) ? NAN : bv;
        /* any element may become the extreme within its own bound */
        res->b[o] = (best < 0) ? 0.0 : finite_or_zero_bound(bv, bmax);
      }
    } else if (op == S_PROD) {
      if (cx->is_int) {
        uint64_t p = 1;
        for (int64_t t = 0; t < len; ++t) p *= (uint64_t)x->iv[QPOS(t)];
        res->iv[o] = (int64_t)p;
      } else {
        /* v = m 2^k with 0.5 <= |m| < 1 (frexp): the significands multiply in
         * double-double, the exponents add apart, so no partial product
         * overflows or underflows; zeros, infinities and NaN follow IEEE
         * multiplication; the exact product is rounded once at the end */
        double ph = 1.0, pl = 0.0, rel = 0.0;
        long long E = 0;
        int zero = 0, inf = 0, nan = 0, neg = 0;
        for (int64_t t = 0; t < len; ++t) {
          const int64_t q = QPOS(t);
          const double v = x->v[q];
          if (signbit(v)) neg ^= 1;
          if (isnan(v)) { nan = 1; continue; }
          if (isinf(v)) { inf = 1; continue; }
          if (v == 0.0) { zero = 1; continue; }
          if (x->b[q] != 0.0) rel += x->b[q] / fabs(v);
          int k;
          const double m = fabs(frexp(v, &k));
          E += k;
          const double p = ph * m;
          const double e = fma(ph, m, -p); /* exact error of ph*m */
          pl = fma(pl, m, e);
          ph = p;
          ph = frexp(ph, &k); /* back to [0.5, 1) */
          pl = ldexp(pl, -k);
          E += k;
        }
        double pv;
        if (nan || (inf && zero))
          pv = NAN;
        else if (inf)
          pv = neg ? -INFINITY : INFINITY;
        else if (zero)
          pv = neg ? -0.0 : 0.0;
        else {
          const double mag = (E > 4000) ? INFINITY : (E < -4000 ? 0.0 : ldexp(ph + pl, (int)E));
          pv = neg ? -mag : mag;
        }
        /* the result has the accumulation type: FP32 trees round to float */
        if (cx->ct == ORC_F32) pv = (double)(float)pv;
        res->v[o] = pv;
        res->b[o] = (zero || inf || nan) ? 0.0 : finite_or_zero_bound(pv, fabs(pv) * rel);
      }
    } else { /* S_VAR, S_STD */
      double s2, e2;
      if (len == 0) {
        s2 = NAN;
        e2 = 0.0;
      } else if (len == 1) {
        s2 = 0.0;
        e2 = 0.0;
      } else {
        for (int64_t t = 0; t < len; ++t) buf[t] = x->v[QPOS(t)];
        const double mu = orc_sum_neumaier(buf, len) / (double)len;
        double eb = 0.0;
        for (int64_t t = 0; t < len; ++t) {
          const double d = buf[t] - mu;
          eb += mulb(2.0 * d, x->b[QPOS(t)]);
          buf[t] = d * d;
        }
        const double den = (norm == 0) ? (double)(len - 1) : (double)len;
        s2 = orc_sum_neumaier(buf, len) / den;
        e2 = eb / den;
      }
      if (op == S_VAR) {
        res->v[o] = s2;
        res->b[o] = finite_or_zero_bound(s2, e2);
      } else {
        const double sd = sqrt(s2);
        res->v[o] = sd;
        res->b[o] = finite_or_zero_bound(sd, e2 == 0.0 ? 0.0 : (sd > 0.0 ? e2 / (2.0 * sd) : sqrt(e2)));
      }
    }
#undef QPOS
  }
  free(buf);
  return 0;
}

/* token -> (op, dim, norm) for reduce_stat; returns 0 if not a statistic */
static int parse_stat(const char* tok, int* op, int* dim, int* norm) {
  static const struct { const char* name; int op; } names[] = {
      {"min", S_MIN}, {"max", S_MAX}, {"index_min", S_IMIN}, {"index_max", S_IMAX}, {"prod", S_PROD}};
  *dim = -1;
  *norm = 0;
  for (size_t i = 0; i < sizeof names / sizeof names[0]; ++i) {
    size_t n = strlen(names[i].name);
    if (!strncmp(tok, names[i].name, n) && (tok[n] == 0 || (tok[n] == ':' && (tok[n + 1] == '0' || tok[n + 1] == '1') &&
                                                              tok[n + 2] == 0))) {
      *op = names[i].op;
      if (tok[n] == ':') *dim = tok[n + 1] - '0';
      return 1;
    }
  }
  if (!strcmp(tok, "stddev") || !strcmp(tok, "stddev:1")) {
    *op = S_STD;
    *norm = tok[6] == ':' ? 1 : 0;
    return 1;
  }
  int d, nt;
  char tail;
  if (sscanf(tok, "vardim:%d:%d%c", &d, &nt, &tail) == 2 && (d == 0 || d == 1) && (nt == 0 || nt == 1)) {
    *op = S_VAR;
    *dim = d;
    *norm = nt;
    return 1;
  }
  if (sscanf(tok, "stddevdim:%d:%d%c", &d, &nt, &tail) == 2 && (d == 0 || d == 1) && (nt == 0 || nt == 1)) {
    *op = S_STD;
    *dim = d;
    *norm = nt;
    return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* program walker                                                      */
/* ------------------------------------------------------------------ */

#define MAX_STACK 64

static double to_elem_type(ctx_t* cx, double k, int* ok) {
  *ok = 1;
  if (cx->is_int) {
    if (!isfinite(k) || k <= -2147483649.0 || k >= 2147483648.0) {
      *ok = 0;
      return 0;
    }
    return (double)(int32_t)k; /* truncation toward zero */
  }
  if (cx->ct == ORC_F32) return (double)(float)k;
  return k;
}

int orc_eval(const char* program, const orc_mat* leaves, int32_t n_leaves, int32_t out_dtype,
             orc_result* res) {
  memset(res, 0, sizeof *res);
  if (n_leaves < 1) {
    snprintf(res->err, sizeof res->err, "no leaves");
    return -1;
  }
  int dt = leaves[0].dtype;
  for (int i = 1; i < n_leaves; ++i)
    if (leaves[i].dtype != dt) {
      snprintf(res->err, sizeof res->err, "all leaves must share one dtype");
      return -1;
    }
  ctx_t cx;
  cx.is_int = (dt == ORC_I32);
  cx.ct = cx.is_int ? ORC_I32 : (dt == ORC_F64 ? ORC_F64 : ORC_F32);
  cx.div0 = 0;
  cx.err = res->err;
  if (out_dtype < 0) out_dtype = dt;
  res->is_int = cx.is_int;

  val_t st[MAX_STACK];
  int sp = 0, rc = -1, reduced = 0, scanned = 0;
  size_t plen = strlen(program);
  char* buf = (char*)malloc(plen + 1);
  memcpy(buf, program, plen + 1);
  char* save = NULL;
  for (char* tok = strtok_r(buf, " \t\n", &save); tok; tok = strtok_r(NULL, " \t\n", &save)) {
    if (reduced || scanned) {
      snprintf(res->err, sizeof res->err, "tokens after the reduction");
      goto done;
    }
    if (sp >= MAX_STACK - 1) {
      snprintf(res->err, sizeof res->err, "stack overflow");
      goto done;
    }
    if (tok[0] >= 'A' && tok[0] <= 'H' && tok[1] == 0) {
      int li = tok[0] - 'A';
      if (li >= n_leaves) {
        snprintf(res->err, sizeof res->err, "leaf %c not given", tok[0]);
        goto done;
      }
      if (load_leaf(&cx, &leaves[li], &st[sp])) goto done;
      sp++;
      continue;
    }
    if (tok[0] == '#') {
      int ok;
      char* end;
      double k = strtod(tok + 1, &end);
      if (*end) {
        snprintf(res->err, sizeof res->err, "bad scalar '%s'", tok);
        goto done;
      }
      memset(&st[sp], 0, sizeof st[sp]);
      st[sp].kind = V_SCALAR;
      st[sp].k = to_elem_type(&cx, k, &ok);
      if (!ok) {
        snprintf(res->err, sizeof res->err, "scalar %g does not fit INT32", k);
        goto done;
      }
      sp++;
      continue;
    }
    int bop = -1, uop = -1, rop = -1;
    if (!strcmp(tok, "+")) bop = B_PLUS;
    else if (!strcmp(tok, "-")) bop = B_MINUS;
    else if (!strcmp(tok, "%")) bop = B_SCHUR;
    else if (!strcmp(tok, "/")) bop = B_DIV;
    else if (!strcmp(tok, "*")) bop = B_TIMES;
    else if (!strcmp(tok, "neg")) uop = U_NEG;
    else if (!strcmp(tok, "exp")) uop = U_EXP;
    else if (!strcmp(tok, "log")) uop = U_LOG;
    else if (!strcmp(tok, "abs")) uop = U_ABS;
    else if (!strcmp(tok, "square")) uop = U_SQUARE;
    else if (!strcmp(tok, "sqrt")) uop = U_SQRT;
    else if (!strcmp(tok, "trans")) uop = U_TRANS;
    else if (!strcmp(tok, "accu")) rop = R_ACCU;
    else if (!strcmp(tok, "sum:0")) rop = R_SUM0;
    else if (!strcmp(tok, "sum:1")) rop = R_SUM1;
    else if (!strcmp(tok, "mean")) rop = R_MEAN;
    else if (!strcmp(tok, "mean:0")) rop = R_MEAN0;
    else if (!strcmp(tok, "mean:1")) rop = R_MEAN1;
    else if (!strcmp(tok, "dot")) rop = R_DOT;
    else if (!strcmp(tok, "norm")) rop = R_NORM;
    else if (!strcmp(tok, "norm:fro")) rop = R_NORMFRO;
    else if (!strcmp(tok, "var") || !strcmp(tok, "var:0")) rop = R_VAR0;
    else if (!strcmp(tok, "var:1")) rop = R_VAR1;

    if (!strcmp(tok, "cumsum") || !strcmp(tok, "cumsum:0") || !strcmp(tok, "cumsum:1")) {
      if (sp != 1 || st[0].kind != V_MAT) {
        snprintf(res->err, sizeof res->err, "cumsum needs exactly one matrix operand");
        goto done;
      }
      val_t out;
      if (cumsum(&cx, tok[6] == ':' ? tok[7] - '0' : -1, &st[0], &out)) goto done;
      val_free(&st[0]);
      st[0] = out;
      scanned = 1;
      continue;
    }
    int sop, sdim, snorm;
    if (rop < 0 && parse_stat(tok, &sop, &sdim, &snorm)) {
      if (sp != 1 || st[0].kind != V_MAT) {
        snprintf(res->err, sizeof res->err, "statistic '%s' needs exactly one matrix operand", tok);
        goto done;
      }
      if (reduce_stat(&cx, sop, sdim, snorm, &st[0], res)) goto done;
      reduced = 1;
      continue;
    }
    {
      long long garg = 0;
      int gop = -1;
      if (!strcmp(tok, "mm")) {
        if (sp < 2) goto underflow;
        val_t out;
        if (matmul(&cx, &st[sp - 2], &st[sp - 1], &out)) goto done;
        val_free(&st[sp - 2]);
        val_free(&st[sp - 1]);
        st[sp - 2] = out;
        sp--;
        continue;
      }
      if (!strncmp(tok, "each_col:", 9) && sscanf(tok + 9, "%lld", &garg) == 1) gop = G_EACH_COL;
      else if (!strncmp(tok, "each_row:", 9) && sscanf(tok + 9, "%lld", &garg) == 1) gop = G_EACH_ROW;
      else if (!strcmp(tok, "diag")) gop = G_DIAG;
      else if (!strncmp(tok, "diag:", 5) && sscanf(tok + 5, "%lld", &garg) == 1) gop = G_DIAG;
      if (gop >= 0) {
        if (sp < 1) goto underflow;
        val_t out;
        if (broadcast_or_diag(&cx, gop, garg, &st[sp - 1], &out)) goto done;
        val_free(&st[sp - 1]);
        st[sp - 1] = out;
        continue;
      }
    }
    if (!strncmp(tok, "submat:", 7)) {
      long long r0, c0, nr, nc;
      if (sscanf(tok + 7, "%lld:%lld:%lld:%lld", &r0, &c0, &nr, &nc) != 4) {
        snprintf(res->err, sizeof res->err, "bad submat token '%s'", tok);
        goto done;
      }
      if (sp < 1) goto underflow;
      val_t out;
      if (submat(&cx, &st[sp - 1], r0, c0, nr, nc, &out)) goto done;
      val_free(&st[sp - 1]);
      st[sp - 1] = out;
    } else if (bop >= 0) {
      if (sp < 2) goto underflow;
      val_t out;
      if (binary(&cx, bop, &st[sp - 2], &st[sp - 1], &out)) goto done;
      val_free(&st[sp - 2]);
      val_free(&st[sp - 1]);
      st[sp - 2] = out;
      sp--;
    } else if (uop >= 0) {
      if (sp < 1) goto underflow;
      if (st[sp - 1].kind != V_MAT) {
        snprintf(res->err, sizeof res->err, "'%s' needs a matrix", tok);
        goto done;
      }
      val_t out;
      if (unary(&cx, uop, &st[sp - 1], &out)) goto done;
      val_free(&st[sp - 1]);
      st[sp - 1] = out;
    } else if (rop >= 0) {
      int need = (rop == R_DOT) ? 2 : 1;
      if (sp != need) {
        snprintf(res->err, sizeof res->err, "reduction '%s' needs exactly %d matrix operand(s) on the stack",
                 tok, need);
        goto done;
      }
      for (int q = 0; q < need; ++q)
        if (st[q].kind != V_MAT) {
          snprintf(res->err, sizeof res->err, "reduction of a scalar");
          goto done;
        }
      if (rop == R_DOT && (st[0].r * st[0].c != st[1].r * st[1].c)) {
        snprintf(res->err, sizeof res->err, "dot: operands differ in number of elements");
        goto done;
      }
      if (rop == R_DOT && (st[0].r != st[1].r || st[0].c != st[1].c)) {
        snprintf(res->err, sizeof res->err, "dot: incompatible matrix dimensions");
        goto done;
      }
      if (reduce(&cx, rop, &st[0], need == 2 ? &st[1] : NULL, res)) goto done;
      reduced = 1;
    } else {
      snprintf(res->err, sizeof res->err, "unknown token '%s'", tok);
      goto done;
    }
    continue;
  underflow:
    snprintf(res->err, sizeof res->err, "stack underflow at '%s'", tok);
    goto done;
  }
  if (!reduced) {
    if (sp != 1 || st[0].kind != V_MAT) {
      snprintf(res->err, sizeof res->err, "program must leave exactly one matrix");
      goto done;
    }
    res->is_reduction = 0;
    res->n_rows = st[0].r;
    res->n_cols = st[0].c;
    if (cx.is_int) {
      res->iv = st[0].iv;
      st[0].iv = NULL;
    } else {
      int64_t n = st[0].r * st[0].c;
      /* the stored result is rounded once more when it is narrower than
       * the compute type */
      if (out_dtype == ORC_BF16 || out_dtype == ORC_F16)
        for (int64_t t = 0; t < n; ++t)
          if (isfinite(st[0].v[t])) {
            if (fabs(st[0].v[t]) >= overflow_threshold(out_dtype)) {
              st[0].v[t] = copysign(INFINITY, st[0].v[t]); /* storage overflow */
              st[0].b[t] = 0.0;
            } else {
              st[0].b[t] += 0.5 * orc_ulp(fabs(st[0].v[t]) + st[0].b[t], out_dtype);
            }
          }
      res->v = st[0].v;
      res->b = st[0].b;
      st[0].v = st[0].b = NULL;
    }
  }
  rc = 0;
done:
  for (int i = 0; i < sp; ++i) val_free(&st[i]);
  free(buf);
  res->div_by_zero = cx.div0;
  if (rc) {
    free(res->v);
    free(res->b);
    free(res->iv);
    res->v = res->b = NULL;
    res->iv = NULL;
  }
  return rc;
}

void orc_free(orc_result* res) {
  free(res->v);
  free(res->b);
  free(res->iv);
  res->v = res->b = NULL;
  res->iv = NULL;
}

/* ------------------------------------------------------------------ */
/* gradient of a scalar loss (reverse mode over the materialised tape)  */
/* ------------------------------------------------------------------ */
/*
 * For L = red(tree) with red accu / sum (all elements) / mean, the gradient
 * with respect to each leaf is the plain chain rule: every node's adjoint
 * matrix is the sum over its consumers of the consumer's adjoint times the
 * local derivative, starting from dL/d(root) = 1 (accu) or 1/N (mean).  A
 * second sweep over magnitudes -- node values formed with absolute values
 * throughout, |a| + |b| for a +- b and |a||b| for a*b, and the local
 * derivatives taken from those magnitudes -- gives the scale of every
 * rounding a device makes in the forward and the reverse sweep, against which
 * the device gradient is bounded (a running error bound).
 */
typedef struct {
  int kind;    /* 0 leaf, 1 scalar, 2 unary, 3 binary, 4 submat */
  int op;      /* U_* / B_* */
  int a, b;    /* operand tape indices */
  int leaf;
  int64_t r0, c0;
  val_t v;     /* forward value (materialised) */
} tape_t;

int orc_grad(const char* program, const orc_mat* leaves, int32_t n_leaves, double** grads, double** absgrads,
             double* loss, char* err) {
  err[0] = 0;
  int dt = leaves[0].dtype;
  for (int i = 1; i < n_leaves; ++i)
    if (leaves[i].dtype != dt) {
      snprintf(err, 256, "all leaves must share one dtype");
      return -1;
    }
  if (dt == ORC_I32) {
    snprintf(err, 256, "gradients are defined for floating trees only");
    return -1;
  }
  ctx_t cx;
  cx.is_int = 0;
  cx.ct = (dt == ORC_F64) ? ORC_F64 : ORC_F32;
  cx.div0 = 0;
  cx.err = err;
  tape_t tp[MAX_STACK];
  int nt = 0, st[MAX_STACK], sp = 0, rc = -1, red = -1;
  size_t plen = strlen(program);
  char* buf = (char*)malloc(plen + 1);
  memcpy(buf, program, plen + 1);
  char* save = NULL;
  for (char* tok = strtok_r(buf, " \t\n", &save); tok; tok = strtok_r(NULL, " \t\n", &save)) {
    if (red >= 0 || nt >= MAX_STACK - 1) {
      snprintf(err, 256, "malformed program");
      goto done;
    }
    tape_t* t = &tp[nt];
    memset(t, 0, sizeof *t);
    int uop = -1, bop = -1;
    if (tok[0] >= 'A' && tok[0] <= 'H' && tok[1] == 0) {
      t->kind = 0;
      t->leaf = tok[0] - 'A';
      if (t->leaf >= n_leaves) {
        snprintf(err, 256, "leaf %c not given", tok[0]);
        goto done;
      }
      if (load_leaf(&cx, &leaves[t->leaf], &t->v)) goto done;
      st[sp++] = nt++;
      continue;
    }
    if (tok[0] == '#') {
      int ok;
      t->kind = 1;
      t->v.kind = V_SCALAR;
      t->v.k = to_elem_type(&cx, strtod(tok + 1, NULL), &ok);
      st[sp++] = nt++;
      continue;
    }
    if (!strcmp(tok, "accu") || !strcmp(tok, "sum") || !strcmp(tok, "mean")) {
      if (sp != 1) {
        snprintf(err, 256, "reduction needs one operand");
        goto done;
      }
      red = !strcmp(tok, "mean") ? 1 : 0;
      continue;
    }
    if (!strncmp(tok, "submat:", 7)) {
      long long r0, c0, nr, nc;
      if (sp < 1 || sscanf(tok + 7, "%lld:%lld:%lld:%lld", &r0, &c0, &nr, &nc) != 4) {
        snprintf(err, 256, "bad submat");
        goto done;
      }
      t->kind = 4;
      t->a = st[sp - 1];
      t->r0 = r0;
      t->c0 = c0;
      if (submat(&cx, &tp[t->a].v, r0, c0, nr, nc, &t->v)) goto done;
      st[sp - 1] = nt++;
      continue;
    }
    if (!strcmp(tok, "+")) bop = B_PLUS;
    else if (!strcmp(tok, "-")) bop = B_MINUS;
    else if (!strcmp(tok, "%")) bop = B_SCHUR;
    else if (!strcmp(tok, "/")) bop = B_DIV;
    else if (!strcmp(tok, "*")) bop = B_TIMES;
    else if (!strcmp(tok, "neg")) uop = U_NEG;
    else if (!strcmp(tok, "exp")) uop = U_EXP;
    else if (!strcmp(tok, "log")) uop = U_LOG;
    else if (!strcmp(tok, "abs")) uop = U_ABS;
    else if (!strcmp(tok, "square")) uop = U_SQUARE;
    else if (!strcmp(tok, "sqrt")) uop = U_SQRT;
    else if (!strcmp(tok, "trans")) uop = U_TRANS;
    if (bop >= 0) {
      if (sp < 2) goto underflow;
      t->kind = 3;
      t->op = bop;
      t->a = st[sp - 2];
      t->b = st[sp - 1];
      if (binary(&cx, bop, &tp[t->a].v, &tp[t->b].v, &t->v)) goto done;
      st[sp - 2] = nt++;
      sp--;
    } else if (uop >= 0) {
      if (sp < 1) goto underflow;
      t->kind = 2;
      t->op = uop;
      t->a = st[sp - 1];
      if (tp[t->a].v.kind != V_MAT) {
        snprintf(err, 256, "unary op of a scalar");
        goto done;
      }
      if (unary(&cx, uop, &tp[t->a].v, &t->v)) goto done;
      st[sp - 1] = nt++;
    } else {
      snprintf(err, 256, "token '%s' not supported by the gradient", tok);
      goto done;
    }
    continue;
  underflow:
    snprintf(err, 256, "stack underflow at '%s'", tok);
    goto done;
  }
  if (red < 0 || sp != 1 || tp[st[0]].v.kind != V_MAT) {
    snprintf(err, 256, "the program must end with accu / sum / mean of a matrix");
    goto done;
  }
  {
    const int root = st[0];
    const int64_t N = tp[root].v.r * tp[root].v.c;
    *loss = orc_sum_neumaier(tp[root].v.v, N) / (red ? (double)N : 1.0);
    /* magnitudes of every node, evaluated with absolute values throughout
     * (|a| + |b| for a +- b, |a||b| for a*b, ...): the scale of the
     * rounding errors a device makes while forming that node */
    double** mag = (double**)calloc((size_t)nt, sizeof(double*));
    for (int i = 0; i < nt; ++i) {
      tape_t* t = &tp[i];
      if (t->v.kind != V_MAT) continue;
      const int64_t r = t->v.r, c = t->v.c, n = r * c;
      mag[i] = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
      for (int64_t j = 0; j < c; ++j)
        for (int64_t k = 0; k < r; ++k) {
          int64_t q = k + j * r;
          double m = fabs(t->v.v[q]);
          if (t->kind == 4) {
            m = mag[t->a][(t->r0 + k) + (t->c0 + j) * tp[t->a].v.r];
          } else if (t->kind == 2) {
            double ma = (t->op == U_TRANS) ? mag[t->a][j + k * tp[t->a].v.r] : mag[t->a][q];
            switch (t->op) {
              case U_NEG: case U_ABS: case U_TRANS: m = ma; break;
              case U_SQUARE: m = ma * ma; break;
              default: m = fabs(t->v.v[q]); break; /* exp, log, sqrt: their own value */
            }
          } else if (t->kind == 3) {
            val_t *x = &tp[t->a].v, *y = &tp[t->b].v;
            double ma = (x->kind == V_SCALAR) ? fabs(x->k) : mag[t->a][q];
            double mb = (y->kind == V_SCALAR) ? fabs(y->k) : mag[t->b][q];
            double b = (y->kind == V_SCALAR) ? y->k : y->v[q];
            switch (t->op) {
              case B_PLUS: case B_MINUS: m = ma + mb; break;
              case B_SCHUR: case B_TIMES: m = ma * mb; break;
              case B_DIV: m = ma / fabs(b); break;
            }
          }
          mag[i][q] = m;
        }
    }
    /* adjoints (value and magnitude sweep) per tape entry */
    double** adj = (double**)calloc((size_t)nt, sizeof(double*));
    double** aab = (double**)calloc((size_t)nt, sizeof(double*));
    for (int i = 0; i < nt; ++i)
      if (tp[i].v.kind == V_MAT) {
        size_t n = (size_t)(tp[i].v.r * tp[i].v.c);
        adj[i] = (double*)calloc(n ? n : 1, sizeof(double));
        aab[i] = (double*)calloc(n ? n : 1, sizeof(double));
      }
    for (int64_t q = 0; q < N; ++q) {
      adj[root][q] = red ? 1.0 / (double)N : 1.0;
      aab[root][q] = adj[root][q];
    }
    for (int li = 0; li < n_leaves; ++li) {
      size_t n = (size_t)(leaves[li].n_rows * leaves[li].n_cols);
      memset(grads[li], 0, n * sizeof(double));
      memset(absgrads[li], 0, n * sizeof(double));
    }
    for (int i = nt - 1; i >= 0; --i) {
      tape_t* t = &tp[i];
      if (t->v.kind != V_MAT) continue;
      const int64_t r = t->v.r, c = t->v.c, n = r * c;
      double *g = adj[i], *ga = aab[i];
      if (t->kind == 0) {
        /* a leaf occurrence: accumulate into the leaf's gradient */
        for (int64_t q = 0; q < n; ++q) {
          grads[t->leaf][q] += g[q];
          absgrads[t->leaf][q] += ga[q];
        }
      } else if (t->kind == 4) {
        val_t* x = &tp[t->a].v;
        for (int64_t j = 0; j < c; ++j)
          for (int64_t k = 0; k < r; ++k) {
            int64_t s = (t->r0 + k) + (t->c0 + j) * x->r;
            adj[t->a][s] += g[k + j * r];
            aab[t->a][s] += ga[k + j * r];
          }
      } else if (t->kind == 2) {
        val_t* x = &tp[t->a].v;
        for (int64_t j = 0; j < c; ++j)
          for (int64_t k = 0; k < r; ++k) {
            int64_t q = k + j * r;
            if (t->op == U_TRANS) {
              /* trans(X)(k,j) = X(j,k) */
              int64_t s = j + k * x->r;
              adj[t->a][s] += g[q];
              aab[t->a][s] += ga[q];
              continue;
            }
            double a = x->v[q], d = 0.0, dm;
            switch (t->op) {
              case U_NEG: d = -1.0; break;
              case U_EXP: d = exp(a); break;
              case U_LOG: d = 1.0 / a; break;
              case U_ABS: d = (a > 0) - (a < 0); break;
              case U_SQUARE: d = 2.0 * a; break;
              case U_SQRT: d = 0.5 / sqrt(a); break;
            }
            dm = (t->op == U_SQUARE) ? 2.0 * mag[t->a][q] : (t->op == U_ABS ? 1.0 : fabs(d));
            adj[t->a][q] += d * g[q];
            aab[t->a][q] += dm * ga[q];
          }
      } else if (t->kind == 3) {
        val_t *x = &tp[t->a].v, *y = &tp[t->b].v;
        int xs = x->kind == V_SCALAR, ys = y->kind == V_SCALAR;
        for (int64_t q = 0; q < n; ++q) {
          double a = xs ? x->k : x->v[q], b = ys ? y->k : y->v[q], da = 0.0, db = 0.0;
          double ma = xs ? fabs(x->k) : mag[t->a][q], mb = ys ? fabs(y->k) : mag[t->b][q];
          double dam = 1.0, dbm = 1.0;
          switch (t->op) {
            case B_PLUS: da = 1.0; db = 1.0; break;
            case B_MINUS: da = 1.0; db = -1.0; break;
            case B_SCHUR:
            case B_TIMES: da = b; db = a; dam = mb; dbm = ma; break;
            case B_DIV: da = 1.0 / b; db = -a / (b * b); dam = fabs(da); dbm = ma / (b * b); break;
          }
          if (!xs) {
            adj[t->a][q] += da * g[q];
            aab[t->a][q] += dam * ga[q];
          }
          if (!ys) {
            adj[t->b][q] += db * g[q];
            aab[t->b][q] += dbm * ga[q];
          }
        }
      }
    }
    for (int i = 0; i < nt; ++i) {
      free(adj[i]);
      free(aab[i]);
      free(mag[i]);
    }
    free(adj);
    free(aab);
    free(mag);
  }
  rc = 0;
done:
  for (int i = 0; i < nt; ++i) val_free(&tp[i].v);
  free(buf);
  return rc;
}
