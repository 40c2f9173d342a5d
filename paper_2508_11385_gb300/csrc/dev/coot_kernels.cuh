// coot_kernels.cuh -- kernel bodies instantiated per expression tree.
//
// Families (one generated __global__ wrapper per instantiation):
//   str   element-wise map over a column-major 2-D range without transposed
//         reads (a contiguous tree is walked as one long column), with an
//         optional full reduction; 128-bit vector loads/stores when every
//         read and the output are 16-byte aligned along columns.
//   col   the same map with a per-column reduction (sum/mean along dim 0):
//         a group of warps per column.
//   row   the same map with a per-row reduction (dim 1): a thread owns V
//         consecutive rows and walks a range of columns; column ranges are
//         combined by the last block of each row block.
//   tile  any tree with transposed reads: 32x32 output tiles, transposed
//         reads staged through a padded shared-memory tile so that both the
//         read and the write are coalesced; full, dim-0 and dim-1 reductions.
//   adj   fused adjoint of a scalar loss sum(tree): forward values are
//         recomputed per element and the reverse sweep writes every leaf's
//         gradient.
//   batch persistent kernel over many problems pulling chunks of 32x32 tiles
//         from a queue, with a per-problem reduction.
// Cross-block combines use a ticket counter: the block that arrives last
// combines the partials in a fixed order and resets the counter.  Nothing
// ever waits on another block.
#pragma once
#include "coot_params.h"
#include "coot_dev.cuh"

namespace coot {

// ld.global.cg: read a value another block wrote (at L2, not L1)
template <class A> __device__ __forceinline__ A load_cg(const A* p) {
  A r;
  const unsigned int* src = (const unsigned int*)p;
  unsigned int* dst = (unsigned int*)&r;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(A) / 4); ++i) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(dst[i]) : "l"(src + i));
  return r;
}

template <class S> __device__ __forceinline__ const S* at(const void* base, long long i, long long j, long long ld) {
  return (const S*)base + (i + j * ld);
}
template <class S> __device__ __forceinline__ S* at_out(void* base, long long i, long long j, long long ld) {
  return (S*)base + (i + j * ld);
}

// General slots and outputs.  A program defines COOT_GM: bit s (s < 8) marks
// slot s as general (rows not one element apart: a broadcast row vector, a
// diagonal, a row-strided view), bit 8 a general output (a diagonal).
// General reads and writes go one element at a time through the row stride;
// the others keep their vector accesses.  The slot index is a constant after
// unrolling, so the tests below fold away.
#ifndef COOT_GM
#define COOT_GM 0
#endif
constexpr int GM_OUT = 1 << COOT_MAX_SLOTS;
__device__ __forceinline__ constexpr bool gen_slot(int s) { return (COOT_GM >> s) & 1; }

// Bounds-check build: with COOT_DEBUG_BOUNDS defined, every slot read and
// every output write of the Params kernel families is checked against the
// extent the host computed from the leaf's (or output's) shape and strides;
// an access outside it is not made (a read gives 0) and sets device flag
// bit 2 (COOT_FLAG_OUT_OF_BOUNDS).  Without it the checks compile away.
#ifdef COOT_DEBUG_BOUNDS
template <class S> __device__ __forceinline__ bool slot_ok(const Params& p, int s, const S* ptr, long long n) {
  const long long off = ptr - (const S*)p.src[s];
  const bool ok = off >= 0 && off + n <= p.ext[s];
  if (!ok) atomicOr(p.err_flag, 4u);
  return ok;
}
template <class S> __device__ __forceinline__ bool out_ok(const Params& p, const S* ptr, long long n) {
  const long long off = ptr - (const S*)p.out;
  const bool ok = off >= 0 && off + n <= p.out_ext;
  if (!ok) atomicOr(p.err_flag, 4u);
  return ok;
}
#else
template <class S> __device__ __forceinline__ constexpr bool slot_ok(const Params&, int, const S*, long long) {
  return true;
}
template <class S> __device__ __forceinline__ constexpr bool out_ok(const Params&, const S*, long long) { return true; }
#endif
// one element of slot s / of the output, checked in the bounds-check build
template <class S> __device__ __forceinline__ typename IO<S>::C sload1(const Params& p, int s, const S* ptr) {
  return slot_ok<S>(p, s, ptr, 1) ? IO<S>::load1(ptr) : typename IO<S>::C(0);
}
template <class S> __device__ __forceinline__ void sstore1(const Params& p, S* ptr, typename IO<S>::C v) {
  if (out_ok<S>(p, ptr, 1)) IO<S>::store1(ptr, v);
}

template <class S> __device__ __forceinline__ const S* at_slot(const Params& p, int s, long long i, long long j) {
  if (gen_slot(s)) return (const S*)p.src[s] + (i * p.rs[s] + j * p.ld[s]);
  return at<S>(p.src[s], i, j, p.ld[s]);
}
// column j of slot s (row 0), and row i of a column of slot s
template <class S> __device__ __forceinline__ const S* col_of(const Params& p, int s, long long j) {
  return (const S*)p.src[s] + j * p.ld[s];
}
template <class S> __device__ __forceinline__ const S* row_in(const Params& p, int s, const S* col, long long i) {
  return gen_slot(s) ? col + i * p.rs[s] : col + i;
}
// V consecutive rows of slot s from row i of the column that starts at col,
// all inside the tree
template <class S, int V, class C>
__device__ __forceinline__ void load_rows_at(const Params& p, int s, const S* col, long long i, C (&v)[V]) {
  if (gen_slot(s)) {
    const S* b = col + i * p.rs[s];
    if (p.rs[s] == 0) {  // a row broadcast: one element for all V rows
      const C x = sload1<S>(p, s, b);
#pragma unroll
      for (int l = 0; l < V; ++l) v[l] = x;
    } else {
#pragma unroll
      for (int l = 0; l < V; ++l) v[l] = sload1<S>(p, s, b + l * p.rs[s]);
    }
  } else if (slot_ok<S>(p, s, col + i, V)) {
    IO<S>::template load<V>(col + i, v);
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = C(0);
  }
}
// 16-bit storage: the same V rows as V/2 raw words (element 2q in the low
// half of word q), converted only when they are used, so that several
// loads in flight cost half the registers; rows at or past `lim` read 0
template <class S, int V>
__device__ __forceinline__ void load_rows_raw(const Params& p, int s, const S* col, long long i, long long lim,
                                              u32 (&w)[V / 2]) {
  static_assert(sizeof(S) == 2 && V % 2 == 0, "16-bit storage, whole words");
  if (!gen_slot(s) && i + V <= lim) {
    if (slot_ok<S>(p, s, col + i, V)) {
      ldg_words(col + i, w);
    } else {
#pragma unroll
      for (int q = 0; q < V / 2; ++q) w[q] = 0u;
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < V / 2; ++q) {
    const long long r0 = i + 2 * q, r1 = r0 + 1;
    const S* a0 = row_in<S>(p, s, col, r0);
    const S* a1 = row_in<S>(p, s, col, r1);
    const u32 lo = (r0 < lim && slot_ok<S>(p, s, a0, 1)) ? (u32)ldg_u16(a0) : 0u;
    const u32 hi = (r1 < lim && slot_ok<S>(p, s, a1, 1)) ? (u32)ldg_u16(a1) : 0u;
    w[q] = lo | (hi << 16);
  }
}
// V consecutive rows of slot s from (i, j), all inside the tree
template <class S, int V, class C>
__device__ __forceinline__ void load_rows(const Params& p, int s, long long i, long long j, C (&v)[V]) {
  load_rows_at<S, V>(p, s, col_of<S>(p, s, j), i, v);
}
// V rows of slot s from q, the address of this thread's first row in some
// column (a row broadcast reads one element for all V rows)
template <class S, int V, class C>
__device__ __forceinline__ void rows_from(const Params& p, int s, const S* q, C (&v)[V]) {
  if (gen_slot(s)) {
    if (p.rs[s] == 0) {
      const C x = sload1<S>(p, s, q);
#pragma unroll
      for (int l = 0; l < V; ++l) v[l] = x;
    } else {
#pragma unroll
      for (int l = 0; l < V; ++l) v[l] = sload1<S>(p, s, q + l * p.rs[s]);
    }
  } else if (slot_ok<S>(p, s, q, V)) {
    IO<S>::template load<V>(q, v);
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = C(0);
  }
}

template <class S> __device__ __forceinline__ S* at_out_g(const Params& p, long long i, long long j) {
  if (COOT_GM & GM_OUT) return (S*)p.out + (i * p.out_rs + j * p.out_ld);
  return at_out<S>(p.out, i, j, p.out_ld);
}
// column j of the output (row 0), and row i of a column of the output
template <class S> __device__ __forceinline__ S* out_col(const Params& p, long long j) {
  return (S*)p.out + j * p.out_ld;
}
template <class S> __device__ __forceinline__ S* out_row_in(const Params& p, S* col, long long i) {
  return (COOT_GM & GM_OUT) ? col + i * p.out_rs : col + i;
}
// V consecutive rows of the output from row i of the column that starts at col
template <class S, int V, class C>
__device__ __forceinline__ void store_rows_at(const Params& p, S* col, long long i, const C (&v)[V]) {
  if (COOT_GM & GM_OUT) {
#pragma unroll
    for (int l = 0; l < V; ++l) sstore1<S>(p, col + (i + l) * p.out_rs, v[l]);
  } else if (out_ok<S>(p, col + i, V)) {
    IO<S>::template store<V>(col + i, v);
  }
}
// V rows of the output at o, this thread's first row in some output column
// (FULL: all V rows inside the tree; else rows from `lim` on are skipped)
template <bool FULL, class S, int V, class C>
__device__ __forceinline__ void rows_to(const Params& p, S* o, long long i, long long lim, const C (&v)[V]) {
  if (COOT_GM & GM_OUT) {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (FULL || i + l < lim) sstore1<S>(p, o + l * p.out_rs, v[l]);
  } else if (FULL) {
    if (out_ok<S>(p, o, V)) IO<S>::template store<V>(o, v);
  } else {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < lim) sstore1<S>(p, o + l, v[l]);
  }
}
// V consecutive rows of the output from (i, j)
template <class S, int V, class C> __device__ __forceinline__ void store_rows(const Params& p, long long i, long long j,
                                                                             const C (&v)[V]) {
  if (COOT_GM & GM_OUT) {
#pragma unroll
    for (int l = 0; l < V; ++l) sstore1<S>(p, at_out_g<S>(p, i + l, j), v[l]);
  } else if (out_ok<S>(p, at_out<S>(p.out, i, j, p.out_ld), V)) {
    IO<S>::template store<V>(at_out<S>(p.out, i, j, p.out_ld), v);
  }
}

// ---------------------------------------------------------------------------
// 16-byte groups of the compute type in shared memory
// ---------------------------------------------------------------------------
// V values of the compute type from 16-byte aligned shared memory, one
// 16-byte access per 16 bytes
struct __align__(16) W4 {
  u32 w[4];
};
template <class C> struct FromWords;
template <> struct FromWords<float> {
  static constexpr int per = 4;
  __device__ static float get(const u32* w, int l) { return __uint_as_float(w[l]); }
};
template <> struct FromWords<int> {
  static constexpr int per = 4;
  __device__ static int get(const u32* w, int l) { return (int)w[l]; }
};
template <> struct FromWords<double> {
  static constexpr int per = 2;
  __device__ static double get(const u32* w, int l) { return __hiloint2double((int)w[2 * l + 1], (int)w[2 * l]); }
};
template <class C> struct ToWords;
template <> struct ToWords<float> {
  __device__ static void put(u32* w, int l, float x) { w[l] = __float_as_uint(x); }
};
template <> struct ToWords<int> {
  __device__ static void put(u32* w, int l, int x) { w[l] = (u32)x; }
};
template <> struct ToWords<double> {
  __device__ static void put(u32* w, int l, double x) {
    w[2 * l] = (u32)__double2loint(x);
    w[2 * l + 1] = (u32)__double2hiint(x);
  }
};
// one 16-byte group of the compute type to 16-byte aligned shared memory
template <class C, int G> __device__ __forceinline__ void sts_group(C* p, const C (&v)[G]) {
  static_assert(G * sizeof(C) == 16, "one 16-byte group");
  W4 t;
#pragma unroll
  for (int l = 0; l < G; ++l) ToWords<C>::put(t.w, l, v[l]);
  *reinterpret_cast<W4*>(p) = t;
}
template <class C, int V> __device__ __forceinline__ void lds_vec(const C* p, C (&v)[V]) {
  constexpr int PER = FromWords<C>::per;
  static_assert(V % PER == 0, "whole 16-byte groups");
  const W4* q = reinterpret_cast<const W4*>(p);
#pragma unroll
  for (int n = 0; n < V / PER; ++n) {
    W4 t = q[n];
#pragma unroll
    for (int l = 0; l < PER; ++l) v[n * PER + l] = FromWords<C>::get(t.w, l);
  }
}

// ---------------------------------------------------------------------------
// per-element contribution of the root to the reduction
// ---------------------------------------------------------------------------
// pos: the element's position in its reduction (column-major linear index for
// a full reduction, row index along dim 0, column index along dim 1); only
// index_min / index_max read it (and min / max, to keep the first of equal
// values), everywhere else the expression is dead code.
template <class T, int RED, class X, class K, class A, class Q>
__device__ __forceinline__ typename X::C eval_elem(const X& x, const K& k, u32& err, int l, A& acc, const Q& csq,
                                                   long long pos) {
  typedef typename X::C C;
  if constexpr (red_extreme(RED)) {
    C y = T::ev(x, k, err, l);
    acc.add_at(y, pos);
    return y;
  } else if constexpr (RED == RED_PROD) {
    C y = T::ev(x, k, err, l);
    acc.mul(y);
    return y;
  } else if constexpr (RED == RED_DOT) {
    C a = T::A::ev(x, k, err, l), b = T::B::ev(x, k, err, l);
    acc.add_prod(a, b);
    return op_mul(a, b);
  } else {
    C y = T::ev(x, k, err, l);
    if constexpr (RED == RED_SUM || RED == RED_MEAN1) acc.add(y);
    if constexpr (RED == RED_SSQ) acc.add_prod(y, y);
    if constexpr (RED == RED_CSQ) {
      C d = csq.centred(y);
      acc.add(op_mul(d, d));
    }
    return y;
  }
}

// The element's value y and, in c, its term of the reduction, for the
// pairwise path: the V terms of one vector load are summed pairwise in FP32
// before a single float-float addition.  16-bit storage: products and
// squares of two 16-bit values are exact in FP32 (at most 22 significant
// bits), and sums of two such terms are exact unless their exponents differ
// by more than 15.  FP32 sums of squares (norm, var's second pass): every
// term is positive, so a rounded square (relative error u) and the pairwise
// sums (u per level) add at most (1 + log2 V) u to the relative error of the
// result -- rounding errors of positive terms cannot cancel into more.
template <class T, int RED, class X, class K, class Q>
__device__ __forceinline__ typename X::C eval_term(const X& x, const K& k, u32& err, int l, const Q& csq,
                                                   typename X::C& c) {
  typedef typename X::C C;
  if constexpr (RED == RED_DOT) {
    C a = T::A::ev(x, k, err, l), b = T::B::ev(x, k, err, l);
    c = op_mul(a, b);
    return c;
  } else {
    C y = T::ev(x, k, err, l);
    if constexpr (RED == RED_SSQ) c = op_mul(y, y);
    else if constexpr (RED == RED_CSQ) {
      C d = csq.centred(y);
      c = op_mul(d, d);
    } else
      c = y;
    return y;
  }
}

// the final value written for one reduction output
template <class C, int RED, class A>
__device__ __forceinline__ void write_result(const Params& p, const A& a, long long idx, double div) {
  typedef typename rtype<C>::type R;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if constexpr (RED == RED_IMIN || RED == RED_IMAX) {
    // positions are int64 for every element type; -1: no element (or all NaN)
    ((long long*)p.red_out)[idx] = (a.pos == POS_NONE) ? -1ll : (long long)a.pos;
  } else if constexpr (RED == RED_MIN || RED == RED_MAX) {
    if constexpr (is_int_c<C>::value)
      ((long long*)p.red_out)[idx] = (a.pos == POS_NONE) ? 0ll : (long long)a.v;
    else
      ((R*)p.red_out)[idx] = (a.pos == POS_NONE) ? (R)qnan : (R)a.v;
  } else if constexpr (is_int_c<C>::value) {
    // integer trees: exact int64 sums and products (sum / dot / prod)
    ((long long*)p.red_out)[idx] = a.ivalue();
  } else {
    if constexpr (RED == RED_SUM || RED == RED_DOT) {
      ((R*)p.red_out)[idx] = (R)(a.value() / div);
    } else if constexpr (RED == RED_PROD) {
      ((R*)p.red_out)[idx] = (R)a.value();
    } else if constexpr (RED == RED_SSQ) {
      ((R*)p.red_out)[idx] = (R)sqrt(a.value());
    } else if constexpr (RED == RED_MEAN1) {
      p.mu[idx] = a.value() / (double)p.count;  // count: elements per output
    } else if constexpr (RED == RED_CSQ) {
      double v;
      if (p.count == 0)
        v = qnan;  // no elements
      else if (p.count == 1)
        v = 0.0;
      else
        v = a.value() / p.den;
      if (p.flags & PF_SQRT) v = sqrt(v);
      ((R*)p.red_out)[idx] = (R)v;
    }
  }
}

// block-level partial -> ticket -> last block combines all partials in order
template <class C, int RED, class A> __device__ __forceinline__ void finish_full(const Params& p, A acc, A* smem) {
  __shared__ int am_last;
  acc = block_reduce(acc, smem);
  if (threadIdx.x == 0) {
    ((A*)p.partials)[blockIdx.x] = acc;
    __threadfence();
    unsigned int t = atomicAdd(p.tickets, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    A a;
    a.init();
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) a.merge(load_cg(&((const A*)p.partials)[b]));
    a = block_reduce(a, smem);
    if (threadIdx.x == 0) {
      write_result<C, RED>(p, a, 0, p.div);
      *p.tickets = 0u;  // ready for the next launch
    }
  }
}

// ---------------------------------------------------------------------------
// The units of a grid-stride 2-D walk over cpc chunks per column, each unit
// `per` consecutive chunks in column-major chunk order: the first chunk of
// unit u is q = u * per, for u = blockIdx.x, blockIdx.x + gridDim.x, ...  It
// is kept as (column j, chunk r within the column) and advanced by additions
// (one division per block, not one per unit).  Invariant: q = j * cpc + r
// with 0 <= r < cpc, so q < cpc * n_cols exactly when j < n_cols.
// ---------------------------------------------------------------------------
struct UnitWalk {
  long long j, r;
  const long long cpc, qg, rg;
  __device__ __forceinline__ UnitWalk(long long cpc_, long long per = 1)
      : j((long long)blockIdx.x * per / cpc_),
        r((long long)blockIdx.x * per - j * cpc_),
        cpc(cpc_),
        qg((long long)gridDim.x * per / cpc_),
        rg((long long)gridDim.x * per - qg * cpc_) {}
  __device__ __forceinline__ void next() {
    j += qg;
    r += rg;
    if (r >= cpc) {
      r -= cpc;
      ++j;
    }
  }
};

// ---------------------------------------------------------------------------
// str: map (+ full reduction) over n_rows x n_cols, no transposed reads
// ---------------------------------------------------------------------------
// One unit of the walk: U chunks from chunk r of column j.  FAST: the unit
// stays inside column j and every row of its chunks is inside the tree (the
// same for the whole block), so nothing is checked and no chunk wraps.
template <bool FAST, class T, class S, int NS, int NK, int RED, int V, int U, bool OUT, class A, class K, class Q>
__device__ __forceinline__ void str_unit(const Params& p, const K& k, const Q& csq, u32& err, A (&accs)[V],
                                         long long j, long long r) {
  typedef typename ctype<S>::type C;
  const long long nr = p.n_rows, nc = p.n_cols, cpc = p.units_per_col;
  const long long step = (long long)blockDim.x * V;
  const long long tv = (long long)threadIdx.x * V;
  // the current chunk's column of every slot and of the output: formed once
  // per unit, then moved one column on when the chunks wrap
  const S* col[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) col[s] = col_of<S>(p, s, j);
  S* oc = nullptr;
  if constexpr (OUT) oc = out_col<S>(p, j);
  // 16-bit storage keeps its loads as raw words until they are used
  constexpr bool RAW = sizeof(S) == 2 && V >= 2;
  Vals<C, NS, V> x[RAW ? 1 : U];
  u32 raw[RAW ? U : 1][RAW ? NS : 1][RAW ? V / 2 : 1];
  bool valid[U], full[U];
  long long ig[U], jg[U];
  S* og[U];
#pragma unroll
  for (int g = 0; g < U; ++g) {
    const long long i = r * step + tv;
    valid[g] = FAST || (j < nc);
    full[g] = FAST || (valid[g] && (i + V <= nr));
    ig[g] = i;
    jg[g] = j;
    og[g] = oc;
    if constexpr (RAW) {
#pragma unroll
      for (int s = 0; s < NS; ++s) load_rows_raw<S, V>(p, s, col[s], i, (FAST || valid[g]) ? nr : 0, raw[g][s]);
    } else if (full[g]) {
#pragma unroll
      for (int s = 0; s < NS; ++s) load_rows_at<S, V>(p, s, col[s], i, x[g].v[s]);
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int l = 0; l < V; ++l)
          x[g].v[s][l] = (valid[g] && i + l < nr) ? sload1<S>(p, s, row_in<S>(p, s, col[s], i + l)) : C(0);
    }
    if constexpr (FAST) {
      ++r;
    } else if (g + 1 < U && ++r == cpc) {  // the next chunk starts the next column
      r = 0;
      ++j;
#pragma unroll
      for (int s = 0; s < NS; ++s) col[s] += p.ld[s];
      if constexpr (OUT) oc += p.out_ld;
    }
  }
#pragma unroll
  for (int g = 0; g < U; ++g) {
    const long long i = ig[g];
    const Vals<C, NS, V>* xg = &x[RAW ? 0 : g];
    if constexpr (RAW) {
      if (valid[g]) {
#pragma unroll
        for (int s = 0; s < NS; ++s) IO<S>::template convert<V>(raw[g][s], x[0].v[s]);
      }
    }
    if (full[g]) {
      C y[V];
      if constexpr ((sizeof(S) == 2 && red_additive(RED)) ||
                    (is_f32_c<S>::value && (RED == RED_SSQ || RED == RED_CSQ))) {
        // pairwise sum of the vector's terms, then one float-float
        // addition (spread over the accumulators by group)
        C c[V];
#pragma unroll
        for (int l = 0; l < V; ++l) y[l] = eval_term<T, RED>(*xg, k, err, l, csq, c[l]);
#pragma unroll
        for (int w = V / 2; w >= 1; w /= 2)
#pragma unroll
          for (int l = 0; l < w; ++l) c[l] = op_add(c[l], c[l + w]);
        accs[g % V].add(c[0]);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(*xg, k, err, l, accs[l], csq, i + l + jg[g] * nr);
      }
      if constexpr (OUT) store_rows_at<S, V>(p, og[g], i, y);
    } else if (valid[g]) {
#pragma unroll
      for (int l = 0; l < V; ++l)
        if (i + l < nr) {
          C y = eval_elem<T, RED>(*xg, k, err, l, accs[l], csq, i + l + jg[g] * nr);
          if constexpr (OUT) sstore1<S>(p, out_row_in<S>(p, og[g], i + l), y);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// str: map (+ full reduction) over n_rows x n_cols, no transposed reads
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT>
__device__ __forceinline__ void str_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ A smem[32];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  if constexpr (RED == RED_CSQ) csq.set_mean(*p.mu);
  u32 err = 0;
  // one accumulator per vector lane: V independent addition chains
  A accs[V];
#pragma unroll
  for (int l = 0; l < V; ++l) accs[l].init();
  // chunks of `step` rows, cpc of them per column; a unit is U consecutive
  // chunks in column-major order, so a unit continues into the next column
  // when columns are shorter than U chunks and every thread keeps U vector
  // loads in flight whatever the column length
  const long long nr = p.n_rows, nc = p.n_cols, cpc = p.units_per_col;
  const long long step = (long long)blockDim.x * V;
  for (UnitWalk walk(cpc, U); walk.j < nc; walk.next()) {
    if (walk.r + U <= cpc && (walk.r + U) * step <= nr)
      str_unit<true, T, S, NS, NK, RED, V, U, OUT>(p, k, csq, err, accs, walk.j, walk.r);
    else
      str_unit<false, T, S, NS, NK, RED, V, U, OUT>(p, k, csq, err, accs, walk.j, walk.r);
  }
  if (err) atomicOr(p.err_flag, err);
  if constexpr (RED != RED_NONE) {
#pragma unroll
    for (int l = 1; l < V; ++l) accs[0].merge(accs[l]);
    finish_full<C, RED>(p, accs[0], smem);
  }
}

// ---------------------------------------------------------------------------
// col: map + per-column reduction (dim 0).  A group of G warps (G =
// p.n_splits, a divisor of the warps per block) owns one column at a time and
// splits its rows; the group's warp results are combined in shared memory in
// warp order.  Every block runs the same number of column steps, so the
// barriers are uniform.
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT>
__device__ __forceinline__ void col_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ A wsum[32];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  u32 err = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long wpb = blockDim.x >> 5;
  const long long G = p.n_splits;  // warps per column
  const long long gpb = wpb / G;   // columns per block step
  const long long gi = warp / G, wm = warp % G;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long step = 32LL * V;
  for (long long base = (long long)blockIdx.x * gpb; base < nc; base += (long long)gridDim.x * gpb) {
    const long long j = base + gi;
    A acc;
    acc.init();
    if constexpr (RED == RED_CSQ) csq.set_mean(p.mu[j < nc ? j : 0]);
    // column j of every slot (row 0), formed once per column
    const S* cj[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cj[s] = col_of<S>(p, s, j < nc ? j : 0);
    for (long long i0 = (wm * 32 + lane) * V; j < nc && i0 < nr; i0 += G * step * U) {
      Vals<C, NS, V> x[U];
      if (i0 + (U - 1) * G * step + V <= nr) {
        // every group's V rows inside the tree: nothing checked
#pragma unroll
        for (int g = 0; g < U; ++g) {
          const long long i = i0 + g * G * step;
#pragma unroll
          for (int s = 0; s < NS; ++s) rows_from<S, V>(p, s, row_in<S>(p, s, cj[s], i), x[g].v[s]);
        }
#pragma unroll
        for (int g = 0; g < U; ++g) {
          const long long i = i0 + g * G * step;
          C y[V];
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc, csq, i + l);
          if constexpr (OUT) store_rows<S, V>(p, i, j, y);
        }
        continue;
      }
      bool full[U];
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long i = i0 + g * G * step;
        full[g] = (i + V <= nr);
        if (full[g]) {
#pragma unroll
          for (int s = 0; s < NS; ++s) load_rows<S, V>(p, s, i, j, x[g].v[s]);
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < V; ++l)
              x[g].v[s][l] = (i + l < nr) ? sload1<S>(p, s, at_slot<S>(p, s, i + l, j)) : C(0);
        }
      }
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long i = i0 + g * G * step;
        if (full[g]) {
          C y[V];
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc, csq, i + l);
          if constexpr (OUT) store_rows<S, V>(p, i, j, y);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (i + l < nr) {
              C y = eval_elem<T, RED>(x[g], k, err, l, acc, csq, i + l);
              if constexpr (OUT) sstore1<S>(p, at_out_g<S>(p, i + l, j), y);
            }
        }
      }
    }
    acc = warp_reduce(acc);
    if (G == 1) {
      if (lane == 0 && j < nc) write_result<C, RED>(p, acc, j, p.div);
    } else {
      if (lane == 0) wsum[warp] = acc;
      __syncthreads();
      if (wm == 0 && lane == 0 && j < nc) {
        A a = wsum[gi * G];
        for (long long w = 1; w < G; ++w) a.merge(wsum[gi * G + w]);
        write_result<C, RED>(p, a, j, p.div);
      }
      __syncthreads();
    }
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// row: map + per-row reduction (dim 1)
//   block b -> row block rb = b % n_row_blocks, column split sp = b / n_row_blocks
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT, int TRMASK = 0>
__device__ __forceinline__ void row_kernel(const Params& p) {
  static_assert(TRMASK == 0 || V == 1, "transposed slots: one row per thread");
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ int am_last;
  // transposed runs read by a whole warp (blocks of up to 8 warps): a tile of
  // 32 rows of U values per warp, rows padded by 16 bytes
  constexpr int PER = 16 / (int)sizeof(S), CPR = U / PER > 0 ? U / PER : 1, GC = 16 / (int)sizeof(C);
  constexpr bool COOP = TRMASK != 0 && U % PER == 0 && 32 % CPR == 0;
  constexpr int TRS = U + GC;
  __shared__ __align__(16) C rtiles[COOP ? 8 : 1][COOP ? 32 * TRS : 4];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long nrb = p.n_row_blocks, nsp = p.n_splits, cps = p.units_per_col;
  const long long rb = blockIdx.x % nrb, sp = blockIdx.x / nrb;
  const long long i = (rb * blockDim.x + threadIdx.x) * V;
  const long long j0 = sp * cps;
  const long long j1 = (j0 + cps < nc) ? j0 + cps : nc;
  const bool fullv = (i + V <= nr);
  // segmented (a Cube's slices side by side): split sp is output column sp
  const bool segd = (p.flags & PF_SEGMENTED) != 0;
  const long long o0 = segd ? sp * nr : 0, pbase = segd ? j0 : 0;
  A acc[V];
  typename CsqOf<C>::type csq[V];  // var along dim 1: one mean per row
#pragma unroll
  for (int l = 0; l < V; ++l) {
    acc[l].init();
    if constexpr (RED == RED_CSQ) csq[l].set_mean(i + l < nr ? p.mu[o0 + i + l] : 0.0);
  }
  if (i < nr) {
    long long jb = j0;
    if (fullv) {
      // groups of U columns inside the segment with all V rows inside the
      // tree: row pointers stepped by the column strides, nothing checked
      const S* rp[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s)
        rp[s] = (const S*)p.src[s] + ((gen_slot(s) || ((TRMASK >> s) & 1)) ? i * p.rs[s] : i);
      S* op = nullptr;
      if constexpr (OUT) op = (S*)p.out + ((COOT_GM & GM_OUT) ? i * p.out_rs : i);
      // a warp whose 32 rows are all inside the tree reads transposed runs
      // together (uniform over the warp)
      const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
      const long long iw = i - lane;
      const bool coop = COOP && blockDim.x <= 256 && iw + 32 <= nr && j0 % PER == 0;
      C* tile = rtiles[COOP ? (wp & 7) : 0];
      for (; jb + U <= j1; jb += U) {
        Vals<C, NS, V> x[U];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if ((TRMASK >> s) & 1) {
            // a transposed slot: this row's U columns are consecutive in
            // memory (16-byte vectors where the host found the rows aligned
            // and the segment starts on a whole vector)
            const S* q = rp[s] + jb;
            if (COOP && coop && (p.flags & (PF_TRUN0 << s))) {
              // lanes CPR apart read consecutive 16-byte pieces of one row's
              // run; the pieces go to their rows below
#pragma unroll
              for (int g = 0; g < CPR; ++g) {
                const S* qq = (const S*)p.src[s] + (iw + g * (32 / CPR) + lane / CPR) * p.rs[s] + jb +
                              (lane % CPR) * PER;
                C t[PER];
                if (slot_ok<S>(p, s, qq, PER)) {
                  IO<S>::template load<PER>(qq, t);
                } else {
#pragma unroll
                  for (int e = 0; e < PER; ++e) t[e] = C(0);
                }
#pragma unroll
                for (int e = 0; e < PER; ++e) x[g * PER + e].v[s][0] = t[e];
              }
            } else if (U % PER == 0 && j0 % PER == 0 && (p.flags & (PF_TRUN0 << s)) && slot_ok<S>(p, s, q, U)) {
#pragma unroll
              for (int g0 = 0; g0 < U / PER; ++g0) {
                C t[PER];
                IO<S>::template load<PER>(q + g0 * PER, t);
#pragma unroll
                for (int e = 0; e < PER; ++e) x[g0 * PER + e].v[s][0] = t[e];
              }
            } else {
#pragma unroll
              for (int g = 0; g < U; ++g) x[g].v[s][0] = sload1<S>(p, s, q + g);
            }
            continue;
          }
          const long long ld = p.ld[s];
          const S* q = rp[s] + jb * ld;
#pragma unroll
          for (int g = 0; g < U; ++g, q += ld) rows_from<S, V>(p, s, q, x[g].v[s]);
        }
        if constexpr (COOP) {
          if (coop) {
            // every cooperatively read slot: the pieces through the warp's
            // tile, each lane taking back its own row's U values
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              if (!((TRMASK >> s) & 1) || !(p.flags & (PF_TRUN0 << s))) continue;
              __syncwarp();
#pragma unroll
              for (int g = 0; g < CPR; ++g) {
                C* d = tile + (g * (32 / CPR) + lane / CPR) * TRS + (lane % CPR) * PER;
#pragma unroll
                for (int e0 = 0; e0 < PER; e0 += GC) {
                  C v[GC];
#pragma unroll
                  for (int e = 0; e < GC; ++e) v[e] = x[g * PER + e0 + e].v[s][0];
                  sts_group<C, GC>(d + e0, v);
                }
              }
              __syncwarp();
              C r[U];
              lds_vec<C, U>(tile + lane * TRS, r);
#pragma unroll
              for (int u = 0; u < U; ++u) x[u].v[s][0] = r[u];
            }
          }
        }
#pragma unroll
        for (int g = 0; g < U; ++g) {
          C y[V];
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc[l], csq[l], jb + g - pbase);
          if constexpr (OUT) rows_to<true, S, V>(p, op + (jb + g) * p.out_ld, i, nr, y);
        }
      }
    }
    for (; jb < j1; jb += U) {
      Vals<C, NS, V> x[U];
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long j = jb + g;
        if (j < j1) {
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if ((TRMASK >> s) & 1) {  // element (i, j) at i rs + j
              x[g].v[s][0] = sload1<S>(p, s, (const S*)p.src[s] + (i * p.rs[s] + j));
            } else if (fullv) {
              load_rows<S, V>(p, s, i, j, x[g].v[s]);
            } else {
#pragma unroll
              for (int l = 0; l < V; ++l)
                x[g].v[s][l] = (i + l < nr) ? sload1<S>(p, s, at_slot<S>(p, s, i + l, j)) : C(0);
            }
          }
        }
      }
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long j = jb + g;
        if (j < j1) {
          if (fullv) {
            C y[V];
#pragma unroll
            for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc[l], csq[l], j - pbase);
            if constexpr (OUT) store_rows<S, V>(p, i, j, y);
          } else {
#pragma unroll
            for (int l = 0; l < V; ++l)
              if (i + l < nr) {
                C y = eval_elem<T, RED>(x[g], k, err, l, acc[l], csq[l], j - pbase);
                if constexpr (OUT) sstore1<S>(p, at_out_g<S>(p, i + l, j), y);
              }
          }
        }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
  if (nsp == 1 || segd) {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < nr) write_result<C, RED>(p, acc[l], o0 + i + l, p.div);
    return;
  }
#pragma unroll
  for (int l = 0; l < V; ++l)
    if (i + l < nr) ((A*)p.partials)[sp * nr + i + l] = acc[l];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(&p.tickets[rb], 1u);
    am_last = (t == (unsigned int)(nsp - 1));
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < nr) {
        A a;
        a.init();
        for (long long s = 0; s < nsp; ++s) a.merge(load_cg(&((const A*)p.partials)[s * nr + i + l]));
        write_result<C, RED>(p, a, i + l, p.div);
      }
    if (threadIdx.x == 0) p.tickets[rb] = 0u;
  }
}

// ---------------------------------------------------------------------------
// tile: any tree with transposed reads; TRMASK marks the transposed slots.
//   32x32 output tile, 256 threads as 32 (rows) x 8 (column phases); each
//   thread evaluates rows i = 32 ti + tx of columns j = 32 tj + ty + 8 q.
//   A transposed slot reads view(j, i): its 32x32 source block is read with
//   consecutive threads on consecutive source rows and parked in shared
//   memory with one column of padding, then read back transposed.
//   DIM -1 (full reduction or none): blocks stride over all tiles.
//   DIM 0 / 1 (per column / per row): the outputs of one strip of 32 columns
//   (DIM 0) or 32 rows (DIM 1) depend on that strip's tiles only.  Block b
//   owns segment b % n_splits of strip b / n_splits and keeps its
//   accumulators in registers across the segment's tiles (a thread's four
//   columns, or its row, stay the same), so it reduces across threads once;
//   with several segments per strip the last block of the strip (ticket)
//   combines the segment partials in segment order.
// ---------------------------------------------------------------------------
constexpr int TILE = 32;
constexpr int TILE_PH = 8;  // blockDim.x == TILE * TILE_PH
constexpr int TILE_Q = TILE / TILE_PH;

template <int M> struct popc { static constexpr int value = (M & 1) + popc<(M >> 1)>::value; };
template <> struct popc<0> { static constexpr int value = 0; };

// the operand values of this thread's four elements of tile (ti, tj)
template <class S, int NS, int TRMASK, int NTR, class C>
__device__ __forceinline__ void tile_load(const Params& p, long long ti, long long tj, Vals<C, NS, TILE_Q>& x,
                                          C (*stage)[TILE][TILE + 1]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long i = ti * TILE + tx;
  // direct reads first: they stay in flight while transposed blocks are staged
#pragma unroll
  for (int w = 0; w < TILE_Q; ++w) {
    const long long j = tj * TILE + ty + TILE_PH * w;
    const bool ok = (i < nr && j < nc);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (!((TRMASK >> s) & 1)) x.v[s][w] = ok ? sload1<S>(p, s, at_slot<S>(p, s, i, j)) : C(0);
  }
  if constexpr (NTR > 0) {
    __syncthreads();  // the previous tile's shared reads are done
    int q = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if ((TRMASK >> s) & 1) {
        const long long vr = tj * TILE + tx;  // view row  = output column
#pragma unroll
        for (int w = 0; w < TILE_Q; ++w) {
          const long long vc = ti * TILE + ty + TILE_PH * w;  // view column = output row
          stage[q][ty + TILE_PH * w][tx] = (vr < nc && vc < nr) ? sload1<S>(p, s, at<S>(p.src[s], vr, vc, p.ld[s])) : C(0);
        }
        ++q;
      }
    __syncthreads();
    q = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if ((TRMASK >> s) & 1) {
#pragma unroll
        for (int w = 0; w < TILE_Q; ++w) x.v[s][w] = stage[q][tx][ty + TILE_PH * w];
        ++q;
      }
  }
}

// End of a strip segment: blk[q] holds this block's value for output
// o = OS strip + q (q < OS).  One segment: write the results.  Several: park
// the value in the partials (segment-major), and the strip's last block
// (ticket) merges the segments in order and writes the results.
template <class C, int RED, int OS, class A>
__device__ __forceinline__ void strip_finish(const Params& p, const A* blk, long long strip, long long seg,
                                             long long nseg, long long no, int* am_last) {
  const int q = threadIdx.x;
  const long long o = strip * OS + q;
  if (nseg == 1) {
    if (q < OS && o < no) write_result<C, RED>(p, blk[q], o, p.div);
    return;
  }
  if (q < OS && o < no) ((A*)p.partials)[seg * no + o] = blk[q];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int tk = atomicAdd(&p.tickets[strip], 1u);
    *am_last = (tk == (unsigned int)(nseg - 1));
  }
  __syncthreads();
  if (*am_last) {
    __threadfence();
    if (q < OS && o < no) {
      A a = load_cg(&((const A*)p.partials)[o]);
      for (long long sg = 1; sg < nseg; ++sg) a.merge(load_cg(&((const A*)p.partials)[sg * no + o]));
      write_result<C, RED>(p, a, o, p.div);
    }
    if (threadIdx.x == 0) p.tickets[strip] = 0u;
  }
}

template <class T, class S, int NS, int NK, int RED, int DIM, int TRMASK, bool OUT>
__device__ __forceinline__ void tile_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  __shared__ C stage[NTR > 0 ? NTR : 1][TILE][TILE + 1];
  __shared__ A smem[32];
  __shared__ A rsum[TILE_PH][TILE];
  __shared__ int am_last;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long ntr = (nr + TILE - 1) / TILE, ntc = (nc + TILE - 1) / TILE;
  if constexpr (DIM == -1) {
    typename CsqOf<C>::type csq;
    if constexpr (RED == RED_CSQ) csq.set_mean(*p.mu);
    const long long tiles = ntr * ntc;
    A acc;
    acc.init();
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
      const long long ti = t % ntr, tj = t / ntr;
      const long long i = ti * TILE + tx;
      Vals<C, NS, TILE_Q> x;
      tile_load<S, NS, TRMASK, NTR>(p, ti, tj, x, stage);
#pragma unroll
      for (int w = 0; w < TILE_Q; ++w) {
        const long long j = tj * TILE + ty + TILE_PH * w;
        if (i < nr && j < nc) {
          C y = eval_elem<T, RED>(x, k, err, w, acc, csq, i + j * nr);
          if constexpr (OUT) sstore1<S>(p, at_out_g<S>(p, i, j), y);
        }
      }
    }
    if (err) atomicOr(p.err_flag, err);
    if constexpr (RED != RED_NONE) finish_full<C, RED>(p, acc, smem);
  } else {
    const long long nseg = p.n_splits;
    // the strips' segments, taken by the blocks in turn
    const long long units = ((DIM == 0) ? ntc : ntr) * nseg;
    for (long long unit = blockIdx.x; unit < units; unit += gridDim.x) {
    const long long strip = unit / nseg, seg = unit % nseg;
    const long long len = (DIM == 0) ? ntr : ntc;  // tiles along the strip
    const long long per = (len + nseg - 1) / nseg;
    const long long t0 = seg * per, t1 = (t0 + per < len) ? t0 + per : len;
    // DIM 0: one accumulator per column phase w (output j = 32 strip + ty + 8 w);
    // DIM 1: one per thread (output i = 32 strip + tx)
    A acc[DIM == 0 ? TILE_Q : 1];
    typename CsqOf<C>::type csq[DIM == 0 ? TILE_Q : 1];
#pragma unroll
    for (int w = 0; w < (DIM == 0 ? TILE_Q : 1); ++w) {
      acc[w].init();
      if constexpr (RED == RED_CSQ) {
        const long long o = (DIM == 0) ? strip * TILE + ty + TILE_PH * w : strip * TILE + tx;
        const long long no = (DIM == 0) ? nc : nr;
        csq[w].set_mean(o < no ? p.mu[o] : 0.0);
      }
    }
    for (long long t = t0; t < t1; ++t) {
      const long long ti = (DIM == 0) ? t : strip, tj = (DIM == 0) ? strip : t;
      const long long i = ti * TILE + tx;
      Vals<C, NS, TILE_Q> x;
      tile_load<S, NS, TRMASK, NTR>(p, ti, tj, x, stage);
#pragma unroll
      for (int w = 0; w < TILE_Q; ++w) {
        const long long j = tj * TILE + ty + TILE_PH * w;
        if (i < nr && j < nc) {
          C y;
          if constexpr (DIM == 0)
            y = eval_elem<T, RED>(x, k, err, w, acc[w], csq[w], i);
          else
            y = eval_elem<T, RED>(x, k, err, w, acc[0], csq[0], j);
          if constexpr (OUT) sstore1<S>(p, at_out_g<S>(p, i, j), y);
        }
      }
    }
    const long long no = (DIM == 0) ? nc : nr;
    // this block's value for each output of the strip: rsum[0][o % 32]
    if constexpr (DIM == 0) {
#pragma unroll
      for (int w = 0; w < TILE_Q; ++w) {
        A a = warp_reduce(acc[w]);  // the block's rows of column 32 strip + ty + 8 w
        if (tx == 0) rsum[0][ty + TILE_PH * w] = a;
      }
      __syncthreads();
    } else {
      rsum[ty][tx] = acc[0];
      __syncthreads();
      if (ty == 0) {
        A a = rsum[0][tx];
        for (int r = 1; r < TILE_PH; ++r) a.merge(rsum[r][tx]);
        rsum[0][tx] = a;
      }
      __syncthreads();
    }
    strip_finish<C, RED, TILE>(p, &rsum[0][0], strip, seg, nseg, no, &am_last);
    __syncthreads();  // rsum is read by the finish before the next unit writes it
    }  // units
    if (err) atomicOr(p.err_flag, err);
  }
}

// ---------------------------------------------------------------------------
// tilev: vectorised variant of tile.
//   Tile of TM = 32 V rows x 32 columns; thread (tx, ty) owns rows
//   32 V ti + V tx .. + V-1 of columns 32 tj + ty + 8 w (w < 4), so direct
//   reads and the output move V elements (16 bytes) per access.  A transposed
//   slot's 32 x TM source block is read with consecutive threads on
//   consecutive source rows into stage[q][column][row] (row stride TM + 4, a
//   multiple of 16 bytes) and read back as one 16-byte vector per thread.
//   Reductions along a dim use the strip segments of the tile kernel, with
//   strips of 32 columns (DIM 0) or TM rows (DIM 1).
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int DIM, int TRMASK, bool OUT, int V>
__device__ __forceinline__ void tilev_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  constexpr int TM = TILE * V;
  constexpr int SP = TM + 16 / (int)sizeof(C);
  // DIM -1: V accumulators (one per vector lane); DIM 0: one per column
  // phase w; DIM 1: one per row of the thread's vector
  constexpr int NA = (DIM == 0) ? TILE_Q : V;
  __shared__ __align__(16) C stage[NTR > 0 ? NTR : 1][TILE][SP];
  __shared__ A smem[32];
  __shared__ A rsum[TILE_PH][TILE];
  __shared__ A blk[DIM == 1 ? TM : TILE];
  __shared__ int am_last;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long ntr = (nr + TM - 1) / TM, ntc = (nc + TILE - 1) / TILE;
  // work units: DIM -1, one unit, all tiles strided over the grid; DIM 0 / 1,
  // the segments of the strips (DIM 0: column strip tj, DIM 1: row strip ti),
  // strips x n_splits of them, taken by the blocks in turn (a grid of about
  // the resident blocks, so no partial last wave)
  const long long nseg = (DIM == -1) ? 1 : p.n_splits;
  const long long units = (DIM == -1) ? 1 : ((DIM == 0) ? ntc : ntr) * nseg;
  for (long long unit = (DIM == -1) ? 0 : blockIdx.x; unit < units; unit += (DIM == -1) ? 1 : gridDim.x) {
  long long t_first, t_end, t_step, strip = 0, seg = 0;
  if constexpr (DIM == -1) {
    t_first = blockIdx.x;
    t_end = ntr * ntc;
    t_step = gridDim.x;
  } else {
    strip = unit / nseg;
    seg = unit % nseg;
    const long long len = (DIM == 0) ? ntr : ntc;
    const long long per = (len + nseg - 1) / nseg;
    t_first = seg * per;
    t_end = (t_first + per < len) ? t_first + per : len;
    t_step = 1;
  }
  A acc[NA];
  typename CsqOf<C>::type csq[NA];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    acc[a].init();
    if constexpr (RED == RED_CSQ) {
      if constexpr (DIM == -1) {
        csq[a].set_mean(*p.mu);
      } else if constexpr (DIM == 0) {
        const long long o = strip * TILE + ty + TILE_PH * a;
        csq[a].set_mean(o < nc ? p.mu[o] : 0.0);
      } else {
        const long long o = strip * TM + (long long)tx * V + a;
        csq[a].set_mean(o < nr ? p.mu[o] : 0.0);
      }
    }
  }
  for (long long t = t_first; t < t_end; t += t_step) {
    long long ti, tj;
    if constexpr (DIM == -1) {
      ti = t % ntr;
      tj = t / ntr;
    } else if constexpr (DIM == 0) {
      ti = t;
      tj = strip;
    } else {
      ti = strip;
      tj = t;
    }
    const long long i0 = ti * TM + (long long)tx * V;
    const bool fullr = (i0 + V <= nr);
    const bool interior = (ti + 1) * TM <= nr && (tj + 1) * TILE <= nc;  // block-uniform
    Vals<C, NS, V> x[TILE_Q];
    // direct reads first: in flight while transposed blocks are staged
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((TRMASK >> s) & 1) continue;
        if (j < nc && fullr) {
          load_rows<S, V>(p, s, i0, j, x[w].v[s]);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            x[w].v[s][l] = (j < nc && i0 + l < nr) ? sload1<S>(p, s, at_slot<S>(p, s, i0 + l, j)) : C(0);
        }
      }
    }
    if constexpr (NTR > 0) {
      __syncthreads();  // the previous tile's shared reads are done
      int q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
          // thread (tx, ty) reads view row tj 32 + tx at the view columns of
          // 16-byte groups ty, ty + 8, ...: a warp reads 32 consecutive
          // elements per column, and writes each group with one 16-byte
          // shared store (row stride TM + GE: eight consecutive rows fall on
          // eight different 16-byte bank groups, no conflict)
          constexpr int GE = 16 / (int)sizeof(C);
          constexpr int NG = TM / GE / TILE_PH;
          const long long vr = tj * TILE + tx;  // view row = output column
          C v[NG][GE];  // all of this thread's staging loads in flight at once
          if (interior) {
            // whole tile inside the view: one base pointer, constant steps
            const long long ld = p.ld[s];
            const S* b = at<S>(p.src[s], vr, ti * TM + ty * GE, ld);
#pragma unroll
            for (int g = 0; g < NG; ++g)
#pragma unroll
              for (int e = 0; e < GE; ++e) v[g][e] = sload1<S>(p, s, b + ((long long)(TILE_PH * g * GE + e)) * ld);
          } else {
#pragma unroll
            for (int g = 0; g < NG; ++g)
#pragma unroll
              for (int e = 0; e < GE; ++e) {
                const long long vc = ti * TM + (ty + TILE_PH * g) * GE + e;  // view column = output row
                v[g][e] = (vr < nc && vc < nr) ? sload1<S>(p, s, at<S>(p.src[s], vr, vc, p.ld[s])) : C(0);
              }
          }
#pragma unroll
          for (int g = 0; g < NG; ++g) sts_group<C, GE>(&stage[q][tx][(ty + TILE_PH * g) * GE], v[g]);
          ++q;
        }
      __syncthreads();
      q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
#pragma unroll
          for (int w = 0; w < TILE_Q; ++w) lds_vec<C, V>(&stage[q][ty + TILE_PH * w][tx * V], x[w].v[s]);
          ++q;
        }
    }
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
      if (j >= nc) continue;
      // element (i0 + l, j) into its accumulator, with its position
      auto elem = [&](int l) -> C {
        if constexpr (DIM == -1)
          return eval_elem<T, RED>(x[w], k, err, l, acc[l], csq[l], i0 + l + j * nr);
        else if constexpr (DIM == 0)
          return eval_elem<T, RED>(x[w], k, err, l, acc[w], csq[w], i0 + l);
        else
          return eval_elem<T, RED>(x[w], k, err, l, acc[l], csq[l], j);
      };
      if (fullr) {
        C y[V];
#pragma unroll
        for (int l = 0; l < V; ++l) y[l] = elem(l);
        if constexpr (OUT) store_rows<S, V>(p, i0, j, y);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l)
          if (i0 + l < nr) {
            C y = elem(l);
            if constexpr (OUT) sstore1<S>(p, at_out_g<S>(p, i0 + l, j), y);
          }
      }
    }
  }
  if constexpr (DIM == -1) {
    if constexpr (RED != RED_NONE) {
#pragma unroll
      for (int l = 1; l < V; ++l) acc[0].merge(acc[l]);
      finish_full<C, RED>(p, acc[0], smem);
    }
  } else if constexpr (DIM == 0) {
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      A a = warp_reduce(acc[w]);  // the block's rows of column 32 strip + ty + 8 w
      if (tx == 0) blk[ty + TILE_PH * w] = a;
    }
    __syncthreads();
    strip_finish<C, RED, TILE>(p, blk, strip, seg, nseg, nc, &am_last);
  } else {
    // rows 32 V strip + V tx + l: combine the 8 column phases, one lane at a time
#pragma unroll
    for (int l = 0; l < V; ++l) {
      rsum[ty][tx] = acc[l];
      __syncthreads();
      if (ty == 0) {
        A a = rsum[0][tx];
        for (int r = 1; r < TILE_PH; ++r) a.merge(rsum[r][tx]);
        blk[tx * V + l] = a;
      }
      __syncthreads();
    }
    strip_finish<C, RED, TM>(p, blk, strip, seg, nseg, nr, &am_last);
  }
  if constexpr (DIM != -1) __syncthreads();  // blk is read by the finish before the next unit writes it
  }  // units
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// scan: cumsum of the tree along dim 0 (down each column) or dim 1 (along
// each row), written to the output in the storage type.
//   Each scan line is cut into n_splits segments.  With one segment a single
//   launch scans; with several, a first launch (PASS 1) writes each
//   segment's total to the partials and the scan (PASS 2) starts each
//   segment from the sum of the totals before it, in segment order.
//   dim 0: a warp per (column, segment), 32 V rows per step: each lane sums
//   its V values, a warp scan of the lane totals gives every lane its start,
//   the step total carries to the next step.  dim 1: a thread per V rows of
//   a (row block, segment), walking the segment's columns in order.
// Running sums: float-float for FP32 compute (the output is hi + lo rounded
// once), plain FP64, wrapping INT32.
// ---------------------------------------------------------------------------
template <class C> struct ScanAcc;
template <> struct ScanAcc<float> {
  float hi, lo;
  __device__ __forceinline__ void init() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add(const ScanAcc& o) {
    add(o.hi);
    lo = __fadd_rn(lo, o.lo);
  }
  __device__ __forceinline__ float out() const {
    return (hi - hi == 0.f) ? __fadd_rn(hi, lo) : hi;  // inf / NaN as they are
  }
  __device__ __forceinline__ ScanAcc shfl_up(int d) const {
    ScanAcc o;
    o.hi = __shfl_up_sync(0xffffffffu, hi, d);
    o.lo = __shfl_up_sync(0xffffffffu, lo, d);
    return o;
  }
  __device__ __forceinline__ ScanAcc shfl_xor(int m) const {
    ScanAcc o;
    o.hi = __shfl_xor_sync(0xffffffffu, hi, m);
    o.lo = __shfl_xor_sync(0xffffffffu, lo, m);
    return o;
  }
  __device__ __forceinline__ ScanAcc shfl(int src) const {
    ScanAcc o;
    o.hi = __shfl_sync(0xffffffffu, hi, src);
    o.lo = __shfl_sync(0xffffffffu, lo, src);
    return o;
  }
};
template <> struct ScanAcc<double> {
  double s;
  __device__ __forceinline__ void init() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s = __dadd_rn(s, x); }
  __device__ __forceinline__ void add(const ScanAcc& o) { s = __dadd_rn(s, o.s); }
  __device__ __forceinline__ double out() const { return s; }
  __device__ __forceinline__ ScanAcc shfl_up(int d) const { return ScanAcc{__shfl_up_sync(0xffffffffu, s, d)}; }
  __device__ __forceinline__ ScanAcc shfl_xor(int m) const { return ScanAcc{__shfl_xor_sync(0xffffffffu, s, m)}; }
  __device__ __forceinline__ ScanAcc shfl(int src) const { return ScanAcc{__shfl_sync(0xffffffffu, s, src)}; }
};
template <> struct ScanAcc<int> {
  u32 s, pad;
  __device__ __forceinline__ void init() { s = 0u; pad = 0u; }
  __device__ __forceinline__ void add(int x) { s += (u32)x; }
  __device__ __forceinline__ void add(const ScanAcc& o) { s += o.s; }
  __device__ __forceinline__ int out() const { return (int)s; }
  __device__ __forceinline__ ScanAcc shfl_up(int d) const { return ScanAcc{__shfl_up_sync(0xffffffffu, s, d), 0u}; }
  __device__ __forceinline__ ScanAcc shfl_xor(int m) const { return ScanAcc{__shfl_xor_sync(0xffffffffu, s, m), 0u}; }
  __device__ __forceinline__ ScanAcc shfl(int src) const { return ScanAcc{__shfl_sync(0xffffffffu, s, src), 0u}; }
};

template <class T, class S, int NS, int NK, int V, int PASS>
__device__ __forceinline__ void scan_col_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef ScanAcc<C> A;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const int lane = threadIdx.x & 31;
  const long long nr = p.n_rows, nc = p.n_cols, nseg = p.n_splits;
  const long long seg_rows = p.units_per_col * 32LL * V;
  const long long units = nc * nseg;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < units; u += nw) {
    const long long j = u / nseg, sg = u % nseg;
    const long long r0 = sg * seg_rows;
    const long long r1 = (r0 + seg_rows < nr) ? r0 + seg_rows : nr;
    A carry;
    carry.init();
    if constexpr (PASS == 2) {
      for (long long q = 0; q < sg; ++q) carry.add(load_cg(&((const A*)p.partials)[j * nseg + q]));
    }
    for (long long c0 = r0; c0 < r1; c0 += 32LL * V) {
      const long long i = c0 + (long long)lane * V;
      const bool full = (i + V <= r1);
      Vals<C, NS, V> x;
      if (full) {
#pragma unroll
        for (int s = 0; s < NS; ++s) load_rows<S, V>(p, s, i, j, x.v[s]);
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int l = 0; l < V; ++l) x.v[s][l] = (i + l < r1) ? sload1<S>(p, s, at_slot<S>(p, s, i + l, j)) : C(0);
      }
      C y[V];
      A tot;
      tot.init();
#pragma unroll
      for (int l = 0; l < V; ++l) {
        y[l] = (i + l < r1) ? T::ev(x, k, err, l) : C(0);
        tot.add(y[l]);
      }
      // inclusive warp scan of the lane totals (lanes in order)
      A inc = tot;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        A o = inc.shfl_up(d);
        if (lane >= d) {
          o.add(inc);
          inc = o;
        }
      }
      const A step_total = inc.shfl(31);
      if constexpr (PASS == 2) {
        A run = inc.shfl_up(1);  // exclusive: the lanes before this one
        if (lane == 0) run.init();
        A base = carry;
        base.add(run);
        C out[V];
#pragma unroll
        for (int l = 0; l < V; ++l) {
          base.add(y[l]);
          out[l] = base.out();
        }
        if (full)
          store_rows<S, V>(p, i, j, out);
        else
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (i + l < r1) sstore1<S>(p, at_out_g<S>(p, i + l, j), out[l]);
      }
      carry.add(step_total);
    }
    if constexpr (PASS == 1) {
      if (lane == 0) ((A*)p.partials)[j * nseg + sg] = carry;
    }
  }
  if (err) atomicOr(p.err_flag, err);
}

template <class T, class S, int NS, int NK, int V, int U, int PASS>
__device__ __forceinline__ void scan_row_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef ScanAcc<C> A;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long nrb = p.n_row_blocks, nseg = p.n_splits, cps = p.units_per_col;
  const long long rb = blockIdx.x % nrb, sg = blockIdx.x / nrb;
  const long long i = (rb * blockDim.x + threadIdx.x) * V;
  const long long j0 = sg * cps;
  const long long j1 = (j0 + cps < nc) ? j0 + cps : nc;
  const bool fullv = (i + V <= nr);
  if (i >= nr) return;
  A run[V];
#pragma unroll
  for (int l = 0; l < V; ++l) {
    run[l].init();
    if constexpr (PASS == 2)
      if (i + l < nr && !(p.flags & PF_SEGMENTED))
        for (long long q = 0; q < sg; ++q) run[l].add(load_cg(&((const A*)p.partials)[q * nr + i + l]));
  }
  for (long long jb = j0; jb < j1; jb += U) {
    Vals<C, NS, V> x[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long j = jb + g;
      if (j < j1) {
        if (fullv) {
#pragma unroll
          for (int s = 0; s < NS; ++s) load_rows<S, V>(p, s, i, j, x[g].v[s]);
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < V; ++l)
              x[g].v[s][l] = (i + l < nr) ? sload1<S>(p, s, at_slot<S>(p, s, i + l, j)) : C(0);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long j = jb + g;
      if (j < j1) {
        C out[V];
#pragma unroll
        for (int l = 0; l < V; ++l) {
          if (i + l < nr) run[l].add(T::ev(x[g], k, err, l));  // rows past the end are not evaluated
          out[l] = run[l].out();
        }
        if constexpr (PASS == 2) {
          if (fullv)
            store_rows<S, V>(p, i, j, out);
          else
#pragma unroll
            for (int l = 0; l < V; ++l)
              if (i + l < nr) sstore1<S>(p, at_out_g<S>(p, i + l, j), out[l]);
        }
      }
    }
  }
  if constexpr (PASS == 1) {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < nr) ((A*)p.partials)[sg * nr + i + l] = run[l];
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// scanp: cumsum along dim 1 in one pass.  A block owns a band of 32 V rows
// (lane = V rows) and walks the columns in panels of NW x UC: warp w takes
// UC consecutive columns of the panel, evaluates the tree there and forms its
// rows' partial sums; the partials go to shared memory, and after one block
// barrier warp w starts from the band's carry plus the partials of warps
// 0 .. w-1, in that order, and writes its columns.  The last warp forms the
// next panel's carry.  Every row is read and written once and no block waits
// on another; the order of additions is fixed by (V, UC, NW), so results are
// deterministic.  The next panel's loads are issued before the barrier.
// Transposed slots (TRMASK, V = 1) and a transposed output (a general output
// of column stride 1) have each row's UC columns consecutive in memory; in a
// band whose 32 rows are all inside the tree a warp moves those runs together
// through its tile in shared memory (scanp_load / scanp_unstage / scanp_write).
// ---------------------------------------------------------------------------
// the UC columns from c0 of every slot at this thread's rows.  FULL: all V
// rows and all UC columns are inside the tree (no checks); else rows at or
// past nr read 0 and columns at or past nc are not read.  A transposed slot
// (bit s of TRMASK; V = 1) has its columns one element apart: the thread's
// UC values are consecutive in memory, read as 16-byte vectors when the host
// found them aligned (flag PF_TRUN0 << s).
template <bool FULL, int TRMASK, class S, int NS, int V, int UC, class X>
__device__ __forceinline__ void scanp_load(const Params& p, const S* const (&rp)[NS], long long i, long long c0,
                                           long long nr, long long nc, X (&x)[UC], bool coop, long long i0) {
  typedef typename X::C C;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if ((TRMASK >> s) & 1) {
      static_assert(TRMASK == 0 || V == 1, "transposed slots: one row per thread");
      const S* q = rp[s] + c0;
      constexpr int PER = 16 / (int)sizeof(S);
      constexpr int CPR = UC / PER > 0 ? UC / PER : 1;  // 16-byte pieces of a row's run
      if (FULL && UC % PER == 0 && 32 % CPR == 0 && coop && (p.flags & (PF_TRUN0 << s))) {
        // the warp reads the band's runs together: lanes CPR apart take
        // consecutive pieces of one row, so a load instruction covers
        // 32 / CPR whole runs; x[] holds the pieces until scanp_unstage
        // hands every lane its own row
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int g = 0; g < CPR; ++g) {
          const long long row = i0 + g * (32 / CPR) + lane / CPR;
          const S* qq = (const S*)p.src[s] + row * p.rs[s] + c0 + (lane % CPR) * PER;
          C t[PER];
          if (slot_ok<S>(p, s, qq, PER)) {
            IO<S>::template load<PER>(qq, t);
          } else {
#pragma unroll
            for (int e = 0; e < PER; ++e) t[e] = C(0);
          }
#pragma unroll
          for (int e = 0; e < PER; ++e) x[g * PER + e].v[s][0] = t[e];
        }
      } else if (FULL && UC % PER == 0 && (p.flags & (PF_TRUN0 << s)) && slot_ok<S>(p, s, q, UC)) {
#pragma unroll
        for (int g = 0; g < UC / PER; ++g) {
          C t[PER];
          IO<S>::template load<PER>(q + g * PER, t);
#pragma unroll
          for (int e = 0; e < PER; ++e) x[g * PER + e].v[s][0] = t[e];
        }
      } else {
#pragma unroll
        for (int u = 0; u < UC; ++u)
          if (FULL || (c0 + u < nc && i < nr)) x[u].v[s][0] = sload1<S>(p, s, q + u);
      }
      continue;
    }
    const long long ld = p.ld[s];
    const S* q = rp[s] + c0 * ld;
#pragma unroll
    for (int u = 0; u < UC; ++u, q += ld) {
      if constexpr (FULL) {
        rows_from<S, V>(p, s, q, x[u].v[s]);
      } else if (c0 + u < nc) {
#pragma unroll
        for (int l = 0; l < V; ++l)
          x[u].v[s][l] = (i + l < nr) ? sload1<S>(p, s, gen_slot(s) ? q + l * p.rs[s] : q + l) : C(0);
      }
    }
  }
}

// The pieces of the cooperatively read transposed slots go through the warp's
// shared-memory tile (32 rows of UC values, rows padded by 16 bytes), and
// every lane takes back its own row's UC values.  Called with the whole warp
// (the cooperative form is uniform over it).
template <int TRMASK, class S, int NS, int UC, class X>
__device__ __forceinline__ void scanp_unstage(const Params& p, X (&x)[UC], typename X::C* tile) {
  typedef typename X::C C;
  constexpr int PER = 16 / (int)sizeof(S), CPR = UC / PER > 0 ? UC / PER : 1;
  constexpr int GC = 16 / (int)sizeof(C), TRS = UC + GC;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (!((TRMASK >> s) & 1) || !(p.flags & (PF_TRUN0 << s))) continue;
    __syncwarp();
#pragma unroll
    for (int g = 0; g < CPR; ++g) {
      C* d = tile + (g * (32 / CPR) + lane / CPR) * TRS + (lane % CPR) * PER;
#pragma unroll
      for (int e0 = 0; e0 < PER; e0 += GC) {
        C v[GC];
#pragma unroll
        for (int e = 0; e < GC; ++e) v[e] = x[g * PER + e0 + e].v[s][0];
        sts_group<C, GC>(d + e0, v);
      }
    }
    __syncwarp();
    C r[UC];
    lds_vec<C, UC>(tile + lane * TRS, r);
#pragma unroll
    for (int u = 0; u < UC; ++u) x[u].v[s][0] = r[u];
  }
}

// One panel of warp w in two halves around the block barrier, which stays in
// scanp_kernel: a thread takes the checked (FULL = false) or the unchecked
// form of each half by its own rows and columns, so the forms may differ
// between the lanes of a warp and neither half may hold a barrier.
// First half: evaluate the tree on the loaded columns, form the rows' partial
// sums, issue the next panel's loads, publish the partial sums.
template <bool FULL, int TRMASK, class T, class S, int NS, int V, int UC, int NW, class X, class K, class C>
__device__ __forceinline__ void scanp_eval(const Params& p, const K& k, u32& err, X (&x)[UC], C (&y)[UC][V],
                                           ScanAcc<C> (&agg)[V], ScanAcc<C> (&aggs)[NW][32 * V], bool more,
                                           bool more_full, const S* const (&rp)[NS], long long i, long long c0,
                                           long long nr, long long nc, bool coop, bool more_coop, long long i0,
                                           C* tile) {
  constexpr int PW = NW * UC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if constexpr (FULL && TRMASK != 0 && V == 1 && UC % (16 / (int)sizeof(S)) == 0) {
    if (coop) scanp_unstage<TRMASK, S, NS, UC>(p, x, tile);
  }
#pragma unroll
  for (int l = 0; l < V; ++l) agg[l].init();
#pragma unroll
  for (int u = 0; u < UC; ++u)
#pragma unroll
    for (int l = 0; l < V; ++l) {
      if (FULL || ((c0 + u < nc) && (i + l < nr))) {
        y[u][l] = T::ev(x[u], k, err, l);
        agg[l].add(y[u][l]);
      } else {
        y[u][l] = C(0);
      }
    }
  if (more) {
    if (more_full)
      scanp_load<true, TRMASK, S, NS, V, UC>(p, rp, i, c0 + PW, nr, nc, x, more_coop, i0);
    else if (i < nr)
      scanp_load<false, TRMASK, S, NS, V, UC>(p, rp, i, c0 + PW, nr, nc, x, false, i0);
  }
#pragma unroll
  for (int l = 0; l < V; ++l) aggs[w][lane * V + l] = agg[l];
}

// Second half: start from the band's carry plus the partial sums of the warps
// before this one (in warp order), write the panel's columns; the last warp
// forms the next panel's carry.
template <bool FULL, class S, int V, int UC, int NW, class C>
__device__ __forceinline__ void scanp_write(const Params& p, const C (&y)[UC][V], const ScanAcc<C> (&agg)[V],
                                            const ScanAcc<C> (&aggs)[NW][32 * V], const ScanAcc<C> (&carry_in)[32 * V],
                                            ScanAcc<C> (&carry_out)[32 * V], S* op, long long i, long long c0,
                                            long long nr, long long nc, bool coop, long long i0, C* tile) {
  typedef ScanAcc<C> A;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  A base[V];
#pragma unroll
  for (int l = 0; l < V; ++l) {
    base[l] = carry_in[lane * V + l];
    for (int q = 0; q < w; ++q) base[l].add(aggs[q][lane * V + l]);
  }
  if (w == NW - 1) {
#pragma unroll
    for (int l = 0; l < V; ++l) {
      A nx = base[l];
      nx.add(agg[l]);
      carry_out[lane * V + l] = nx;
    }
  }
  if (!FULL && i >= nr) return;
  const long long old = p.out_ld;
  S* o = op + c0 * old;
  constexpr int PER = 16 / (int)sizeof(S);
  if constexpr (V == 1 && UC % PER == 0 && (COOT_GM & GM_OUT) != 0) {
    constexpr int CPR = UC / PER, GC = 16 / (int)sizeof(C), TRS = UC + GC;
    if constexpr (FULL && 32 % CPR == 0) {
      if (coop && (p.flags & PF_OUT_RUN)) {
        // a transposed output written by the whole warp: every lane puts its
        // row's UC results in the warp's tile, then lanes CPR apart write
        // consecutive 16-byte pieces of one row's run
        C t[UC];
#pragma unroll
        for (int u = 0; u < UC; ++u) {
          base[0].add(y[u][0]);
          t[u] = base[0].out();
        }
        __syncwarp();
#pragma unroll
        for (int g = 0; g < UC / GC; ++g) {
          C v[GC];
#pragma unroll
          for (int e = 0; e < GC; ++e) v[e] = t[g * GC + e];
          sts_group<C, GC>(tile + lane * TRS + g * GC, v);
        }
        __syncwarp();
#pragma unroll
        for (int g = 0; g < CPR; ++g) {
          const int row = g * (32 / CPR) + lane / CPR, ch = lane % CPR;
          C v[PER];
          lds_vec<C, PER>(tile + row * TRS + ch * PER, v);
          S* d = (S*)p.out + (i0 + row) * p.out_rs + c0 * p.out_ld + ch * PER;
          if (out_ok<S>(p, d, PER)) IO<S>::template store<PER>(d, v);
        }
        return;
      }
    }
    // a transposed output: the thread's UC results are consecutive
    if (FULL && (p.flags & PF_OUT_RUN) && out_ok<S>(p, o, UC)) {
#pragma unroll
      for (int g = 0; g < UC / PER; ++g) {
        C t[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) {
          base[0].add(y[g * PER + e][0]);
          t[e] = base[0].out();
        }
        IO<S>::template store<PER>(o + g * PER, t);
      }
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < UC; ++u, o += old) {
    if (!FULL && c0 + u >= nc) break;
    C out[V];
#pragma unroll
    for (int l = 0; l < V; ++l) {
      base[l].add(y[u][l]);
      out[l] = base[l].out();
    }
    if (COOT_GM & GM_OUT) {
#pragma unroll
      for (int l = 0; l < V; ++l)
        if (FULL || i + l < nr) sstore1<S>(p, o + l * p.out_rs, out[l]);
    } else if (FULL) {
      if (out_ok<S>(p, o, V)) IO<S>::template store<V>(o, out);
    } else {
#pragma unroll
      for (int l = 0; l < V; ++l)
        if (i + l < nr) sstore1<S>(p, o + l, out[l]);
    }
  }
}

template <class T, class S, int NS, int NK, int V, int UC, int NW, int TRMASK = 0>
__device__ __forceinline__ void scanp_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef ScanAcc<C> A;
  constexpr int RB = 32 * V, PW = NW * UC;
  __shared__ A aggs[2][NW][RB];
  __shared__ A carry_s[2][RB];
  // a warp's tile for its band's transposed runs (reads and a transposed
  // output): 32 rows of UC values, rows padded by 16 bytes
  constexpr bool STAGE = V == 1 && (TRMASK != 0 || (COOT_GM & GM_OUT) != 0);
  constexpr int TRS = UC + 16 / (int)sizeof(C);
  __shared__ __align__(16) C tiles[STAGE ? NW : 1][STAGE ? 32 * TRS : 4];
  if (blockDim.x != 32 * NW) return;  // the panel needs exactly NW warps (uniform over the block)
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long i = (long long)blockIdx.x * RB + (long long)lane * V;
  const bool fullv = (i + V <= nr);
  if (w == 0) {
#pragma unroll
    for (int l = 0; l < V; ++l) carry_s[0][lane * V + l].init();
  }
  // this thread's first row in column 0 of every slot and of the output
  // (formed only for rows inside the tree)
  const long long ii = (i < nr) ? i : 0;
  const S* rp[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s)
    rp[s] = (const S*)p.src[s] + ((gen_slot(s) || ((TRMASK >> s) & 1)) ? ii * p.rs[s] : ii);
  S* op = (S*)p.out + ((COOT_GM & GM_OUT) ? ii * p.out_rs : ii);
  const long long npan = (nc + PW - 1) / PW;
  C* tile = tiles[STAGE ? w : 0];
  // the band's first row, and whether all its rows are inside the tree (then
  // a warp whose UC columns are inside reads and writes transposed runs
  // together: uniform over the warp)
  const long long i0 = (long long)blockIdx.x * RB;
  const bool band_full = STAGE && (i0 + RB <= nr);
  Vals<C, NS, V> x[UC];
  {
    const long long c0 = (long long)w * UC;
    if (fullv && c0 + UC <= nc)
      scanp_load<true, TRMASK, S, NS, V, UC>(p, rp, i, c0, nr, nc, x, band_full, i0);
    else if (i < nr)
      scanp_load<false, TRMASK, S, NS, V, UC>(p, rp, i, c0, nr, nc, x, false, i0);
  }
  // every thread runs every panel and reaches the one barrier below once per
  // panel, whatever form of the halves it takes
  for (long long pan = 0; pan < npan; ++pan) {
    const int b = (int)(pan & 1);
    const long long c0 = pan * PW + (long long)w * UC;
    const bool full = fullv && (c0 + UC <= nc);
    const bool more = pan + 1 < npan;
    const bool more_full = fullv && (c0 + PW + UC <= nc);
    C y[UC][V];
    A agg[V];
    const bool coop = band_full && full, more_coop = band_full && more_full;
    if (full)
      scanp_eval<true, TRMASK, T, S, NS, V, UC, NW>(p, k, err, x, y, agg, aggs[b], more, more_full, rp, i, c0, nr,
                                                    nc, coop, more_coop, i0, tile);
    else
      scanp_eval<false, TRMASK, T, S, NS, V, UC, NW>(p, k, err, x, y, agg, aggs[b], more, more_full, rp, i, c0, nr,
                                                     nc, false, false, i0, tile);
    __syncthreads();
    if (full)
      scanp_write<true, S, V, UC, NW>(p, y, agg, aggs[b], carry_s[b], carry_s[b ^ 1], op, i, c0, nr, nc, coop, i0,
                                      tile);
    else
      scanp_write<false, S, V, UC, NW>(p, y, agg, aggs[b], carry_s[b], carry_s[b ^ 1], op, i, c0, nr, nc, false, i0,
                                       tile);
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// adj: gradient of L = mult * sum(tree) with respect to every slot
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int V, int U>
__device__ __forceinline__ void adj_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const C g0 = (C)((double)(*(const C*)p.upstream) * p.grad_mult);
  const long long nr = p.n_rows, nc = p.n_cols, cpc = p.units_per_col;
  const long long step = (long long)blockDim.x * V;
  const long long CH = step * U;
  for (UnitWalk walk(cpc); walk.j < nc; walk.next()) {
    const long long j = walk.j;
    const long long i0 = walk.r * CH + (long long)threadIdx.x * V;
    Vals<C, NS, V> x[U];
    bool full[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      full[g] = (i + V <= nr);
      if (full[g]) {
#pragma unroll
        for (int s = 0; s < NS; ++s) load_rows<S, V>(p, s, i, j, x[g].v[s]);
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int l = 0; l < V; ++l) x[g].v[s][l] = (i + l < nr) ? sload1<S>(p, s, at_slot<S>(p, s, i + l, j)) : C(0);
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      C gs[NS][V];
#pragma unroll
      for (int l = 0; l < V; ++l) {
        C gl[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) gl[s] = C(0);
        if (full[g] || i + l < nr) T::bw(x[g], k, err, l, g0, gl);
#pragma unroll
        for (int s = 0; s < NS; ++s) gs[s][l] = gl[s];
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (p.grad[s] == nullptr) continue;
        if (full[g]) {
          IO<S>::template store<V>(at_out<S>(p.grad[s], i, j, p.grad_ld[s]), gs[s]);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (i + l < nr) IO<S>::store1(at_out<S>(p.grad[s], i + l, j, p.grad_ld[s]), gs[s][l]);
        }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// batch: persistent kernel over the 32x32 tiles of many problems, one warp
// per tile.  Every warp takes `chunk` consecutive tiles at a time from an
// atomic queue (the next pop is issued before the current chunk is worked
// on, so its latency is hidden) and synchronises only with itself: a
// transposed read goes through the warp's own padded shared-memory tile.
// A problem's tiles inside one chunk are accumulated in registers and
// flushed once -- a problem whose tiles all lie in one chunk writes its
// result directly; otherwise each flush leaves one partial per tile range and
// the flush that completes the problem combines its partials in tile order.
// Chunks start at multiples of `chunk`, so the grouping -- and the result --
// does not depend on which warp took which chunk.
// ---------------------------------------------------------------------------
constexpr int BATCH_WARPS = 8;  // warps per block when shared memory allows
constexpr int BATCH_COLS = 16;  // tile columns loaded per step

// warps per block: each warp owns NTR padded tiles of the compute type, and
// the block's static shared memory stays within 48 KiB (the host launches
// blockDim.x = 32 * batch_warps)
template <int NTR, int CSIZE> struct BatchWarps {
  static constexpr int per = TILE * (TILE + 1) * CSIZE * (NTR > 0 ? NTR : 1);
  static constexpr int fit = 49152 / per;
  static constexpr int value = NTR == 0 ? BATCH_WARPS : (fit < 1 ? 1 : (fit > BATCH_WARPS ? BATCH_WARPS : fit));
};

template <class C, class A>
__device__ __forceinline__ void batch_write(const BatchParams& bp, long long p, const A& a, long long count) {
  typedef typename rtype<C>::type R;
  if constexpr (is_int_c<C>::value) {
    ((long long*)bp.red_out)[p] = a.ivalue();
  } else {
    double v = a.value();
    if (bp.mean) v /= (double)count;
    ((R*)bp.red_out)[p] = (R)v;
  }
}

template <class C, class A>
__device__ __forceinline__ void batch_flush(const BatchParams& bp, long long p, long long ta, long long tb, A acc) {
  const int lane = threadIdx.x & 31;
  acc = warp_reduce(acc);  // every lane holds the sum
  const BatchProblem& pr = bp.probs[p];
  const long long ntile = bp.tile_begin[p + 1] - pr.tile_begin;
  const long long count = pr.n_rows * pr.n_cols;
  if (tb - ta == ntile) {  // the whole problem is in this group
    if (lane == 0) batch_write<C>(bp, p, acc, count);
    return;
  }
  A zero;
  zero.init();
  for (long long t = ta + 1 + lane; t < tb; t += 32) ((A*)bp.partials)[t] = zero;
  if (lane == 0) ((A*)bp.partials)[ta] = acc;
  __threadfence();
  __syncwarp();
  unsigned int d = 0;
  if (lane == 0) d = atomicAdd(&bp.done[p], (unsigned int)(tb - ta));
  d = __shfl_sync(0xffffffffu, d, 0);
  if ((long long)d + (tb - ta) == ntile) {
    __threadfence();
    A a;
    a.init();
    for (long long s = lane; s < ntile; s += 32) a.merge(load_cg(&((const A*)bp.partials)[pr.tile_begin + s]));
    a = warp_reduce(a);
    if (lane == 0) {
      batch_write<C>(bp, p, a, count);
      bp.done[p] = 0u;
    }
  }
}

template <class T, class S, int NS, int NK, int TRMASK, bool RED>
__device__ __forceinline__ void batch_kernel(const BatchParams bp) {
  typedef typename ctype<S>::type C;
  typedef typename AccOf<C>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  constexpr int BW = BatchWarps<NTR, (int)sizeof(C)>::value;
  __shared__ C stage_all[BW][NTR > 0 ? NTR : 1][TILE][TILE + 1];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(bp.k[q]);
  typename CsqOf<C>::type csq;
  u32 err = 0;
  const int tx = threadIdx.x & 31, wid = threadIdx.x >> 5;
  C (*stage)[TILE][TILE + 1] = stage_all[wid];
  unsigned int pop = 0;
  if (tx == 0) pop = atomicAdd(&bp.queue[0], (unsigned int)bp.chunk);
  long long t0 = (long long)__shfl_sync(0xffffffffu, pop, 0);
  while (t0 < bp.n_tiles) {
    unsigned int nxt = 0;
    if (tx == 0) nxt = atomicAdd(&bp.queue[0], (unsigned int)bp.chunk);  // used after the chunk
    const long long t1 = (t0 + bp.chunk < bp.n_tiles) ? t0 + bp.chunk : bp.n_tiles;
    // the chunk's owning problems, one lane per tile (chunk <= 32)
    const int myp = (t0 + tx < t1) ? bp.tile_prob[t0 + tx] : 0;
    A acc;
    acc.init();
    long long cur = -1, gfirst = t0;
    for (long long t = t0; t < t1; ++t) {
      const long long p = __shfl_sync(0xffffffffu, myp, (int)(t - t0));
      if constexpr (RED) {
        if (p != cur && cur >= 0) {
          batch_flush<C>(bp, cur, gfirst, t, acc);
          acc.init();
          gfirst = t;
        }
      }
      cur = p;
      // the problem record in registers: the tile's stores to Y could alias
      // it as far as the compiler knows, which would reload every field
      const BatchProblem pr = bp.probs[p];
      const long long nr = pr.n_rows, nc = pr.n_cols;
      const long long lt = t - pr.tile_begin;
      const long long ti = lt % pr.n_tile_rows, tj = lt / pr.n_tile_rows;
      const long long r0 = ti * TILE, c0 = tj * TILE;
      const int nrows = (int)((nr - r0 < TILE) ? nr - r0 : TILE);  // warp-uniform extents
      const int ncols = (int)((nc - c0 < TILE) ? nc - c0 : TILE);
      if constexpr (NTR > 0) {
        // stage the transposed blocks: view(c0 + tx, r0 + m) -> stage[q][m][tx]
        int q = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if ((TRMASK >> s) & 1) {
            // 32 loads in flight per lane, then 32 shared stores
            for (int m0 = 0; m0 < nrows; m0 += 32) {
              C v[32];
#pragma unroll
              for (int u = 0; u < 32; ++u)
                v[u] = (tx < ncols && m0 + u < nrows) ? IO<S>::load1(at<S>(pr.src[s], c0 + tx, r0 + m0 + u, pr.ld[s]))
                                                      : C(0);
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (m0 + u < nrows) stage[q][m0 + u][tx] = v[u];
            }
            ++q;
          }
        __syncwarp();
      }
      const bool row_ok = tx < nrows;
      for (int jb = 0; jb < ncols; jb += BATCH_COLS) {
        Vals<C, NS, BATCH_COLS> x;
#pragma unroll
        for (int jj = 0; jj < BATCH_COLS; ++jj) {
          const bool ok = row_ok && (jb + jj < ncols);
          int q = 0;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if ((TRMASK >> s) & 1) {
              x.v[s][jj] = ok ? stage[q][tx][jb + jj] : C(0);
              ++q;
            } else {
              x.v[s][jj] = ok ? IO<S>::load1(at<S>(pr.src[s], r0 + tx, c0 + jb + jj, pr.ld[s])) : C(0);
            }
          }
        }
#pragma unroll
        for (int jj = 0; jj < BATCH_COLS; ++jj) {
          if (row_ok && jb + jj < ncols) {
            C y = eval_elem<T, RED ? RED_SUM : RED_NONE>(x, k, err, jj, acc, csq, 0);
            if (bp.has_out) IO<S>::store1(at_out<S>(pr.out, r0 + tx, c0 + jb + jj, pr.out_ld), y);
          }
        }
      }
      if constexpr (NTR > 0) __syncwarp();  // stage reads done before the next tile
    }
    if constexpr (RED) {
      if (cur >= 0) batch_flush<C>(bp, cur, gfirst, t1, acc);
    }
    t0 = (long long)__shfl_sync(0xffffffffu, nxt, 0);
  }
  if (err) atomicOr(bp.err_flag, err);
  // the last warp out resets the queue for the next launch
  if (tx == 0) {
    unsigned int e = atomicAdd(&bp.queue[1], 1u);
    if (e == gridDim.x * (blockDim.x >> 5) - 1) {
      bp.queue[0] = 0u;
      bp.queue[1] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// batchf: persistent kernel over work items (rectangles of one problem each,
// see BatchItem), one block per item at a time.  The block's 8 worker warps
// first copy the item's block of every transposed slot into shared memory
// (coalesced runs along the source's columns, stored with an odd row stride
// so that both the stores and the later reads are free of bank conflicts),
// then walk the item's elements in column-major order -- consecutive threads
// on consecutive rows, so direct slots and the output are read and written in
// coalesced runs, U elements per thread in flight.  A ninth warp meanwhile
// pops the next item from the queue and loads its records (item, problem
// pointers and strides) into the other half of a double buffer, so workers
// never wait on that chain of dependent loads.  The block's sum of the item
// is one partial; a problem with one item writes its result directly,
// otherwise the block that completes the problem (a per-problem counter)
// combines the partials in item order.
// ---------------------------------------------------------------------------
constexpr int BATCHF_U = 8;

// what the workers need of one item (filled by the fetch warp)
template <int NS> struct BatchfInfo {
  long long idx;  // item index (>= n_items: no more items)
  const void* src[NS];
  long long ld[NS];
  void* out;
  long long out_ld;
  long long count;  // elements of the problem (mean)
  int q, i0, j0, h, w, nk, first;
  unsigned mh, mw;
  int dih, djh, diw, djw;
};

template <int NS>
__device__ __forceinline__ void batchf_fetch(const BatchParams& bp, BatchfInfo<NS>& f, int lane) {
  unsigned int pop = 0;
  if (lane == 0) pop = atomicAdd(&bp.queue[0], 1u);
  const long long idx = (long long)__shfl_sync(0xffffffffu, pop, 0);
  if (lane == 0) f.idx = idx;
  if (idx >= bp.n_items) return;
  const BatchItem it = bp.items[idx];
  const BatchProblem& pr = bp.probs[it.q];
  if (lane < NS) {
    f.src[lane] = pr.src[lane];
    f.ld[lane] = pr.ld[lane];
  }
  if (lane == 0) {
    f.out = pr.out;
    f.out_ld = pr.out_ld;
    f.count = pr.n_rows * pr.n_cols;
    f.q = it.q;
    f.i0 = it.i0;
    f.j0 = it.j0;
    f.h = it.h;
    f.w = it.w;
    f.nk = it.nk;
    f.first = it.first;
    f.mh = it.mh;
    f.mw = it.mw;
    f.dih = it.dih;
    f.djh = it.djh;
    f.diw = it.diw;
    f.djw = it.djw;
  }
}

// The element walk of one item by the worker threads.  Thread tid takes
// elements e = tid + NB u in column-major order of the item (row i, column
// j, advanced by additions).  CONTIG: every direct slot and the output hold
// the item's columns back to back (column stride h, first row 0), so element
// e of a slot is base + e; otherwise a pointer per slot and for the output
// follows (i, j).  The walk takes U = 8 elements per thread per step while 8
// remain, then one step each of 4, 2 and 1 as needed, so no step carries
// elements that are switched off.
template <bool CONTIG, int NS, class S> struct BatchfPos {
  int e, i, si;
  const S* ps[CONTIG ? 1 : NS];
  S* po;
};

template <int U, bool CONTIG, int BE, class T, class S, int NS, int TRMASK, bool RED, class C, class K, class A,
          class Q>
__device__ __forceinline__ void batchf_step(const BatchParams& bp, const S* const (&src)[NS],
                                            const long long (&ld)[NS], S* out, long long out_ld, int h, int di,
                                            int dj, int ds, int dw, BatchfPos<CONTIG, NS, S>& p, const C* stage,
                                            const K& k, A& acc, const Q& csq, u32& err) {
  constexpr int NB = BATCHF_BLOCK;
  Vals<C, NS, U> x;
  S* og[CONTIG ? 1 : U];
#pragma unroll
  for (int g = 0; g < U; ++g) {
    const int eg = p.e + g * NB;
    if constexpr (!CONTIG) og[g] = p.po;
    int q = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if ((TRMASK >> s) & 1) {
        x.v[s][g] = stage[q * BE + p.si];
        ++q;
      } else if constexpr (CONTIG) {
        x.v[s][g] = IO<S>::load1(src[s] + eg);
      } else {
        x.v[s][g] = IO<S>::load1(p.ps[s]);
      }
    }
    p.i += di;
    p.si += ds;
    const bool wrap = p.i >= h;
    if (wrap) {
      p.i -= h;
      p.si += dw;
    }
    if constexpr (!CONTIG) {
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (!((TRMASK >> s) & 1)) p.ps[s] += di + dj * ld[s] + (wrap ? ld[s] - h : 0);
      p.po += di + dj * out_ld + (wrap ? out_ld - h : 0);
    }
  }
#pragma unroll
  for (int g = 0; g < U; ++g) {
    C y = eval_elem<T, RED ? RED_SUM : RED_NONE>(x, k, err, g, acc, csq, 0);
    if (bp.has_out) {
      if constexpr (CONTIG)
        IO<S>::store1(out + (p.e + g * NB), y);
      else
        IO<S>::store1(og[g], y);
    }
  }
  p.e += U * NB;
}

template <bool CONTIG, int BE, class T, class S, int NS, int TRMASK, bool RED, class C, class K, class A, class Q,
          class F>
__device__ __forceinline__ void batchf_walk(const BatchParams& bp, const S* const (&src)[NS], const long long (&ld)[NS],
                                            S* out, long long out_ld, const F& f, int n, int sst, const C* stage,
                                            const K& k, A& acc, const Q& csq, u32& err) {
  constexpr int NB = BATCHF_BLOCK;
  const int h = f.h, di = f.dih, dj = f.djh;
  // the staged index j sst + i moves with (i, j): + dj sst + di, and
  // sst - h more when i wraps into the next column
  const int ds = dj * sst + di, dw = sst - h;
  BatchfPos<CONTIG, NS, S> p;
  p.e = threadIdx.x;
  const int j = (int)(((unsigned long long)(unsigned)p.e * f.mh) >> 24);
  p.i = p.e - j * h;
  p.si = j * sst + p.i;
  if constexpr (!CONTIG) {
#pragma unroll
    for (int s = 0; s < NS; ++s) p.ps[s] = src[s] + ((long long)p.i + (long long)j * ld[s]);
    p.po = out + ((long long)p.i + (long long)j * out_ld);
  }
  constexpr int UM = CONTIG ? BATCHF_U : BATCHF_U / 2;  // the general walk keeps a pointer per element
  while (p.e + (UM - 1) * NB < n)
    batchf_step<UM, CONTIG, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, out_ld, h, di, dj, ds, dw, p, stage, k, acc,
                                                       csq, err);
  if (UM > 4 && p.e + 3 * NB < n)
    batchf_step<4, CONTIG, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, out_ld, h, di, dj, ds, dw, p, stage, k, acc,
                                                      csq, err);
  if (p.e + NB < n)
    batchf_step<2, CONTIG, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, out_ld, h, di, dj, ds, dw, p, stage, k, acc,
                                                      csq, err);
  if (p.e < n)
    batchf_step<1, CONTIG, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, out_ld, h, di, dj, ds, dw, p, stage, k, acc,
                                                      csq, err);
}

template <class T, class S, int NS, int NK, int TRMASK, bool RED, int BE>
__device__ __forceinline__ void batchf_kernel(const BatchParams bp) {
  typedef typename ctype<S>::type C;
  typedef typename AccOf<C>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  constexpr int NB = BATCHF_BLOCK;
  constexpr int SU = 4;  // staging loads in flight per thread
  __shared__ C stage[NTR > 0 ? NTR * BE : 1];
  __shared__ A smem[32];
  __shared__ BatchfInfo<NS> info[2];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(bp.k[q]);
  typename CsqOf<C>::type csq;
  u32 err = 0;
  const int tid = threadIdx.x;
  const bool worker = tid < NB;
  if (tid >= NB) batchf_fetch<NS>(bp, info[0], tid - NB);
  __syncthreads();
  int cur = 0;
  while (info[cur].idx < bp.n_items) {
    const BatchfInfo<NS>& f = info[cur];
    const long long it = f.idx;
    const int h = f.h, w = f.w, n = h * w, i0 = f.i0, j0 = f.j0;
    const int sst = h | 1;  // odd row stride of the staged blocks
    if (!worker) batchf_fetch<NS>(bp, info[cur ^ 1], tid - NB);  // the next item, while this one runs
    if constexpr (NTR > 0) {
      // staged element (jj, ii) = view(j0 + jj, i0 + ii) = src[(j0 + jj) + (i0 + ii) ld]
      if (worker && n > 0) {
        const int dj = f.diw, di = f.djw;
        int q = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if ((TRMASK >> s) & 1) {
            const S* b = (const S*)f.src[s] + j0;
            const long long lds = f.ld[s];
            int e = tid, ii = (int)(((unsigned long long)(unsigned)e * f.mw) >> 24), jj = e - ii * w;
            // SU loads in flight per step while SU elements remain, then one at a time
            for (; e + (SU - 1) * NB < n; e += SU * NB) {
              C v[SU];
              int pj[SU], pi[SU];
#pragma unroll
              for (int g = 0; g < SU; ++g) {
                pj[g] = jj;
                pi[g] = ii;
                v[g] = IO<S>::load1(b + (jj + (long long)(i0 + ii) * lds));
                jj += dj;
                ii += di;
                if (jj >= w) {
                  jj -= w;
                  ++ii;
                }
              }
#pragma unroll
              for (int g = 0; g < SU; ++g) stage[q * BE + pj[g] * sst + pi[g]] = v[g];
            }
            for (; e < n; e += NB) {
              stage[q * BE + jj * sst + ii] = IO<S>::load1(b + (jj + (long long)(i0 + ii) * lds));
              jj += dj;
              ii += di;
              if (jj >= w) {
                jj -= w;
                ++ii;
              }
            }
            ++q;
          }
      }
      __syncthreads();
    }
    A acc;
    acc.init();
    if (worker && n > 0) {
      // contiguous item: every direct slot and the output have column stride h
      // and the item starts at row 0
      bool contig = (i0 == 0) && (!bp.has_out || f.out_ld == h);
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (!((TRMASK >> s) & 1)) contig = contig && f.ld[s] == h;
      // every slot and the output from the item's first element (i0, j0)
      const S* src[NS];
      long long ld[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        ld[s] = f.ld[s];
        src[s] = (const S*)f.src[s] + ((long long)i0 + (long long)j0 * ld[s]);
      }
      S* out = (S*)f.out + ((long long)i0 + (long long)j0 * f.out_ld);
      if (contig)
        batchf_walk<true, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, f.out_ld, f, n, sst, stage, k, acc, csq, err);
      else
        batchf_walk<false, BE, T, S, NS, TRMASK, RED>(bp, src, ld, out, f.out_ld, f, n, sst, stage, k, acc, csq, err);
    }
    if constexpr (RED) {
      acc = block_reduce(acc, smem);  // every lane of warp 0 holds the block's sum
      if (tid < 32) {
        if (f.nk == 1) {
          if (tid == 0) batch_write<C>(bp, f.q, acc, f.count);
        } else {
          unsigned int d = 0;
          if (tid == 0) {
            ((A*)bp.partials)[it] = acc;
            __threadfence();
            d = atomicAdd(&bp.done[f.q], 1u);
          }
          d = __shfl_sync(0xffffffffu, d, 0);
          if (d == (unsigned int)(f.nk - 1)) {  // the problem's last item: combine in item order
            __threadfence();
            A a;
            a.init();
            for (int kk = tid; kk < f.nk; kk += 32) a.merge(load_cg(&((const A*)bp.partials)[f.first + kk]));
            a = warp_reduce(a);
            if (tid == 0) {
              batch_write<C>(bp, f.q, a, f.count);
              bp.done[f.q] = 0u;
            }
          }
        }
      }
    }
    // the next item's records are in place, and nobody reads this item's
    // stage or records any more
    __syncthreads();
    cur ^= 1;
  }
  if (err) atomicOr(bp.err_flag, err);
  // the last block out resets the queue for the next launch
  if (tid == 0) {
    unsigned int e = atomicAdd(&bp.queue[1], 1u);
    if (e == gridDim.x - 1) {
      bp.queue[0] = 0u;
      bp.queue[1] = 0u;
    }
  }
}

}  // namespace coot
