/*
 * oracle.h -- FP64 CPU oracle for Armadillo-style matrix expression trees.
 *
 * TEST INFRASTRUCTURE ONLY.  This evaluator exists so that the tests, the
 * smoke check and the CPU-baseline leg of the benchmark can compare the GPU
 * library against the plain definition of each operation.  The product path
 * never links, loads or calls it, and it shares no code, header or table with
 * the GPU library.
 *
 * What it computes (Bandicoot paper, Sec. 3: an expression is a tree of Op /
 * eOp / Glue / eGlue nodes that is evaluated when assigned; Sec. 4: data is a
 * column-major matrix): the tree is walked one operation at a time, every node
 * materialising a full FP64 (or int64 for INT32 inputs) matrix, and the
 * reduction at the root is applied to the materialised matrix with
 * Neumaier-compensated FP64 summation.
 *
 * Alongside every FP64 value the oracle carries a first-order forward error
 * bound for a device that evaluates the same tree in the compute type
 * (FP32 for FP32/BF16/FP16 storage, FP64 for FP64 storage): each node adds its
 * own allowance (2 ulp of its result for + - * / and the scalar forms, 4 ulp
 * for exp, log and sqrt, 0 for abs, neg, trans and views) and propagates the
 * bounds of its children through the node's derivative.  For a single-op tree
 * the bound is exactly the per-op ulp allowance.
 *
 * Program format (a reverse-Polish token string, whitespace separated):
 *   A..H              push leaf 0..7
 *   #<number>         push a scalar (converted to the element type, as an
 *                     Armadillo scalar of type eT is)
 *   + - % /           element-wise binary op on two matrices; with one scalar
 *                     operand:  k+X X+k  X-k k-X  X/k k/X
 *   *                 scalar times matrix (k*X or X*k); matrix*matrix is not
 *                     element-wise and is rejected
 *   neg exp log abs square sqrt trans
 *   submat:r0:c0:nr:nc   view of the matrix on top (0-based first row/col,
 *                        number of rows/cols)
 *   each_col:n  each_row:n   the column (row) vector on top repeated n times
 *                        (the operand of X.each_col() / X.each_row())
 *   diag  diag:k         diagonal k of the matrix on top as a column vector
 *   mm                   matrix product of the two matrices on top (x y)
 * Optionally one final reduction token:
 *   accu  sum:0 sum:1  mean mean:0 mean:1  dot (pops two matrices)
 *   norm (vector 2-norm)  norm:fro  var var:1 (norm_type 0 -> N-1, 1 -> N)
 *   min max index_min index_max prod  (all elements; index is the column-major
 *                     linear index)  and  min:D max:D index_min:D index_max:D
 *                     prod:D  along dimension D (0: per column, 1: per row)
 *   stddev stddev:1   vardim:D:N stddevdim:D:N  (N is norm_type as for var)
 *   min/max skip NaN and keep the first of equal values; an empty or all-NaN
 *   range gives NaN (0 for INT32) and index -1.
 * or one final scan, which leaves a matrix of the tree's shape:
 *   cumsum cumsum:0 cumsum:1   prefix sums down each column (0) or along each
 *                     row (1); plain cumsum runs along a vector, else dim 0
 */
#ifndef COOT_ORACLE_H
#define COOT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_F32 = 0, ORC_F64 = 1, ORC_BF16 = 2, ORC_F16 = 3, ORC_I32 = 4 };

/* A host matrix, column-major: element (i,j) at data[i + j*ld]. Not owned. */
typedef struct {
  const void* data;
  int32_t dtype;
  int64_t n_rows, n_cols, ld;
} orc_mat;

enum { ORC_RES_MATRIX = 0, ORC_RES_SCALAR = 1 };

/* Result of orc_eval. Arrays are allocated by the oracle and released by
 * orc_free.  Shapes: a matrix result is n_rows x n_cols (contiguous,
 * column-major); a reduction is a scalar (1x1) or a row/column vector. */
typedef struct {
  int32_t is_int;        /* 1: integer results in iv, 0: FP results in v/b    */
  int32_t is_reduction;  /* 1 if the program ended with a reduction token     */
  int64_t n_rows, n_cols;
  double* v;             /* FP64 values                                       */
  double* b;             /* forward error bound for the compute-type device   */
  int64_t* iv;           /* integer values (INT32 element-wise results are    */
                         /* wrapped to int32; reductions are exact int64)     */
  int32_t div_by_zero;   /* an integer division had a zero divisor            */
  char err[256];         /* message when orc_eval returns non-zero            */
} orc_result;

/* Evaluate `program` over `leaves`.  All leaves must share one dtype.
 * `out_dtype` is the storage type of a matrix result (its final rounding is
 * added to the bound); pass -1 for "same as the leaves".
 * Returns 0 on success, non-zero (and res->err) on a malformed program,
 * a shape mismatch or an unsupported dtype/op combination. */
int orc_eval(const char* program, const orc_mat* leaves, int32_t n_leaves,
             int32_t out_dtype, orc_result* res);

void orc_free(orc_result* res);

/* Gradient of L = accu / sum / mean(tree) with respect to every leaf, in
 * FP64 by reverse mode over the materialised tree (the program ends with
 * "accu", "sum" or "mean").  grads[i] and absgrads[i] are caller-allocated
 * contiguous column-major arrays of leaf i's shape; absgrads receives the
 * same sweep over magnitudes (forward values formed with absolute values,
 * |a| + |b| for a +- b, and derivatives taken from them): the scale of the
 * roundings a device makes along each gradient element.  *loss gets
 * L.  Returns 0, or non-zero with a message in err (256 bytes). */
int orc_grad(const char* program, const orc_mat* leaves, int32_t n_leaves, double** grads, double** absgrads,
             double* loss, char* err);

/* Neumaier-compensated FP64 sum of x[0..n) (exposed for the pin tests). */
double orc_sum_neumaier(const double* x, int64_t n);

/* ulp of |x| in the given floating dtype (spacing of that format at x). */
double orc_ulp(double x, int32_t dtype);

/* Threads the element-wise loops use: 1 in the plain build, the OpenMP
 * thread count in the -fopenmp build. */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
