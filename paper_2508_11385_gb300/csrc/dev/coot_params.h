// coot_params.h -- the one kernel-argument block of every generated kernel.
// Included by the host library (to fill it) and by the device code compiled
// through NVRTC (to read it), so the layout is defined once.
#pragma once

#define COOT_MAX_SLOTS 8
#define COOT_MAX_SCALARS_DEV 16

#if defined(__CUDACC__)
#define COOT_HD __host__ __device__
#else
#define COOT_HD
#endif

namespace coot {

// reduction modes of a kernel pass
enum {
  RED_NONE = 0, RED_SUM = 1, RED_DOT = 2, RED_SSQ = 3, RED_MEAN1 = 4, RED_CSQ = 5,
  RED_MIN = 6, RED_MAX = 7, RED_IMIN = 8, RED_IMAX = 9, RED_PROD = 10
};
// RED_SUM   accu / sum / mean                     sum of y
// RED_DOT   root a%b                              sum of a*b, products kept exactly
// RED_SSQ   norm                                  sum of y*y, products kept exactly
// RED_MEAN1 first pass of var/stddev: sum of y, writes the mean(s) to the workspace
// RED_CSQ   second pass of var/stddev: sum of (y - mean)^2
// RED_MIN / RED_MAX / RED_IMIN / RED_IMAX   extreme value, or its position
// RED_PROD  product of y
COOT_HD constexpr bool red_additive(int r) { return r >= RED_SUM && r <= RED_CSQ; }
COOT_HD constexpr bool red_extreme(int r) { return r >= RED_MIN && r <= RED_IMAX; }

// Params::flags
//   PF_SQRT       var's second pass writes the square root (stddev)
//   PF_SEGMENTED  dim-1 reduction / scan: every column split is its own
//                 segment (no combine across splits; output i + split * n_rows;
//                 positions relative to the segment)
//   PF_OUT_RUN    one-pass row scan with a general output of column stride 1
//                 (a transposed output): each thread's runs of consecutive
//                 columns are 16-byte aligned and written as vectors
//   PF_TRUN0 << s one-pass row scan, transposed slot s: each thread's runs of
//                 consecutive columns are 16-byte aligned and read as vectors
enum { PF_SQRT = 1u, PF_SEGMENTED = 2u, PF_OUT_RUN = 4u, PF_TRUN0 = 256u };

struct Params {
  // leaf reads ("slots"): device address of element (0,0) of the view read
  // and its column stride in elements
  const void* src[COOT_MAX_SLOTS];
  long long ld[COOT_MAX_SLOTS];
  // row strides of general slots (broadcast rows, diagonals, row-strided
  // views): their element (i,j) is src[s] + i*rs[s] + j*ld[s]; other slots
  // have rows one element apart
  long long rs[COOT_MAX_SLOTS];
  // the tree's scalars, bit patterns of the compute type
  unsigned long long k[COOT_MAX_SCALARS_DEV];
  // materialised result Y (nullable) and its column stride
  void* out;
  long long out_ld;
  long long out_rs;  // row stride of a general output (a diagonal), else unused
  // iteration shape (a contiguous tree is walked as one long column)
  long long n_rows, n_cols;
  // kernel-family specific: str -- chunks per column; row -- columns per split
  long long units_per_col;
  // row -- number of column splits; tile -- unused
  long long n_splits;
  // row -- number of row blocks
  long long n_row_blocks;
  // elements reduced (mean / var finals) and divisors
  long long count;
  double div;  // mean: count (or length along dim); sum: 1
  double den;  // var: N-1 or N
  unsigned int flags;  // PF_*
  // reduction result (device) and workspace
  void* red_out;
  void* partials;
  unsigned int* tickets;
  unsigned int* err_flag;
  double* mu;
  // bounds-check build (COOT_DEBUG_BOUNDS): elements addressable from src[s]
  // and from out (the leaf's extent past the slot's first element)
  long long ext[COOT_MAX_SLOTS];
  long long out_ext;
  // adjoint: gradient outputs per slot (nullable) and the upstream scalar
  void* grad[COOT_MAX_SLOTS];
  long long grad_ld[COOT_MAX_SLOTS];
  const void* upstream;
  double grad_mult;  // 1 for accu, 1/N for mean
};

// GEMM with the tree fused onto the product: Y = tree(op(A) op(B), leaves).
// op(A) is m x k, op(B) is k x n, both BF16 or FP16.  ka: op(A)(i,t) at
// a[t + i*lda] (K adjacent), else a[i + t*lda]; kb: op(B)(t,j) at
// b[t + j*ldb], else b[j + t*ldb] (the kernel's template flags).
constexpr int GEMM_TILE = 128;  // output rows and columns per block
struct GemmParams {
  Params p;  // the epilogue: slots, scalars, output (the product is a slot without memory)
  const void* a;
  const void* b;
  long long lda, ldb;
  long long m, n, k;
  int vec;  // 16-byte copies: aligned bases, lda and ldb multiples of 8
  // tcgen05 kernel: TMA descriptors (CUtensorMap, 128 bytes) of op(A) and
  // op(B) as K x rows arrays, and the output tile grid
  alignas(64) unsigned long long tma_a[16];
  alignas(64) unsigned long long tma_b[16];
  long long tiles_m, tiles_n;
};
// tcgen05 kernel: 256 x 256 output tiles (two M = 128 MMAs per K step, one
// for each half of the rows), 64 K values per stage, 3 stages
constexpr int GEMM_TC_BM = 256, GEMM_TC_BN = 256, GEMM_TC_BK = 64, GEMM_TC_STAGES = 3;
constexpr int GEMM_TC_MMA_M = 128;
// threads of the tcgen05 kernel: a producer warp, an MMA warp and 8
// epilogue warps (two per quarter of the tensor-memory lanes, each taking
// half of the accumulator's columns)
constexpr int GEMM_TC_THREADS = 320;
// dynamic shared memory of the tcgen05 kernel: the stages, barriers and
// 1 KiB of slack to align the stages to the 1 KiB swizzle atom
constexpr int GEMM_TC_SMEM = GEMM_TC_STAGES * (GEMM_TC_BM + GEMM_TC_BN) * GEMM_TC_BK * 2 + 256 + 1024;

// Batched evaluation: one record per problem, read by the persistent kernel.
struct BatchProblem {
  const void* src[COOT_MAX_SLOTS];
  long long ld[COOT_MAX_SLOTS];
  // row strides of general slots (broadcast rows, diagonals, row-strided
  // views): their element (i,j) is src[s] + i*rs[s] + j*ld[s]; other slots
  // have rows one element apart
  long long rs[COOT_MAX_SLOTS];
  void* out;
  long long out_ld;
  long long n_rows, n_cols;
  long long tile_begin;  // first global tile index of this problem
  long long n_tile_rows; // tiles along the rows
};

// Work item of the flat batched kernel: a rectangle of one problem's tree,
// rows i0 .. i0+h-1 and columns j0 .. j0+w-1.  Items are listed in problem
// order, a problem's items consecutively (item k of nk, the first at index
// `first`), so a problem's partial results are combined in a fixed order.
// The per-item constants of the walks are computed on the host: a thread
// t < 256 starts at row t % h, column t / h, found as j = (t * mh) >> 24 with
// mh = ceil(2^24 / h) (exact for t < 256 and h < 2^14), and moves by
// (NB % h, NB / h) per step; the staging walk likewise over (w, h).
struct BatchItem {
  int q;
  int i0, j0;
  int h, w;
  int nk;
  int first;
  unsigned mh, mw;
  int dih, djh, diw, djw;
  int pad[3];
};
// Elements of one item: every transposed slot stages its w x h block in
// shared memory with a row stride of h rounded up to odd, and the host keeps
// w * (h | 1) within this count (the blocks of all transposed slots stay
// within 40 KiB of static shared memory; without transposed slots it bounds
// the item's work).  `base` is the count without that limit.
COOT_HD constexpr int batchf_elems(int ntr, int csize, int base = 4096) {
  return (ntr <= 0 || 40960 / (ntr * csize) >= base) ? base : 40960 / (ntr * csize);
}
// worker threads of a block; one more warp fetches the next item's records
constexpr int BATCHF_BLOCK = 256;
constexpr int BATCHF_THREADS = BATCHF_BLOCK + 32;

struct BatchParams {
  const BatchProblem* probs;
  const BatchItem* items;  // flat kernel: the work items
  long long n_items;
  const long long* tile_begin;  // n_problems + 1 prefix of the tile counts
  const int* tile_prob;         // owning problem of every tile
  long long n_problems;
  long long n_tiles;
  long long chunk;              // tiles taken from the queue at a time
  unsigned long long k[COOT_MAX_SCALARS_DEV];
  void* red_out;     // one result per problem (nullable)
  void* partials;    // one accumulator per tile
  unsigned int* done;    // per-problem tile counters (zero between launches)
  unsigned int* queue;   // [0] next tile, [1] exited blocks (zero between launches)
  unsigned int* err_flag;
  double div_unused;
  int has_out;
  int mean;  // divide each problem's sum by its element count
};

}  // namespace coot
