/*
 * coot.h -- C ABI of cootgb: fused evaluation of Armadillo-style matrix
 * expression trees on one GB300 (sm_103a).
 *
 * The computation (Bandicoot paper, Sec. 3): a linear-algebra expression is
 * captured as a tree of Op / eOp / Glue / eGlue nodes and evaluated only when
 * it is assigned (delayed evaluation), so that the whole tree can be mapped
 * onto a minimal set of GPU calls.  Here the element-wise part of a tree, the
 * transposes and submatrix views of its leaves, and the reduction that
 * consumes it are evaluated in one pass by a kernel generated for that tree
 * (two passes for var).  Matrices are column-major device memory (Sec. 2 and
 * Sec. 4: data lives in GPU memory, Armadillo's Mat<eT> layout).
 *
 * Conventions shared by every entry point
 *   - Pointers inside coot_mat are DEVICE pointers; tree descriptors and the
 *     arrays of coot_mat are HOST memory read during the call only.  The
 *     caller owns every matrix and stream; the library never frees them.
 *   - Element (i,j) of a coot_mat is at data[i + j*ld], ld >= n_rows
 *     (ld is ignored when n_cols <= 1); a row stride rs > 1 makes it
 *     data[i*rs + j*ld].
 *   - Every call returns a coot_status and never throws; on failure
 *     coot_last_error() holds a message for the calling thread.
 *   - Launches are asynchronous on the given stream (a cudaStream_t; NULL is
 *     the legacy default stream).  Results are valid once the stream reaches
 *     them.
 *   - Reduction results have the accumulation type of the storage type:
 *     float for F32/BF16/F16, double for F64, int64_t for I32.
 */
#ifndef COOT_H
#define COOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COOT_VERSION_MAJOR 1
#define COOT_VERSION_MINOR 0

#if defined(__GNUC__)
#define COOT_API __attribute__((visibility("default")))
#else
#define COOT_API
#endif

/* cudaStream_t without the CUDA headers (same type). */
typedef struct CUstream_st* coot_stream;

typedef enum {
  COOT_OK = 0,
  COOT_ERR_INVALID = 1,      /* malformed descriptor / argument              */
  COOT_ERR_SHAPE = 2,        /* incompatible matrix dimensions              */
  COOT_ERR_DTYPE = 3,        /* dtype mismatch or op not defined for dtype  */
  COOT_ERR_ALIAS = 4,        /* output overlaps an input in a racy way      */
  COOT_ERR_JIT = 5,          /* NVRTC compile or module load failed         */
  COOT_ERR_OOM = 6,          /* device allocation failed                    */
  COOT_ERR_CUDA = 7,         /* a CUDA runtime call failed                  */
  COOT_ERR_DEVICE_FLAG = 8,  /* a kernel raised a device-side error flag    */
  COOT_ERR_TIMEOUT = 9,      /* reserved; no call returns it: the one kernel
                                that waits (the tcgen05 GEMM, on its own
                                mbarriers) bounds every wait and reports a
                                wait that ran out as device flag
                                COOT_FLAG_WAIT_TIMEOUT instead              */
  COOT_ERR_UNSUPPORTED = 10  /* valid request outside what is implemented   */
} coot_status;

typedef enum { COOT_F32 = 0, COOT_F64 = 1, COOT_BF16 = 2, COOT_F16 = 3, COOT_I32 = 4 } coot_dtype;

/* A column-major matrix (Armadillo Mat<eT>; Col = n_cols 1, Row = n_rows 1). */
typedef struct {
  void* data;       /* device pointer to element (0,0)               */
  int32_t dtype;    /* coot_dtype                                    */
  int32_t rs;       /* row stride in elements: 0 or 1 = adjacent rows
                       (column-major); r > 1 puts element (i,j) at
                       data[i*r + j*ld] -- a diagonal view has r = ld+1.
                       An output with r > 1 must not overlap itself.  */
  int64_t n_rows;
  int64_t n_cols;
  int64_t ld;       /* column stride in elements, >= n_rows for
                       adjacent rows                                  */
} coot_mat;

/* Node kinds (Sec. 3): N_TRANS is Op<T1,op_trans>; the unary and scalar
 * kinds are eOp<T1,eop_type>; N_PLUS..N_DIV are eGlue<T1,T2,eglue_type>
 * (N_SCHUR is Armadillo's element-wise product operator%).  N_SUBMAT is a
 * submatrix view of a leaf; N_EACH_COL / N_EACH_ROW broadcast a vector and
 * N_DIAG takes a diagonal (Sec. 2, views and broadcasting). */
typedef enum {
  COOT_N_LEAF = 0,            /* leaf matrix `leaf`                          */
  COOT_N_SUBMAT = 1,          /* view of node a (an N_LEAF): rows r0..r0+nr-1,
                                 cols c0..c0+nc-1 (0-based)                  */
  COOT_N_TRANS = 2,           /* trans(a)                                    */
  COOT_N_SCAL_TIMES = 3,      /* k * a                                       */
  COOT_N_SCAL_PLUS = 4,       /* a + k                                       */
  COOT_N_SCAL_MINUS_PRE = 5,  /* k - a                                       */
  COOT_N_SCAL_MINUS_POST = 6, /* a - k                                       */
  COOT_N_SCAL_DIV_PRE = 7,    /* k / a                                       */
  COOT_N_SCAL_DIV_POST = 8,   /* a / k                                       */
  COOT_N_PLUS = 9,            /* a + b                                       */
  COOT_N_MINUS = 10,          /* a - b                                       */
  COOT_N_SCHUR = 11,          /* a % b  (element-wise product)               */
  COOT_N_DIV = 12,            /* a / b  (element-wise)                       */
  COOT_N_NEG = 13,            /* -a                                          */
  COOT_N_EXP = 14,
  COOT_N_LOG = 15,
  COOT_N_ABS = 16,
  COOT_N_SQUARE = 17,
  COOT_N_SQRT = 18,
  COOT_N_EACH_COL = 19,       /* a (an n x 1 column) repeated as each of nc
                                 columns: Armadillo's X.each_col() operand  */
  COOT_N_EACH_ROW = 20,       /* a (a 1 x n row) repeated as each of nr rows:
                                 X.each_row()'s operand                     */
  COOT_N_DIAG = 21,           /* diagonal r0 = k of a as a column vector (k > 0
                                 above the main diagonal, k < 0 below):
                                 X.diag(k)                                  */
  COOT_N_COUNT_ = 22
} coot_opcode;

/* One node of a postfix tree.  Operand indices a, b refer to earlier nodes
 * (a, b < own index; unused operands are -1); the root is the last node.
 * Nodes may be shared (a DAG).  The scalar k is converted to the compute
 * type (FP32 for F32/BF16/F16 trees, FP64 for F64, int32 truncation for I32,
 * as an Armadillo scalar of type eT is). */
typedef struct {
  int32_t op;              /* coot_opcode                      */
  int32_t a, b;            /* operand node indices or -1       */
  int32_t leaf;            /* N_LEAF: index into `leaves`      */
  double k;                /* scalar of the N_SCAL_* kinds     */
  int64_t r0, c0, nr, nc;  /* N_SUBMAT view; N_EACH_COL: nc;
                              N_EACH_ROW: nr; N_DIAG: r0 = k   */
} coot_node;

typedef struct {
  int32_t n_nodes;  /* 1 .. COOT_MAX_NODES */
  int32_t reserved;
  const coot_node* nodes;
} coot_tree;

#define COOT_MAX_NODES 64
#define COOT_MAX_LEAVES 8
#define COOT_MAX_SCALARS 16

/* The reduction fused onto the tree (Sec. 2: accu/sum and Armadillo's
 * statistics functions -- mean, var, stddev, min, max, index_min/index_max,
 * prod; Sec. 5 task 1: summation of all elements).  Results have the
 * accumulation type: float for F32/BF16/F16 trees, double for F64, int64 for
 * I32 (sums and products exact modulo 2^64); index kinds are int64 for every
 * dtype.  Along dim 0 there is one result per column, along dim 1 one per
 * row; dim -1 gives one result over all elements (column-major order). */
typedef enum {
  COOT_R_NONE = 0,
  COOT_R_ACCU = 1,     /* sum of all elements -> scalar                           */
  COOT_R_SUM = 2,      /* dim -1: all; 0: per column -> 1 x n_cols; 1: per row    */
  COOT_R_MEAN = 3,     /* as R_SUM divided by the count                           */
  COOT_R_DOT = 4,      /* root must be N_SCHUR a%b: sum of a*b with the products
                          kept exactly (integer: exact int64 products)            */
  COOT_R_NORM2 = 5,    /* vector 2-norm (tree must be a row or column vector)     */
  COOT_R_NORM_FRO = 6, /* Frobenius norm of a matrix                              */
  COOT_R_VAR = 7,      /* two-pass variance (dim -1, 0 or 1); norm_type 0 -> N-1,
                          1 -> N; one element gives 0, none gives NaN; F32/F64  */
  COOT_R_STDDEV = 8,   /* square root of R_VAR                                     */
  COOT_R_MIN = 9,      /* smallest element; NaN elements are skipped; none (or all
                          NaN) gives NaN (0 for I32)                              */
  COOT_R_MAX = 10,     /* largest element, as R_MIN                                */
  COOT_R_INDEX_MIN = 11, /* position of the first smallest element: column-major
                          linear index for dim -1, row index along dim 0, column
                          index along dim 1; -1 when there is none             */
  COOT_R_INDEX_MAX = 12, /* position of the first largest element, as above      */
  COOT_R_PROD = 13,    /* product; no intermediate overflow or underflow (the
                          exponent is carried apart), the result is rounded to
                          the accumulation type; empty gives 1                 */
  COOT_R_CUMSUM = 14   /* not a reduction: the prefix sums of Y along dim (0 down
                          each column, 1 along each row, -1 along a vector or
                          else dim 0) are written to `out` (required, the
                          tree's shape and dtype) instead of Y; red_out is
                          unused.  FP32 compute sums in float-float and rounds
                          each output once; I32 wraps modulo 2^32           */
} coot_red_kind;

typedef struct {
  int32_t kind;      /* coot_red_kind                           */
  int32_t dim;       /* -1 all elements, 0 per column, 1 per row */
  int32_t norm_type; /* R_VAR / R_STDDEV only                   */
  int32_t n_seg;     /* dim 1 only, 0 or 1 = one segment: the columns form
                        n_seg equal segments (n_cols % n_seg == 0), each
                        reduced (or, for cumsum, scanned) on its own: the
                        result is n_rows x n_seg, segment s in column s.
                        A Cube's slices laid side by side are segments
                        (Sec. 2: Cube, collections of matrices).      */
} coot_reduce;

typedef struct coot_ctx coot_ctx;
typedef struct coot_batch coot_batch;
typedef struct coot_graph coot_graph;

/* ---- context -------------------------------------------------------------
 * coot_ctx_create: bind a context to CUDA device `device`.  Defined by Sec. 2
 * (Fig. coot_init): a program optionally picks the backend and the GPU once,
 * at start-up, and may ask for information to be printed; here the backend is
 * always CUDA on sm_103a, `device` is the CUDA device ID and COOT_CTX_LOG is
 * the print-information switch.  The context owns the per-tree kernel cache
 * (in memory and on disk under $COOT_CACHE_DIR, default ~/.cache/cootgb; the
 * cache of run-time compiled kernels is Sec. 4's third difference), the
 * tuning cache and a device workspace that grows on demand.  Returns
 * COOT_ERR_CUDA when the device cannot be used; coot_ctx_destroy releases
 * what the context owns (never caller memory) after synchronising its
 * device.  Flags: */
#define COOT_CTX_TUNE 1u          /* autotune launch configs on first use    */
#define COOT_CTX_NO_DISK_CACHE 2u /* keep compiled kernels in memory only    */
#define COOT_CTX_LOG 4u           /* print JIT / cache / tuning decisions    */
#define COOT_CTX_NO_TCGEN05 8u    /* GEMM: always the mma.sync kernel        */
#define COOT_CTX_DEBUG_BOUNDS 16u /* bounds-check build of the streaming
                                     kernels (str, col, row, tile, scan, adj):
                                     every leaf read and output write is
                                     checked against the extent computed from
                                     its matrix's shape and strides; an access
                                     outside it is skipped (a read gives 0) and
                                     raises COOT_FLAG_OUT_OF_BOUNDS.  Slower;
                                     for testing.  Batches and the GEMM are not
                                     checked.                                 */
COOT_API coot_status coot_ctx_create(int device, unsigned flags, coot_ctx** out);
COOT_API coot_status coot_ctx_destroy(coot_ctx* ctx);

/* ---- fused evaluation ----------------------------------------------------
 * Defined by Sec. 3 (delayed evaluation): an expression is a tree of Op /
 * eOp / Glue / eGlue types that is evaluated only when it is assigned, and
 * the whole tree is analysed to pick the fewest GPU calls; Sec. 4 (fourth
 * difference) names the alternative this replaces -- a chain of calls to
 * predefined kernels -- and Sec. 7 announces kernels generated per expression
 * as follow-up work.  coot_eval is that assignment: it evaluates `tree` over
 * `leaves` in one kernel launch (two for R_VAR and R_STDDEV: the second pass
 * reads the first pass's means); the reductions are Sec. 2's sums and
 * statistics functions:
 *   out     (nullable) receives the element-wise result Y, in the leaves'
 *           dtype; it may alias a leaf only when every read of that leaf is
 *           a full, untransposed read with out's exact layout (B += 3*A form);
 *           any other overlap is COOT_ERR_ALIAS.
 *   red     the reduction applied to Y (COOT_R_NONE for none);
 *   red_out (device) scalar or vector of the accumulation type; required
 *           when red.kind != R_NONE.
 * All leaves share one dtype.  The first call for a new tree signature
 * compiles its kernel (NVRTC, sm_103a) and must not happen during stream
 * capture; coot_warmup does that ahead of time. */
COOT_API coot_status coot_eval(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                      const coot_mat* out, coot_reduce red, void* red_out, coot_stream stream);

/* Same result computed eagerly, one kernel launch per node, each node
 * materialised in a device temporary of the compute type (the way Sec. 4
 * describes Bandicoot: one predefined kernel called after another).  This is
 * the unfused baseline; element-wise results are bitwise equal to coot_eval. */
COOT_API coot_status coot_eval_unfused(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves,
                              int32_t n_leaves, const coot_mat* out, coot_reduce red, void* red_out,
                              coot_stream stream);

/* JIT-compile (and, with COOT_CTX_TUNE, autotune) the kernel for this call
 * without writing to out or red_out.  Defined by Sec. 4 (third difference):
 * GPU kernels are compiled at run time for the device that is found and
 * cached, a one-time start-up cost that Sec. 5 leaves out of every timing;
 * coot_warmup pays it ahead of time (and must precede a stream capture).
 * Errors as coot_eval; nothing is launched. */
COOT_API coot_status coot_warmup(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                        const coot_mat* out, coot_reduce red);

/* ---- GEMM with a fused epilogue --------------------------------------------
 * Y = epi(P, extra...) with P = op(A) op(B) (Sec. 3: trans(X)*Y is one GEMM
 * call with a transposed operand; here the element-wise remainder of the
 * expression is evaluated on the product inside the same kernel, before Y is
 * stored):
 *   A, B     BF16, FP16, FP32 or FP64, both the same, rows adjacent
 *            (rs <= 1); op(A) = trans_a ? A^T : A is m x k, op(B) =
 *            trans_b ? B^T : B is k x n.
 *   epi      (nullable) a tree whose leaf 0 is the product P, read whole and
 *            untransposed, and whose leaves 1..n_extra are `extra` (m x n
 *            reads, not transposed); NULL means Y = P.
 *   out      m x n, same dtype; must not overlap A or B.
 * BF16 / FP16: products accumulated in FP32 on the tensor cores.  Operands
 * with 16-byte aligned bases and column strides that are multiples of 8
 * elements (any layout, any m, n, k >= 1) run on the persistent tcgen05
 * kernel (TMA loads, accumulator in tensor memory) unless the context has
 * COOT_CTX_NO_TCGEN05; others on mma.sync.  FP32 / FP64: products
 * accumulated in the storage type with fused multiply-adds on the CUDA
 * cores.  The epilogue runs in the compute type (FP32, or FP64 for FP64)
 * and Y is rounded once.  A tcgen05 wait that runs past its time limit sets
 * device flag COOT_FLAG_WAIT_TIMEOUT (Y is then undefined).
 * COOT_ERR_UNSUPPORTED for INT32 or a transposed epilogue read.  The first
 * call for an epilogue signature compiles its kernel. */
COOT_API coot_status coot_gemm_eval(coot_ctx* ctx, const coot_mat* A, int32_t trans_a, const coot_mat* B,
                                    int32_t trans_b, const coot_tree* epi, const coot_mat* extra, int32_t n_extra,
                                    const coot_mat* out, coot_stream stream);

/* ---- adjoint ---------------------------------------------------------------
 * The paper defines no gradient; Sec. 7 names the numerical optimisation
 * library ensmallen and the machine-learning library mlpack as the next users
 * of these expressions, and their optimisers consume the gradient of a scalar
 * loss written as such an expression -- this entry point computes it.
 * For a scalar loss L = red(tree) with red.kind R_ACCU, R_SUM (dim -1) or
 * R_MEAN (dim -1), writes grads[i] = upstream * dL/dleaves[i] for every i
 * whose grads[i].data is non-NULL (same shape/dtype as the leaf; F32/F64).
 * The forward values are recomputed per element inside the kernel; nothing
 * from a forward pass is stored.  Every leaf must be read through one full,
 * untransposed view (else COOT_ERR_UNSUPPORTED).  upstream is a device
 * scalar of the accumulation type. */
COOT_API coot_status coot_eval_adjoint(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves,
                              int32_t n_leaves, coot_reduce red, const void* upstream,
                              const coot_mat* grads, coot_stream stream);

/* ---- batched evaluation ----------------------------------------------------
 * Sec. 4 (second difference): a GPU is fast only when all of its cores are
 * busy, so one small matrix per call loses to the CPU below roughly
 * 1000 x 1000 elements.  Batching many small problems into one launch keeps
 * the GPU busy without changing any problem's result.
 * Many independent problems of the same tree, each with its own leaf shapes
 * (n_problems * n_leaves coot_mat in `problems`, problem-major, HOST array),
 * evaluated by one persistent kernel that pulls tiles from a work queue.
 * outs (nullable, n_problems entries) receives each problem's Y; red may be
 * R_NONE or R_ACCU/R_SUM(dim -1)/R_MEAN(dim -1) with one result per problem.
 * coot_batch_create validates, uploads the problem table and compiles; it
 * synchronises the device.  coot_batch_run launches once on `stream`;
 * red_out holds n_problems results.  The plan keeps the device pointers it
 * was given; they must stay valid while the plan is used. */
COOT_API coot_status coot_batch_create(coot_ctx* ctx, const coot_tree* tree, int64_t n_problems, int32_t n_leaves,
                              const coot_mat* problems, const coot_mat* outs, coot_reduce red,
                              coot_batch** out);
COOT_API coot_status coot_batch_run(coot_batch* batch, void* red_out, coot_stream stream);
COOT_API coot_status coot_batch_destroy(coot_batch* batch);
/* create + run + destroy in one call (the plan's device table is released in
 * stream order). */
COOT_API coot_status coot_eval_batched(coot_ctx* ctx, const coot_tree* tree, int64_t n_problems, int32_t n_leaves,
                              const coot_mat* problems, const coot_mat* outs, coot_reduce red,
                              void* red_out, coot_stream stream);

/* ---- CUDA graphs ------------------------------------------------------------
 * The paper has no graphs; Sec. 3 and Sec. 4 describe a program as the
 * sequence of GPU calls its assignments generate, issued from host code one
 * after another.  Recording such a sequence once and replaying it removes
 * the host's per-call launch cost while the kernels stay the same.
 * coot_graph_begin starts capturing `stream`; the coot_eval calls that follow
 * on it are recorded (their kernels must already be compiled: coot_warmup);
 * coot_graph_end ends the capture and instantiates the graph;
 * coot_graph_launch replays it on a stream.  Errors: COOT_ERR_INVALID for a
 * NULL context or graph, or capture of the legacy default stream;
 * COOT_ERR_CUDA when capture, instantiation or replay fails (ending a stream
 * that is not being captured included); a coot_eval during capture whose
 * kernel is not compiled yet is refused (COOT_ERR_INVALID) and nothing is
 * recorded for it. */
COOT_API coot_status coot_graph_begin(coot_ctx* ctx, coot_stream stream);
COOT_API coot_status coot_graph_end(coot_ctx* ctx, coot_stream stream, coot_graph** out);
COOT_API coot_status coot_graph_launch(coot_graph* graph, coot_stream stream);
COOT_API coot_status coot_graph_destroy(coot_graph* graph);

/* ---- host-side introspection (no GPU needed) ---------------------------------
 * Sec. 3: an expression's structure is captured as a type, and Sec. 4 (third
 * difference): the kernels are compiled at run time for the device and
 * cached.  The signature is the cache key of one expression type here.
 * coot_signature: validate the call and write its canonical signature (the
 * kernel-cache key: dtype, op structure, leaf layout classes, reduction) to
 * buf.  coot_codegen: write the generated CUDA source of the tree's kernel.
 * coot_compile: NVRTC-compile that source for sm_103a (no device needed) and
 * report the cubin size. */
COOT_API coot_status coot_signature(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                           const coot_mat* out, coot_reduce red, char* buf, size_t len);
COOT_API coot_status coot_codegen(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                         const coot_mat* out, coot_reduce red, char* buf, size_t len);
COOT_API coot_status coot_compile(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                         const coot_mat* out, coot_reduce red, size_t* cubin_bytes);

/* ---- evaluation without allocation -----------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while they run (a host framework that owns
 * every byte it hands out through its own pool or arena, or code in a region
 * where an allocation would synchronise the device or is not allowed).
 *
 * coot_sum_rows_f32_noalloc: per-row sums of an F32 column-major matrix x
 * (sum(X, 1); mean(X, 1) when mean != 0) written to out[0 .. x->n_rows) on
 * the device, with the same per-row reduction kernel and float-float
 * accumulation as coot_eval with R_SUM / R_MEAN along dim 1.  It runs on the
 * current CUDA device, needs no context, compiles nothing at run time and
 * allocates nothing: its scratch (one ticket per block of 1024 rows, 256 for
 * unaligned input, and the partial sums of the column splits) is a static
 * device array of COOT_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress) and queries the device; make that first
 * call before any stream capture.  Every call clears the tickets it uses, so
 * a failed earlier call leaves nothing behind; all calls on a device share
 * the array, so calls that can run at the same time on the GPU (different
 * streams without ordering) race -- issue them on one stream.  The address
 * found by the first call is kept for the process: do not call this entry
 * point on a device after cudaDeviceReset.  x must have adjacent rows
 * (rs 0 or 1; any ld >= n_rows): rs > 1 (a diagonal or row-strided view) is
 * COOT_ERR_UNSUPPORTED, rs < 0 COOT_ERR_INVALID.  A matrix with more rows
 * than the tickets cover (4096 x 1024 = 4,194,304 rows; 1,048,576 when x is
 * not 16-byte aligned) is rejected with COOT_ERR_UNSUPPORTED. */
#define COOT_NOALLOC_SCRATCH_BYTES (4u << 20)
COOT_API coot_status coot_sum_rows_f32_noalloc(const coot_mat* x, int32_t mean, float* out, coot_stream stream);

/* ---- errors and diagnostics --------------------------------------------------
 * Sec. 2 (Fig. coot_init) has an optional print-information switch and Sec. 4
 * (last difference) points out that reading device data from the host is a
 * transfer; errors here are therefore status codes with a host-side message,
 * and device-side conditions are gathered in one flag word read on demand.
 * coot_check_device_flag: wait for `stream`, read and clear the context's
 * device error flags (bit 0: an INT32 division by zero; bit 1: a bounded
 * wait of the tcgen05 GEMM timed out; bit 2: the bounds-check build found
 * an access outside a matrix).  Returns COOT_ERR_DEVICE_FLAG when any flag
 * was set. */
#define COOT_FLAG_INT_DIV_ZERO 1u
#define COOT_FLAG_WAIT_TIMEOUT 2u
#define COOT_FLAG_OUT_OF_BOUNDS 4u
COOT_API coot_status coot_check_device_flag(coot_ctx* ctx, coot_stream stream, uint32_t* flags);

/* Description of the last launch made by coot_eval on this context (kernel
 * family and launch shape, for profiling and the roofline; Sec. 5 times
 * whole operations, this reports what one of them launched).  Returns
 * COOT_ERR_INVALID for a NULL context or info. */
typedef struct {
  char kernel[64];
  int32_t grid, block;
  int32_t vec, unroll;
  int32_t n_launches;
  int64_t algorithmic_bytes; /* distinct operand bytes read + bytes written */
} coot_launch_info;
COOT_API coot_status coot_last_launch(coot_ctx* ctx, coot_launch_info* info);

/* Arithmetic and memory rates of a device, for the rooflines of kernels that
 * are not bound by HBM (Sec. 4, first difference: GPUs run 32-bit floating
 * point much faster than 64-bit, so FP64 trees can be bound by the FP64
 * pipe).  coot_probe_device runs small kernels on `device` (about a second;
 * it allocates 1 GiB or 8x the L2 size, whichever is larger, and frees it)
 * and reports the best of several CUDA-event timings: operations per second
 * of independent dependency chains per thread (exp: one exp and one FMA per
 * step), GB/s of a 16-byte-vector read and copy over buffers larger than
 * L2, and GB/s of a kernel reading and writing 256 MiB of pinned host
 * memory (the host link as kernels see it).  Returns COOT_ERR_OOM or
 * COOT_ERR_CUDA when the device refuses. */
typedef struct {
  double f32_add, f32_fma, f32_div, f32_exp;  /* operations per second */
  double f64_add, f64_fma, f64_div, f64_exp;
  double read_gbs, copy_gbs;                  /* copy: bytes read + written */
  double host_read_gbs, host_write_gbs;       /* kernel access to pinned host memory */
  int64_t buffer_bytes;                       /* bytes read per read probe  */
  int64_t l2_bytes;
  int32_t sms;
  int32_t sm_clock_khz;                       /* the device's rated SM clock */
} coot_probe_result;
COOT_API coot_status coot_probe_device(int device, coot_probe_result* result);

/* coot_last_error: the message of the calling thread's last failed call
 * (thread-local, never NULL, valid until that thread's next call).
 * coot_status_string: a static name for a status code. */
COOT_API const char* coot_last_error(void);
COOT_API const char* coot_status_string(coot_status s);
COOT_API void coot_version(int32_t* major, int32_t* minor);

#ifdef __cplusplus
}
#endif
#endif /* COOT_H */
