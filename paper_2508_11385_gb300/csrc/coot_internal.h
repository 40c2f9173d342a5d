// coot_internal.h -- host-side internals of libcootgb.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "coot.h"
#include "dev/coot_params.h"

// A named NVTX range for the lifetime of the object: profilers (nsys, ncu's
// NVTX filters) see the library's JIT compiles, tuning runs and launches as
// ranges; without a tool attached a push or pop costs a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace cg {

using coot::Params;
using coot::PF_SQRT;
using coot::PF_SEGMENTED;
using coot::PF_OUT_RUN;
using coot::PF_TRUN0;

using coot::RED_NONE;
using coot::RED_SUM;
using coot::RED_DOT;
using coot::RED_SSQ;
using coot::RED_MEAN1;
using coot::RED_CSQ;
using coot::RED_MIN;
using coot::RED_MAX;
using coot::RED_IMIN;
using coot::RED_IMAX;
using coot::RED_PROD;
using coot::red_additive;
using coot::red_extreme;

enum Family { F_STR = 0, F_COL = 1, F_ROW = 2, F_TILE = 3, F_ADJ = 4, F_BATCH = 5, F_SCAN = 6, F_GEMM = 7 };
const char* family_name(Family f);

// compute types
enum { CT_F32 = 0, CT_F64 = 1, CT_I32 = 2 };

// A leaf read after trans(), each_col/each_row and diag() have been pushed
// down to the leaves: tree element (i,j) reads the leaf element at
// off + i*rs + j*cs (in elements from the leaf's data).  Three kinds:
//   direct  (rs == 1): rows adjacent, vector loads; cs is the column stride
//           (0 for a column broadcast with each_col);
//   trans   a transposed view of a leaf with adjacent rows: tree (i,j) is
//           view (j,i) = leaf (r0 + j, c0 + i), staged through shared memory;
//   general any other stride (each_row broadcast rs = 0, a diagonal
//           rs = ld + 1, a row-strided leaf): one element at a time.
struct Slot {
  int leaf;
  int64_t off, rs, cs;
  int64_t r0, c0;  // trans: view origin in the leaf
  int64_t vr, vc;  // trans: view shape (rows, cols)
  bool trans;
  bool gen;
  bool full;           // direct read of the whole leaf in its own layout
  int64_t n_distinct;  // distinct leaf elements read
};

// canonical node: op from coot_opcode (N_LEAF means "slot"), no N_TRANS/N_SUBMAT
struct CNode {
  int op;
  int a = -1, b = -1;
  int slot = -1;
  int kidx = -1;
};

struct Analysis {
  coot_dtype dtype = COOT_F32;
  int esz = 4;
  int ct = CT_F32;
  int64_t nr = 0, nc = 0;  // shape of the tree's result
  std::vector<Slot> slots;
  std::vector<CNode> cn;
  int root = -1;
  std::vector<double> scalars;
  std::string type_str;
  int trmask = 0;
  int gmask = 0;         // general slots (bit s) and a general output (bit COOT_MAX_SLOTS)
  bool any_trans = false;
  int64_t out_rs = 1;    // row stride of the output
  coot_reduce red{};
  int red_mode = RED_NONE;  // device mode of the (last) pass
  bool has_out = false;
  int root_op = -1;         // op of the root (R_DOT needs N_SCHUR)
  int accum = 0;            // FP32 accumulation: 0 float-float, 1 Kahan, 2 plain ($COOT_ACCUM)
  int batch_be = 8192;      // flat batched kernel: elements per work item
  int batch_minb = 5;       // flat batched kernel: resident blocks per SM the registers are capped for
  // cumsum of a tree with transposed reads: scanned in one pass by the row
  // scan (set by the launcher when that kernel fits the shape), else the tree
  // is materialised first
  bool scan_direct = false;
  // GEMM epilogue trees: the slot holding the product, and the operands' layouts
  int gemm_ps = -1;
  bool gemm_ka = false, gemm_kb = false;
  // var / stddev: a first pass writes the mean(s), a second reduces (y - mean)^2
  bool two_pass() const { return red.kind == COOT_R_VAR || red.kind == COOT_R_STDDEV; }
  // bytes of one accumulator in the workspace (partials of cross-block combines)
  int acc_bytes() const { return (red_mode == RED_NONE || red_additive(red_mode)) ? 8 : 16; }
  // number of values the reduction writes (a vector along dim 0/1 may be empty)
  bool scan() const { return red.kind == COOT_R_CUMSUM; }
  // dim-1 segments (a Cube's slices side by side): 1 = the whole row
  int64_t n_seg() const { return red.n_seg > 1 ? red.n_seg : 1; }
  int64_t n_outputs() const {
    if (red.kind == COOT_R_NONE || red.kind == COOT_R_CUMSUM) return 0;
    return red.dim == 0 ? nc : (red.dim == 1 ? nr * n_seg() : 1);
  }
};

// Validate the call and canonicalise the tree.  `out` and `red_out` checks
// are part of it.  Returns COOT_OK or an error with set_error().
coot_status analyse(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves, const coot_mat* out,
                    coot_reduce red, Analysis* an);

// The aliasing rule of an output (part of analyse; the call cache re-checks
// it with each call's pointers).
coot_status check_out_alias(const Analysis& an, const coot_mat* leaves, const coot_mat* out);

// Kernel selection for a fused evaluation.
struct Choice {
  Family fam = F_STR;
  bool collapsed = false;  // contiguous tree walked as one long column
  bool vec_ok = false;     // every read and the output 16-byte aligned along columns
  int64_t it_rows = 0, it_cols = 0;
};
Choice choose(const Analysis& an, const coot_mat* leaves, const coot_mat* out);

struct KernelSpec {
  std::string name;
  int vec = 1, unroll = 1;
  int block = 256;  // threads per block the kernel is built for (max)
};

struct Program {
  std::string signature;  // cache key
  std::string source;     // NVRTC source
  std::vector<KernelSpec> kernels;
};

// Build the program (signature + source + kernel list) for a family.
// bounds: compile the bounds-check build (COOT_DEBUG_BOUNDS defined; its own
// signature and cache entries)
Program make_program(const Analysis& an, Family fam, bool var_two_pass, bool bounds = false);
std::string storage_type_name(coot_dtype d);

// ---- JIT ------------------------------------------------------------------
struct Module {
  cudaLibrary_t lib = nullptr;
  std::map<std::string, cudaKernel_t> kernels;
  std::map<std::string, cudaFuncAttributes> attrs;
  size_t cubin_bytes = 0;
  bool gemm_tc_smem = false;  // coot_gemm_tc: dynamic shared memory limit raised
};

// NVRTC-compile `source` for sm_103a; no device needed.
coot_status nvrtc_compile(const std::string& source, std::vector<char>* cubin, std::string* log);
uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull);
uint64_t headers_hash();

// ---- tuning ---------------------------------------------------------------
struct LaunchCfg {
  int kidx = 0;  // index in Program::kernels
  int block = 256;
  int blocks_per_sm = 4;
  int split = 0;  // col: warps per column (0: heuristic)
  std::string kname;  // the kernel's name (a stored tuning is used only if it still names kernel kidx)
};

// A fused call prepared once per (tree, layouts, alignment, reduction):
// analysis, kernel family, program and launch configuration.
struct CallPlan {
  Analysis an;
  Choice ch;
  Program pg;  // signature and kernel list (the source is dropped once compiled)
  Module* m = nullptr;
  bool have_cfg = false;
  LaunchCfg cfg;
};

}  // namespace cg

struct coot_ctx {
  int device = 0;
  unsigned flags = 0;
  int sms = 0;
  int l2_bytes = 0;
  std::string cache_dir;
  std::recursive_mutex mu;
  std::unordered_map<std::string, std::unique_ptr<cg::Module>> mods;
  std::map<std::string, cg::LaunchCfg> tuned;  // signature|bucket -> config
  // workspace: [tickets][err flag][mu][partials]
  void* ws = nullptr;
  size_t ws_bytes = 0;
  size_t n_tickets = 0;
  size_t partial_bytes = 0;
  unsigned* tickets = nullptr;
  unsigned* err_flag = nullptr;
  double* mean_ptr = nullptr;
  void* partials = nullptr;
  coot_launch_info last{};
  // call cache: everything a fused call derives from the tree, the layouts
  // and the reduction (not from the data pointers), keyed by those inputs
  std::unordered_map<std::string, std::unique_ptr<cg::CallPlan>> plans;
};

struct coot_batch {
  coot_ctx* ctx = nullptr;
  cg::Module* mod = nullptr;
  std::string kname;
  coot::BatchParams bp{};
  void* dev_mem = nullptr;  // problems, prefix, done counters, queue, partials
  int64_t n_problems = 0;
  int grid = 0, block = 256;
  int64_t algorithmic_bytes = 0;
  bool has_red = false;
};

struct coot_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// error helpers (api.cpp)
coot_status set_error(coot_status s, const char* fmt, ...);
coot_status cuda_error(cudaError_t e, const char* what);
bool log_enabled(const coot_ctx* ctx);
