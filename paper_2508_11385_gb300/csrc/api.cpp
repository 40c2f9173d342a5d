// api.cpp -- the C ABI of libcootgb (see include/coot.h).
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched through the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "coot_internal.h"

coot_status coot_get_module(coot_ctx* ctx, const cg::Program& pg, cg::Module** out);

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

coot_status set_error(coot_status s, const char* fmt, ...) {
  char buf[2048];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

coot_status cuda_error(cudaError_t e, const char* what) {
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return set_error(COOT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(COOT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool log_enabled(const coot_ctx* ctx) { return ctx && (ctx->flags & COOT_CTX_LOG); }

extern "C" const char* coot_last_error(void) { return g_err.c_str(); }

extern "C" const char* coot_status_string(coot_status s) {
  switch (s) {
    case COOT_OK: return "COOT_OK";
    case COOT_ERR_INVALID: return "COOT_ERR_INVALID";
    case COOT_ERR_SHAPE: return "COOT_ERR_SHAPE";
    case COOT_ERR_DTYPE: return "COOT_ERR_DTYPE";
    case COOT_ERR_ALIAS: return "COOT_ERR_ALIAS";
    case COOT_ERR_JIT: return "COOT_ERR_JIT";
    case COOT_ERR_OOM: return "COOT_ERR_OOM";
    case COOT_ERR_CUDA: return "COOT_ERR_CUDA";
    case COOT_ERR_DEVICE_FLAG: return "COOT_ERR_DEVICE_FLAG";
    case COOT_ERR_TIMEOUT: return "COOT_ERR_TIMEOUT";
    case COOT_ERR_UNSUPPORTED: return "COOT_ERR_UNSUPPORTED";
  }
  return "COOT_ERR_?";
}

extern "C" void coot_version(int32_t* major, int32_t* minor) {
  if (major) *major = COOT_VERSION_MAJOR;
  if (minor) *minor = COOT_VERSION_MINOR;
}

namespace {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) {
      changed = (cudaSetDevice(d) == cudaSuccess);
    }
    cudaGetLastError();
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

int64_t mat_ld(const coot_mat& m) { return (m.n_cols > 1) ? m.ld : (m.ld > 0 ? m.ld : m.n_rows); }

int rsize(int ct) { return ct == cg::CT_F32 ? 4 : 8; }

// elements addressable from a matrix's first element: its last element's
// offset plus one (0 for an empty matrix)
int64_t mat_extent(const coot_mat& m) {
  if (m.n_rows <= 0 || m.n_cols <= 0) return 0;
  const int64_t rs = m.rs > 1 ? m.rs : 1;
  const int64_t ld = m.n_cols > 1 ? m.ld : 0;
  return (m.n_rows - 1) * rs + (m.n_cols - 1) * ld + 1;
}

// the bounds-check build's extents of a launch's slots and output;
// COOT_DEBUG_BOUNDS_SHRINK=1 (tests of the check itself) declares every
// extent one element short, so that the kernel skips and reports the last
// element of each leaf instead of reading it
void set_extents(const cg::Analysis& an, const coot_mat* leaves, const coot_mat* out, cg::Params* p) {
  const char* sh = getenv("COOT_DEBUG_BOUNDS_SHRINK");
  const int64_t cut = (sh && sh[0] == '1') ? 1 : 0;
  for (size_t i = 0; i < an.slots.size(); ++i) {
    const cg::Slot& sl = an.slots[i];
    p->ext[i] = std::max<int64_t>(0, mat_extent(leaves[sl.leaf]) - sl.off - cut);
  }
  p->out_ext = out ? std::max<int64_t>(0, mat_extent(*out) - cut) : 0;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

const size_t kHeader = 1024;  // err flag at 0, mu at 256

// grow the workspace: tickets (zeroed) and partials
coot_status ws_ensure(coot_ctx* ctx, size_t tickets, size_t partial_bytes, cudaStream_t stream) {
  if (ctx->ws && tickets <= ctx->n_tickets && partial_bytes <= ctx->partial_bytes) return COOT_OK;
  if (capturing(stream))
    return set_error(COOT_ERR_INVALID,
                     "the workspace must grow (%zu tickets, %zu partial bytes) during stream capture; run the "
                     "call once (or coot_warmup) before capturing",
                     tickets, partial_bytes);
  size_t nt = std::max(tickets, std::max(ctx->n_tickets, (size_t)4096));
  size_t pb = std::max(partial_bytes, std::max(ctx->partial_bytes, (size_t)1 << 20));
  if (ctx->ws) {
    nt = std::max(nt, ctx->n_tickets + ctx->n_tickets / 2);
    pb = std::max(pb, ctx->partial_bytes + ctx->partial_bytes / 2);
  }
  nt = (nt + 63) & ~(size_t)63;
  pb = (pb + 255) & ~(size_t)255;
  unsigned old_flag = 0;
  cudaError_t e;
  if (ctx->ws) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
    cudaMemcpy(&old_flag, ctx->err_flag, sizeof old_flag, cudaMemcpyDeviceToHost);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
  }
  size_t tbytes = nt * sizeof(unsigned);
  size_t total = kHeader + tbytes + pb;
  if ((e = cudaMalloc(&ctx->ws, total)) != cudaSuccess) {
    ctx->ws = nullptr;
    ctx->n_tickets = ctx->partial_bytes = 0;
    return cuda_error(e, "workspace cudaMalloc");
  }
  if ((e = cudaMemset(ctx->ws, 0, kHeader + tbytes)) != cudaSuccess) return cuda_error(e, "workspace cudaMemset");
  char* b = (char*)ctx->ws;
  ctx->err_flag = (unsigned*)b;
  ctx->mean_ptr = (double*)(b + 256);
  ctx->tickets = (unsigned*)(b + kHeader);
  ctx->partials = (void*)(b + kHeader + tbytes);
  ctx->n_tickets = nt;
  ctx->partial_bytes = pb;
  if (old_flag) cudaMemcpy(ctx->err_flag, &old_flag, sizeof old_flag, cudaMemcpyHostToDevice);
  return COOT_OK;
}

uint64_t scalar_bits(double k, int ct) {
  uint64_t b = 0;
  if (ct == cg::CT_F32) {
    float f = (float)k;
    uint32_t u;
    memcpy(&u, &f, 4);
    b = u;
  } else if (ct == cg::CT_F64) {
    memcpy(&b, &k, 8);
  } else {
    int32_t i = (int32_t)k;  // truncation toward zero (validated range)
    b = (uint32_t)i;
  }
  return b;
}

int occupancy(cg::Module* m, const std::string& name, int block) {
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)m->kernels[name], block, 0);
  if (e != cudaSuccess || n <= 0) {
    cudaGetLastError();
    const cudaFuncAttributes& fa = m->attrs[name];
    int regs = std::max(fa.numRegs, 16);
    int per_warp = ((regs * 32 + 255) / 256) * 256;
    int by_regs = 65536 / std::max(per_warp * (block / 32), 1);
    int by_thr = 2048 / block;
    int by_smem = fa.sharedSizeBytes ? (int)((227 * 1024) / (fa.sharedSizeBytes + 1024)) : 32;
    n = std::max(1, std::min(std::min(by_regs, by_thr), std::min(by_smem, 32)));
  }
  return n;
}

// what one launch of a fused program needs
struct Launch {
  std::string kname, kname2;  // kname2: second pass of var
  std::string kname_pre;      // launched before kname: the totals pass of a segmented cumsum
  int grid = 1, block = 256, vec = 1, unroll = 1;
  size_t tickets = 1, partial_bytes = 0;
  size_t mu_offset = 0;  // var/stddev along a dim: byte offset of the means in the partials
  cg::Params p{};
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool is_scanp(const std::string& name) { return name.compare(0, 11, "coot_scanp_") == 0; }

// the one-pass scan along rows serves plain matrices (not a Cube's slices)
// with at least one band of 32 rows per SM; else the segmented two-pass scan
bool scanp_fits(const cg::Analysis& an, int sms) {
  return an.scan() && an.red.dim == 1 && an.n_seg() == 1 && an.nr >= 32LL * sms;
}


int64_t n_red_outputs(const cg::Analysis& an) { return an.n_outputs(); }

// fill the launch shape of a fused program for a given kernel variant/config
void shape_launch(coot_ctx* ctx, const cg::Analysis& an, const cg::Choice& ch, cg::Module* m,
                  const cg::KernelSpec& k, int block, int bps, Launch* L, int split = 0) {
  const int64_t R = ch.it_rows, C = ch.it_cols;
  const int64_t ab = an.acc_bytes();
  L->block = block;
  L->vec = k.vec;
  L->unroll = k.unroll;
  const int64_t resident = (int64_t)ctx->sms * std::max(bps, 1);
  cg::Params& p = L->p;
  p.n_rows = R;
  p.n_cols = C;
  if (ch.fam == cg::F_STR || ch.fam == cg::F_ADJ) {
    // str: chunks of block * vec rows per column, a unit is `unroll`
    // consecutive chunks in column-major order (it may span columns); adj: a
    // unit is one chunk of block * vec * unroll rows of one column
    const bool str = ch.fam == cg::F_STR;
    const int64_t chunk = (int64_t)block * k.vec * (str ? 1 : k.unroll);
    p.units_per_col = std::max<int64_t>(1, ceil_div(R, chunk));
    const int64_t units = str ? ceil_div(p.units_per_col * C, k.unroll) : p.units_per_col * C;
    L->grid = (int)std::max<int64_t>(1, std::min(units, resident));
    L->partial_bytes = (size_t)L->grid * ab;
    L->tickets = 1;
  } else if (ch.fam == cg::F_COL) {
    const int64_t wpb = block / 32;
    // warps per column: enough that every column step fills the GPU, a
    // divisor of the warps per block
    int64_t G = split;
    if (G <= 0) {
      G = 1;
      while (G < wpb && (C * 1.0) / (resident * (wpb / G)) < 4.0 && R >= G * 2 * 32 * k.vec * k.unroll) G *= 2;
    }
    G = std::max<int64_t>(1, std::min<int64_t>(G, wpb));
    while (wpb % G) --G;
    p.n_splits = G;
    L->grid = (int)std::max<int64_t>(1, std::min(ceil_div(C, wpb / G), resident));
    L->partial_bytes = 0;
    L->tickets = 1;
  } else if (ch.fam == cg::F_ROW) {
    const int64_t nrb = std::max<int64_t>(1, ceil_div(R, (int64_t)block * k.vec));
    int64_t nsp = std::max<int64_t>(1, std::min<int64_t>(C, resident / nrb));
    int64_t cps = std::max<int64_t>(1, ceil_div(std::max<int64_t>(C, 1), nsp));
    // transposed reads go along each row's columns in 16-byte vectors: every
    // segment starts on a multiple of 16 columns
    if (an.any_trans) cps = ceil_div(cps, 16) * 16;
    nsp = std::max<int64_t>(1, ceil_div(std::max<int64_t>(C, 1), cps));
    if (an.n_seg() > 1) {  // one split per segment, written separately
      nsp = an.n_seg();
      cps = C / nsp;
    }
    p.n_row_blocks = nrb;
    p.n_splits = nsp;
    p.units_per_col = cps;
    L->grid = (int)(nrb * nsp);
    L->partial_bytes = (nsp > 1 && an.n_seg() == 1) ? (size_t)(nsp * R * ab) : 0;
    L->tickets = (size_t)nrb;
  } else if (ch.fam == cg::F_TILE) {
    // tilev tiles are 32 x vec rows tall; the scalar tile kernel's 32
    const int64_t ntr = ceil_div(R, 32 * std::max(k.vec, 1)), ntc = ceil_div(C, 32);
    const int64_t tiles = ntr * ntc;
    if (an.red.dim == 0 || an.red.dim == 1) {
      // units = strips x segments, taken in turn by a grid of at most the
      // resident blocks; `split` segments per strip when given (tuning),
      // else about eight units per resident block, so that the last round
      // of units costs little
      const int64_t strips = std::max<int64_t>(an.red.dim == 0 ? ntc : ntr, 1);
      const int64_t len = std::max<int64_t>(an.red.dim == 0 ? ntr : ntc, 1);
      int64_t nseg = split > 0 ? split : ceil_div(8 * resident, strips);
      nseg = std::max<int64_t>(1, std::min(nseg, len));
      nseg = ceil_div(len, ceil_div(len, nseg));  // no empty segment
      p.n_splits = nseg;
      L->grid = (int)std::min<int64_t>(strips * nseg, resident);
      const int64_t no = (an.red.dim == 0) ? C : R;
      L->partial_bytes = (nseg > 1) ? (size_t)(nseg * no * ab) : 0;
      L->tickets = (size_t)strips;
    } else {
      L->grid = (int)std::max<int64_t>(1, std::min(tiles, resident));
      L->partial_bytes = (size_t)L->grid * ab;
      L->tickets = 1;
    }
  }
  if (ch.fam == cg::F_SCAN) {
    const int64_t ab8 = 8;  // one running sum per (line, segment)
    L->tickets = 1;
    L->kname_pre.clear();
    if (an.red.dim == 0) {
      // a warp per (column, segment) of 32 V-row steps
      const int64_t wpb = block / 32;
      const int64_t steps = std::max<int64_t>(1, ceil_div(R, 32 * (int64_t)k.vec));
      const int64_t resident_warps = resident * wpb;
      int64_t nseg = split > 0 ? split : ceil_div(2 * resident_warps, std::max<int64_t>(C, 1));
      nseg = std::max<int64_t>(1, std::min(nseg, steps));
      const int64_t sps = ceil_div(steps, nseg);
      nseg = ceil_div(steps, sps);
      p.n_splits = nseg;
      p.units_per_col = sps;
      const int64_t units = std::max<int64_t>(C, 1) * nseg;
      L->grid = (int)std::max<int64_t>(1, std::min(ceil_div(units, wpb), 4 * resident));
      L->partial_bytes = (nseg > 1) ? (size_t)(C * nseg * ab8) : 0;
    } else if (is_scanp(k.name)) {
      // one pass: a block (of the kernel's own size) per band of 32 V rows
      L->block = k.block;
      const int64_t nrb = std::max<int64_t>(1, ceil_div(R, 32 * (int64_t)k.vec));
      p.n_row_blocks = nrb;
      p.n_splits = 1;
      p.units_per_col = std::max<int64_t>(C, 1);
      L->grid = (int)nrb;
      L->partial_bytes = 0;
    } else {
      // a thread per V rows of a (row block, column segment)
      const int64_t nrb = std::max<int64_t>(1, ceil_div(R, (int64_t)block * k.vec));
      int64_t nseg = split > 0 ? split : ceil_div(2 * resident, nrb);
      nseg = std::max<int64_t>(1, std::min(nseg, std::max<int64_t>(C, 1)));
      int64_t cps = std::max<int64_t>(1, ceil_div(std::max<int64_t>(C, 1), nseg));
      nseg = std::max<int64_t>(1, ceil_div(std::max<int64_t>(C, 1), cps));
      if (an.n_seg() > 1) {  // a Cube's slices: independent scans, no totals pass
        nseg = an.n_seg();
        cps = C / nseg;
      }
      p.n_row_blocks = nrb;
      p.n_splits = nseg;
      p.units_per_col = cps;
      L->grid = (int)(nrb * nseg);
      L->partial_bytes = (nseg > 1) ? (size_t)(nseg * R * ab8) : 0;
    }
    if (p.n_splits > 1 && an.n_seg() == 1) {
      std::string pre = k.name;
      pre.replace(pre.find("coot_scan_"), 10, "coot_scan_t_");
      L->kname_pre = pre;
    }
  }
  // var / stddev along a dim: the first pass's means follow the partials
  if (an.two_pass() && an.red.dim >= 0) {
    L->mu_offset = (L->partial_bytes + 255) & ~(size_t)255;
    L->partial_bytes = L->mu_offset + (size_t)std::max<int64_t>(an.n_outputs(), 1) * 8;
  }
  (void)m;
}

// workspace pointers of a shaped launch (after ws_ensure)
void bind_workspace(coot_ctx* ctx, const cg::Analysis& an, Launch* L) {
  L->p.tickets = ctx->tickets;
  L->p.err_flag = ctx->err_flag;
  L->p.partials = ctx->partials;
  L->p.mu = (an.two_pass() && an.red.dim >= 0) ? (double*)((char*)ctx->partials + L->mu_offset) : ctx->mean_ptr;
}

int64_t algorithmic_bytes(const cg::Analysis& an, const coot_mat* out) {
  int64_t b = 0;
  for (const cg::Slot& s : an.slots) b += s.n_distinct * an.esz;
  if (an.two_pass()) b *= 2;  // the tree is read by both passes
  if (out) b += an.nr * an.nc * an.esz;
  const bool idx = an.red.kind == COOT_R_INDEX_MIN || an.red.kind == COOT_R_INDEX_MAX;
  return b + an.n_outputs() * ((an.ct == cg::CT_F32 && !idx) ? 4 : 8);
}

// pick the default kernel variant of a program for this call: the vector
// variant with unroll 2 when every column start is 16-byte aligned, else the
// scalar variant (second passes of var are paired by name)
int default_variant(const cg::Program& pg, const cg::Choice& ch) {
  int best = -1;
  for (int i = 0; i < (int)pg.kernels.size(); ++i) {
    const cg::KernelSpec& k = pg.kernels[i];
    if (k.name.find("_p2") != std::string::npos || k.name.find("_t_") != std::string::npos) continue;
    if (is_scanp(k.name)) continue;
    if (!ch.vec_ok && k.vec > 1) continue;
    if (best < 0) best = i;
    if (ch.vec_ok && k.vec > 1 && k.unroll == 2) return i;
    if (!ch.vec_ok && k.vec == 1) return i;
  }
  return best < 0 ? 0 : best;
}

std::string pair_name(const std::string& p1) {
  std::string n = p1;
  size_t at = n.find("_p1");
  if (at != std::string::npos) n.replace(at, 3, "_p2");
  return n;
}

coot_status launch_kernel(cg::Module* m, const std::string& name, int grid, int block, void* params,
                          cudaStream_t stream) {
  void* args[] = {params};
  cudaError_t e = cudaLaunchKernel((const void*)m->kernels[name], dim3(grid), dim3(block), args, 0, stream);
  if (e != cudaSuccess) return cuda_error(e, name.c_str());
  return COOT_OK;
}

coot_status tune(coot_ctx* ctx, const cg::Analysis& an, const cg::Choice& ch, const cg::Program& pg, cg::Module* m,
                 Launch base, cudaStream_t stream, cg::LaunchCfg* best);

// persistent tuning cache: one line per tuned (signature, size bucket)
std::string tune_path(const coot_ctx* ctx) {
  if ((ctx->flags & COOT_CTX_NO_DISK_CACHE) || ctx->cache_dir.empty()) return std::string();
  char name[96];
  snprintf(name, sizeof name, "/tune-%016llx-sm%d.txt", (unsigned long long)cg::headers_hash(), ctx->sms);
  return ctx->cache_dir + name;
}

void load_tuning(coot_ctx* ctx) {
  std::string path = tune_path(ctx);
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "r");
  if (!f) return;
  std::vector<char> line(1 << 16);
  while (fgets(line.data(), (int)line.size(), f)) {
    char* tab = strrchr(line.data(), '\t');
    if (!tab) continue;
    cg::LaunchCfg c;
    char name[128];
    if (sscanf(tab + 1, "%d %d %d %d %127s", &c.kidx, &c.block, &c.blocks_per_sm, &c.split, name) != 5) continue;
    c.kname = name;
    *tab = 0;
    ctx->tuned[std::string(line.data())] = c;
  }
  fclose(f);
}

void save_tuning(coot_ctx* ctx, const std::string& key, const cg::LaunchCfg& c) {
  std::string path = tune_path(ctx);
  if (path.empty()) return;
  FILE* f = fopen(path.c_str(), "a");  // one short line per append
  if (!f) return;
  fprintf(f, "%s\t%d %d %d %d %s\n", key.c_str(), c.kidx, c.block, c.blocks_per_sm, c.split, c.kname.c_str());
  fclose(f);
}

std::string tune_key(const cg::Program& pg, const cg::Choice& ch) {
  int64_t n = ch.it_rows * std::max<int64_t>(ch.it_cols, 1);
  int bucket = 0;
  while ((int64_t(1) << bucket) < n && bucket < 62) ++bucket;
  return pg.signature + "|b" + std::to_string(bucket) + "|v" + std::to_string(ch.vec_ok) + "|r" +
         std::to_string(ch.it_cols > 1 ? 1 : 0);
}

}  // namespace

// The transposed problem: element (i, j) of its result is element (j, i) of
// an's.  Each slot's row and column strides swap; a slot whose columns become
// one element apart is read as a transposed slot (rows rs apart, a thread's
// consecutive columns consecutive in memory), one whose rows become adjacent
// as a direct slot, the others as general slots.  The output view swaps the
// same way (into *out_t).  A cumsum along dim 0 of a tree with transposed
// reads is the cumsum along dim 1 of this problem.
static cg::Analysis transposed_problem(const cg::Analysis& an, const coot_mat& out, coot_mat* out_t) {
  cg::Analysis f = an;
  std::swap(f.nr, f.nc);
  f.trmask = 0;
  f.gmask = 0;
  f.any_trans = false;
  for (size_t s = 0; s < f.slots.size(); ++s) {
    cg::Slot& sl = f.slots[s];
    std::swap(sl.rs, sl.cs);
    std::swap(sl.r0, sl.c0);
    std::swap(sl.vr, sl.vc);
    sl.full = false;
    sl.trans = (sl.cs == 1 && sl.rs != 1);
    sl.gen = !sl.trans && sl.rs != 1;
    if (sl.trans) {
      f.any_trans = true;
      f.trmask |= 1 << s;
    }
    if (sl.gen) f.gmask |= 1 << s;
  }
  // out_t: n_cols x n_rows, rows mat_ld(out) apart, columns out_rs apart
  *out_t = out;
  out_t->n_rows = out.n_cols;
  out_t->n_cols = out.n_rows;
  out_t->rs = mat_ld(out);
  out_t->ld = an.out_rs;
  f.out_rs = out_t->rs;
  if (f.out_rs != 1 && f.nr > 1) f.gmask |= 1 << COOT_MAX_SLOTS;
  if (f.red.kind == COOT_R_CUMSUM) f.red.dim = 1 - f.red.dim;
  return f;
}

// ---------------------------------------------------------------------------
// run one analysed fused evaluation (warm: compile + tune without launching)
// ---------------------------------------------------------------------------
static coot_status run_fused(coot_ctx* ctx, const cg::Analysis& an, const coot_mat* leaves, const coot_mat* out,
                             void* red_out, cudaStream_t stream, bool warm_only, cg::CallPlan* plan = nullptr) {
  if (an.scan() && an.any_trans && !an.scan_direct && an.n_seg() == 1 && out && an.nr > 1 && an.nc > 1) {
    // one pass of the row scan, which reads transposed slots along each
    // thread's runs of columns: along dim 1 directly, along dim 0 over the
    // transposed problem, when its rows fill the SMs
    if (an.red.dim == 1 && scanp_fits(an, ctx->sms)) {
      cg::Analysis d = an;
      d.scan_direct = true;
      return run_fused(ctx, d, leaves, out, red_out, stream, warm_only);
    }
    if (an.red.dim == 0 && an.nc >= 32LL * ctx->sms) {
      coot_mat out_t;
      cg::Analysis d = transposed_problem(an, *out, &out_t);
      d.scan_direct = true;
      return run_fused(ctx, d, leaves, &out_t, red_out, stream, warm_only);
    }
  }
  if (an.scan() && an.any_trans && !an.scan_direct) {
    // a tree with transposed reads is first materialised into out by the
    // tile kernel, then scanned in place (out read and written by the same
    // thread)
    cg::Analysis a1 = an;
    a1.red = coot_reduce{COOT_R_NONE, -1, 0, 0};
    a1.red_mode = cg::RED_NONE;
    coot_status s1 = run_fused(ctx, a1, leaves, out, nullptr, stream, warm_only);
    if (s1) return s1;
    coot_node leaf{};
    leaf.op = COOT_N_LEAF;
    leaf.a = leaf.b = -1;
    coot_tree lt{1, 0, &leaf};
    cg::Analysis a2;
    s1 = cg::analyse(&lt, out, 1, out, an.red, &a2);
    if (s1) return s1;
    const int n1 = ctx->last.n_launches;
    s1 = run_fused(ctx, a2, out, out, nullptr, stream, warm_only);
    if (s1 || warm_only) return s1;
    // report the whole evaluation: both steps' launches, the tree's bytes
    ctx->last.n_launches += n1;
    ctx->last.algorithmic_bytes = algorithmic_bytes(an, out);
    return COOT_OK;
  }
  const bool var = an.two_pass();
  const bool hit = plan && plan->m;  // prepared by an earlier call with the same inputs
  cg::Choice ch = hit ? plan->ch : cg::choose(an, leaves, out);
  const int64_t count = an.nr * an.nc;
  if (!warm_only && count == 0 && an.red.kind != COOT_R_PROD) {
    // nothing to read: reductions of no elements.  All-ones bytes are a NaN
    // in float and double and -1 in int64.
    if (an.red.kind == COOT_R_NONE) return COOT_OK;
    const int k = an.red.kind;
    const bool ones = k == COOT_R_MEAN || k == COOT_R_VAR || k == COOT_R_STDDEV || k == COOT_R_INDEX_MIN ||
                      k == COOT_R_INDEX_MAX || ((k == COOT_R_MIN || k == COOT_R_MAX) && an.ct != cg::CT_I32);
    const size_t esz = (k == COOT_R_INDEX_MIN || k == COOT_R_INDEX_MAX) ? 8 : rsize(an.ct);
    const int64_t nout = an.n_outputs();
    if (nout > 0) {
      cudaError_t e = cudaMemsetAsync(red_out, ones ? 0xff : 0, (size_t)nout * esz, stream);
      if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    }
    return COOT_OK;
  }
  if (count == 0) {
    // an empty product is 1 per output: the column / row / flat kernels
    // write their empty accumulators without reading anything
    if (an.n_outputs() == 0 && !warm_only) return COOT_OK;
    ch.fam = an.red.dim == 0 ? cg::F_COL : (an.red.dim == 1 ? cg::F_ROW : cg::F_STR);
    ch.collapsed = false;
    ch.vec_ok = false;
    ch.it_rows = an.nr;
    ch.it_cols = an.nc;
  }
  cg::Program fresh;
  const bool bounds = (ctx->flags & COOT_CTX_DEBUG_BOUNDS) != 0;
  if (!hit) fresh = cg::make_program(an, ch.fam, var, bounds);
  const cg::Program& pg = hit ? plan->pg : fresh;
  if (!hit && !ctx->mods.count(pg.signature) && capturing(stream))
    return set_error(COOT_ERR_INVALID, "this tree's kernel is not compiled yet; call coot_warmup before capturing");
  cg::Module* m = hit ? plan->m : nullptr;
  coot_status s = COOT_OK;
  if (!hit) {
    s = coot_get_module(ctx, pg, &m);
    if (s) return s;
    if (plan) {
      plan->ch = ch;
      plan->pg.signature = pg.signature;
      plan->pg.kernels = pg.kernels;
      plan->m = m;
    }
  }

  Launch L;
  cg::Params& p = L.p;
  for (size_t i = 0; i < an.slots.size(); ++i) {
    const cg::Slot& sl = an.slots[i];
    const coot_mat& Lf = leaves[sl.leaf];
    p.src[i] = (const char*)Lf.data + sl.off * an.esz;
    // a transposed slot's staging walks its view with the leaf's column
    // stride (the slot's row stride); the others walk columns with cs
    p.ld[i] = sl.trans ? sl.rs : sl.cs;
    p.rs[i] = sl.rs;
  }
  if (bounds) set_extents(an, leaves, out, &p);
  for (size_t i = 0; i < an.scalars.size(); ++i) p.k[i] = scalar_bits(an.scalars[i], an.ct);
  p.out = out ? out->data : nullptr;
  p.out_ld = out ? mat_ld(*out) : 0;
  p.out_rs = an.out_rs;
  // elements per reduction output
  const int64_t per = (an.red.dim == 0) ? an.nr : (an.red.dim == 1 ? an.nc / an.n_seg() : count);
  p.count = per;
  p.div = 1.0;
  if (an.red.kind == COOT_R_MEAN) p.div = (double)per;
  p.den = (an.red.norm_type == 1) ? (double)per : (double)(per - 1);
  p.flags = (an.red.kind == COOT_R_STDDEV) ? cg::PF_SQRT : 0u;
  if (an.n_seg() > 1) p.flags |= cg::PF_SEGMENTED;
  if ((ch.fam == cg::F_SCAN || ch.fam == cg::F_ROW) && an.red.dim == 1) {
    // the row scan's runs of 16 consecutive columns (transposed slots, a
    // transposed output): vectors where every run starts 16-byte aligned
    for (size_t i = 0; i < an.slots.size(); ++i) {
      const cg::Slot& sl = an.slots[i];
      if (sl.trans && (uintptr_t)p.src[i] % 16 == 0 && (sl.rs * an.esz) % 16 == 0)
        p.flags |= cg::PF_TRUN0 << i;
    }
    if (out && ((an.gmask >> COOT_MAX_SLOTS) & 1) && p.out_ld == 1 && (uintptr_t)out->data % 16 == 0 &&
        (an.out_rs * an.esz) % 16 == 0)
      p.flags |= cg::PF_OUT_RUN;
  }
  p.red_out = red_out;

  // launch configuration: the call plan's, else tuned, else the default
  // variant at full occupancy
  cg::LaunchCfg cfg;
  // COOT_FORCE_KERNEL=<kernel name>: that variant of the program at its
  // default launch shape, when the program has it (tests of every variant)
  int forced = -1;
  if (const char* fk = getenv("COOT_FORCE_KERNEL")) {
    for (int i = 0; i < (int)pg.kernels.size(); ++i)
      if (pg.kernels[i].name == fk && (ch.vec_ok || pg.kernels[i].vec == 1) &&
          (!is_scanp(fk) || an.n_seg() == 1))
        forced = i;
  }
  if (forced >= 0) {
    cfg.kidx = forced;
    cfg.block = std::min(pg.kernels[forced].block, 256);
    cfg.blocks_per_sm = occupancy(m, pg.kernels[forced].name, cfg.block);
    cfg.split = 0;
  } else if (hit && plan->have_cfg) {
    cfg = plan->cfg;
  } else {
    const std::string key = tune_key(pg, ch);
    auto tu = ctx->tuned.find(key);
    if (tu != ctx->tuned.end() && tu->second.kidx >= 0 && tu->second.kidx < (int)pg.kernels.size() &&
        pg.kernels[tu->second.kidx].name == tu->second.kname && (ch.vec_ok || pg.kernels[tu->second.kidx].vec == 1)) {
      cfg = tu->second;
    } else {
      cfg.kidx = default_variant(pg, ch);
      if (scanp_fits(an, ctx->sms)) {
        for (int i = 0; i < (int)pg.kernels.size(); ++i)
          if (pg.kernels[i].name == "coot_scanp_v1u16w8") cfg.kidx = i;
      }
      cfg.block = pg.kernels[cfg.kidx].block;
      if (ch.fam == cg::F_ROW) cfg.block = 256;
      cfg.blocks_per_sm = occupancy(m, pg.kernels[cfg.kidx].name, cfg.block);
      if ((ctx->flags & COOT_CTX_TUNE) && !capturing(stream) && count > 0) {
        Launch base = L;
        s = tune(ctx, an, ch, pg, m, base, stream, &cfg);
        if (s) return s;
        cfg.kname = pg.kernels[cfg.kidx].name;
        ctx->tuned[key] = cfg;
        save_tuning(ctx, key, cfg);
      }
    }
    if (plan && !capturing(stream)) {
      plan->cfg = cfg;
      plan->have_cfg = true;
    }
  }
  const cg::KernelSpec& ks = pg.kernels[cfg.kidx];
  shape_launch(ctx, an, ch, m, ks, cfg.block, cfg.blocks_per_sm, &L, cfg.split);
  L.kname = ks.name;
  if (var) L.kname2 = pair_name(ks.name);
  s = ws_ensure(ctx, L.tickets, L.partial_bytes, stream);
  if (s) return s;
  bind_workspace(ctx, an, &L);
  if (warm_only) return COOT_OK;

  if (!L.kname_pre.empty()) {
    s = launch_kernel(m, L.kname_pre, L.grid, L.block, &p, stream);
    if (s) return s;
  }
  s = launch_kernel(m, L.kname, L.grid, L.block, &p, stream);
  if (s) return s;
  if (var) {
    s = launch_kernel(m, L.kname2, L.grid, L.block, &p, stream);
    if (s) return s;
  }
  coot_launch_info& li = ctx->last;
  memset(&li, 0, sizeof li);
  snprintf(li.kernel, sizeof li.kernel, "%s", L.kname.c_str());
  li.grid = L.grid;
  li.block = L.block;
  li.vec = L.vec;
  li.unroll = L.unroll;
  li.n_launches = (var || !L.kname_pre.empty()) ? 2 : 1;
  li.algorithmic_bytes = algorithmic_bytes(an, out);
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// autotuner: kernel variant x block size x resident blocks per SM, timed with
// CUDA events on scratch outputs (user buffers are never written)
// ---------------------------------------------------------------------------
namespace {
coot_status tune(coot_ctx* ctx, const cg::Analysis& an, const cg::Choice& ch, const cg::Program& pg, cg::Module* m,
                 Launch base, cudaStream_t stream, cg::LaunchCfg* best) {
  NvtxRange nvtx_range("cootgb tune");
  const bool var = an.two_pass();
  void* scratch_out = nullptr;
  void* scratch_red = nullptr;
  cudaError_t e;
  // scratch output with the alignment the vector variants need: contiguous
  // when the call walks one long column, else columns padded to 16 bytes
  const int64_t per16 = 16 / an.esz;
  const int64_t sld = ch.collapsed ? std::max<int64_t>(an.nr, 1) : ((an.nr + per16 - 1) / per16) * per16;
  const size_t out_bytes = base.p.out ? (size_t)(std::max<int64_t>(sld, 1) * std::max<int64_t>(an.nc, 1) * an.esz) : 0;
  if (out_bytes && (e = cudaMalloc(&scratch_out, out_bytes)) != cudaSuccess) return cuda_error(e, "tune cudaMalloc");
  const int64_t nred = std::max<int64_t>(an.nr, an.nc) + 1;
  if ((e = cudaMalloc(&scratch_red, (size_t)nred * 8)) != cudaSuccess) {
    cudaFree(scratch_out);
    return cuda_error(e, "tune cudaMalloc");
  }
  // operands that fit in L2 would be read from L2 on every rep after the
  // first, while a call on data that was not just touched streams them from
  // HBM: for such calls a buffer twice the L2 size is overwritten before each
  // rep, outside the timed region (tuned on L2-resident data when the buffer
  // cannot be had)
  int64_t ws = 0;
  for (const cg::Slot& s : an.slots) ws += s.n_distinct * an.esz;
  if (base.p.out) ws += an.nr * an.nc * an.esz;
  const size_t flush_bytes = (size_t)2 * (size_t)std::max(ctx->l2_bytes, 0);
  void* flush = nullptr;
  if (flush_bytes > 0 && ws < (int64_t)flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    flush = nullptr;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  coot_status st = COOT_OK;
  for (int ki = 0; ki < (int)pg.kernels.size() && st == COOT_OK; ++ki) {
    const cg::KernelSpec& k = pg.kernels[ki];
    if (k.name.find("_p2") != std::string::npos || k.name.find("_t_") != std::string::npos) continue;
    if (!ch.vec_ok && k.vec > 1) continue;
    const bool one_pass = is_scanp(k.name);  // its grid is fixed by the rows
    if (one_pass && an.n_seg() != 1) continue;
    std::vector<int> blocks;
    if (ch.fam == cg::F_TILE || ch.fam == cg::F_SCAN) blocks = {256};
    else if (ch.fam == cg::F_ROW) blocks = {128, 256, 512};
    else blocks = {256, 512};
    for (int block : blocks) {
      if (block > k.block) continue;
      int occ = occupancy(m, k.name, block);
      std::vector<int> bpss = {occ};
      for (int b : {1, 2, 4}) if (b < occ && !one_pass) bpss.push_back(b);
      std::vector<int> splits = {0};
      if (ch.fam == cg::F_COL)
        for (int g = 1; g <= block / 32; g *= 2) splits.push_back(g);
      if (ch.fam == cg::F_TILE && an.red.dim >= 0) {
        // segments per strip: one, and about 1, 2, 4, 8, 16 units per
        // resident block
        const int64_t tall = (an.red.dim == 0) ? 32 : 32 * std::max(k.vec, 1);
        const int64_t strips = std::max<int64_t>(ceil_div(an.red.dim == 0 ? an.nc : an.nr, tall), 1);
        const int64_t res = (int64_t)ctx->sms * std::max(occ, 1);
        splits.push_back(1);
        for (int64_t w2 : {1, 2, 4, 8, 16}) splits.push_back((int)std::max<int64_t>(1, ceil_div(w2 * res, strips)));
      }
      if (ch.fam == cg::F_SCAN && !one_pass) splits.push_back(1);  // one pass, no segments
      for (int bps : bpss)
      for (int split : splits) {
        Launch L = base;
        L.p.out = scratch_out;
        if (scratch_out) {
          // the scratch output is plain column-major (rows adjacent, columns
          // sld apart), whatever the strides of the call's output
          L.p.out_ld = sld;
          L.p.out_rs = 1;
          L.p.flags &= ~(unsigned)cg::PF_OUT_RUN;
        }
        L.p.red_out = scratch_red;
        shape_launch(ctx, an, ch, m, k, block, bps, &L, split);
        st = ws_ensure(ctx, L.tickets, L.partial_bytes, stream);
        if (st) break;
        bind_workspace(ctx, an, &L);
        std::string k2 = pair_name(k.name);
        float times[3];
        for (int rep = 0; rep < 4 && st == COOT_OK; ++rep) {
          if (flush) cudaMemsetAsync(flush, rep, flush_bytes, stream);
          cudaEventRecord(e0, stream);
          if (!L.kname_pre.empty()) st = launch_kernel(m, L.kname_pre, L.grid, L.block, &L.p, stream);
          if (!st) st = launch_kernel(m, k.name, L.grid, L.block, &L.p, stream);
          if (!st && var) st = launch_kernel(m, k2, L.grid, L.block, &L.p, stream);
          cudaEventRecord(e1, stream);
          cudaEventSynchronize(e1);
          if (rep > 0) cudaEventElapsedTime(&times[rep - 1], e0, e1);
        }
        if (st) break;
        std::sort(times, times + 3);
        if (log_enabled(ctx))
          fprintf(stderr, "[cootgb]   candidate %s block %d x %d/SM split %d grid %d: %.4f ms\n", k.name.c_str(),
                  block, bps, split, L.grid, times[1]);
        if (times[1] < best_ms) {
          best_ms = times[1];
          best->kidx = ki;
          best->kname = k.name;
          best->block = block;
          best->blocks_per_sm = bps;
          best->split = split;
        }
      }
      if (st) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(stream);
  cudaFree(flush);
  cudaFree(scratch_out);
  cudaFree(scratch_red);
  if (log_enabled(ctx) && st == COOT_OK)
    fprintf(stderr, "[cootgb] tuned %s: %s block %d x %d/SM (%.3f ms)\n", pg.signature.substr(0, 60).c_str(),
            pg.kernels[best->kidx].name.c_str(), best->block, best->blocks_per_sm, best_ms);
  return st;
}
}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" coot_status coot_ctx_create(int device, unsigned flags, coot_ctx** out) {
  if (!out) return set_error(COOT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return set_error(COOT_ERR_INVALID, "device %d not in 0..%d", device, n - 1);
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return set_error(COOT_ERR_UNSUPPORTED, "libcootgb generates sm_103a kernels; device %d is sm_%d%d", device,
                     prop.major, prop.minor);
  coot_ctx* c = new coot_ctx();
  c->device = device;
  c->flags = flags;
  const char* lg = getenv("COOT_LOG");
  if (lg && *lg && strcmp(lg, "0")) c->flags |= COOT_CTX_LOG;
  const char* tu = getenv("COOT_TUNE");
  if (tu && (!strcmp(tu, "on") || !strcmp(tu, "1"))) c->flags |= COOT_CTX_TUNE;
  if (tu && (!strcmp(tu, "off") || !strcmp(tu, "0"))) c->flags &= ~COOT_CTX_TUNE;
  c->sms = prop.multiProcessorCount;
  c->l2_bytes = prop.l2CacheSize;
  const char* cd = getenv("COOT_CACHE_DIR");
  if (cd && *cd)
    c->cache_dir = cd;
  else if (getenv("HOME"))
    c->cache_dir = std::string(getenv("HOME")) + "/.cache/cootgb";
  load_tuning(c);
  {
    DeviceGuard g(device);
    coot_status s = ws_ensure(c, 4096, 1 << 20, nullptr);
    if (s) {
      delete c;
      return s;
    }
  }
  *out = c;
  return COOT_OK;
}

extern "C" coot_status coot_ctx_destroy(coot_ctx* ctx) {
  if (!ctx) return COOT_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->mods)
      if (kv.second->lib) cudaLibraryUnload(kv.second->lib);
    if (ctx->ws) cudaFree(ctx->ws);
    cudaGetLastError();
  }
  delete ctx;
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// fused evaluation
// ---------------------------------------------------------------------------
// call-cache key: every input a fused call's preparation depends on, except
// the data pointers themselves (only their 16-byte alignment and whether they
// are NULL)
static void call_key(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves, const coot_mat* out,
                     coot_reduce red, std::string* key) {
  key->clear();
  auto put = [&](const void* p, size_t n) { key->append((const char*)p, n); };
  put(&tree->n_nodes, sizeof tree->n_nodes);
  put(tree->nodes, sizeof(coot_node) * (size_t)tree->n_nodes);
  put(&n_leaves, sizeof n_leaves);
  auto mat = [&](const coot_mat& m) {
    put(&m.dtype, sizeof m.dtype);
    put(&m.rs, sizeof m.rs);
    put(&m.n_rows, sizeof m.n_rows);
    put(&m.n_cols, sizeof m.n_cols);
    put(&m.ld, sizeof m.ld);
    const unsigned char a = (unsigned char)(((uintptr_t)m.data & 15u) | (m.data ? 0u : 16u));
    put(&a, 1);
  };
  for (int32_t i = 0; i < n_leaves; ++i) mat(leaves[i]);
  const unsigned char has_out = out ? 1 : 0;
  put(&has_out, 1);
  if (out) mat(*out);
  put(&red, sizeof red);
  const char* am = getenv("COOT_ACCUM");  // part of the analysis of FP32 trees
  const unsigned char acc = !am ? 0 : (!strcmp(am, "kahan") ? 1 : (!strcmp(am, "plain") ? 2 : 0));
  put(&acc, 1);
}

extern "C" coot_status coot_eval(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                 const coot_mat* out, coot_reduce red, void* red_out, coot_stream stream) {
  NvtxRange nvtx_range("cootgb eval");
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  const bool keyable = tree && tree->nodes && tree->n_nodes >= 1 && tree->n_nodes <= COOT_MAX_NODES && leaves &&
                       n_leaves >= 1 && n_leaves <= COOT_MAX_LEAVES;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  thread_local std::string key;
  if (keyable) {
    call_key(tree, leaves, n_leaves, out, red, &key);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
      // prepared before: only the checks that depend on the pointers remain
      cg::CallPlan* pl = it->second.get();
      if (red.kind != COOT_R_NONE && !red_out && n_red_outputs(pl->an) > 0)
        return set_error(COOT_ERR_INVALID, "red_out is NULL");
      coot_status s = cg::check_out_alias(pl->an, leaves, out);
      if (s) return s;
      DeviceGuard g(ctx->device);
      return run_fused(ctx, pl->an, leaves, out, red_out, (cudaStream_t)stream, false, pl);
    }
  }
  cg::Analysis an;
  coot_status s = cg::analyse(tree, leaves, n_leaves, out, red, &an);
  if (s) return s;
  if (red.kind != COOT_R_NONE && !red_out && n_red_outputs(an) > 0) return set_error(COOT_ERR_INVALID, "red_out is NULL");
  if (red.kind == COOT_R_NONE && !out) return set_error(COOT_ERR_INVALID, "neither out nor a reduction requested");
  DeviceGuard g(ctx->device);
  // the empty and the two-step (scan of a transposed tree) paths stay uncached
  const bool cacheable = keyable && an.nr * an.nc > 0 && !(an.scan() && an.any_trans);
  if (!cacheable) return run_fused(ctx, an, leaves, out, red_out, (cudaStream_t)stream, false);
  std::unique_ptr<cg::CallPlan> pl(new cg::CallPlan());
  pl->an = an;
  s = run_fused(ctx, pl->an, leaves, out, red_out, (cudaStream_t)stream, false, pl.get());
  if (s) return s;
  if (ctx->plans.size() >= 4096) ctx->plans.clear();  // bounded: a workload of many shapes rebuilds plans
  ctx->plans.emplace(key, std::move(pl));
  return COOT_OK;
}

extern "C" coot_status coot_warmup(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                   const coot_mat* out, coot_reduce red) {
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  cg::Analysis an;
  coot_status s = cg::analyse(tree, leaves, n_leaves, out, red, &an);
  if (s) return s;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  return run_fused(ctx, an, leaves, out, nullptr, nullptr, true);
}

// ---------------------------------------------------------------------------
// unfused baseline: one launch per node, each node materialised
// ---------------------------------------------------------------------------
extern "C" coot_status coot_eval_unfused(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves,
                                         int32_t n_leaves, const coot_mat* out, coot_reduce red, void* red_out,
                                         coot_stream stream_) {
  NvtxRange nvtx_range("cootgb eval unfused");
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  cg::Analysis an;
  coot_status s = cg::analyse(tree, leaves, n_leaves, out, red, &an);
  if (s) return s;
  if (an.dtype == COOT_BF16 || an.dtype == COOT_F16)
    return set_error(COOT_ERR_UNSUPPORTED, "the unfused baseline keeps temporaries in the storage type; use F32/F64/I32");
  if (red.kind != COOT_R_NONE && !red_out && n_red_outputs(an) > 0) return set_error(COOT_ERR_INVALID, "red_out is NULL");
  if (red.kind == COOT_R_NONE && !out) return set_error(COOT_ERR_INVALID, "neither out nor a reduction requested");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  const int nn = tree->n_nodes;
  const int root = nn - 1;
  // reachable nodes (the R_DOT root is folded into the final dot kernel)
  const bool dot = (red.kind == COOT_R_DOT);
  std::vector<char> need(nn, 0);
  std::vector<int> stack = {root};
  while (!stack.empty()) {
    int n = stack.back();
    stack.pop_back();
    if (need[n]) continue;
    need[n] = 1;
    const coot_node& d = tree->nodes[n];
    if (d.op != COOT_N_LEAF) {
      if (d.a >= 0) stack.push_back(d.a);
      if (d.b >= 0 && d.op >= COOT_N_PLUS && d.op <= COOT_N_DIV) stack.push_back(d.b);
    }
  }
  // shape of every node (validated by analyse)
  std::vector<coot_mat> val(nn);
  std::vector<void*> temps;
  auto release = [&]() {
    for (void* t : temps) cudaFreeAsync(t, stream);
  };
  for (int n = 0; n < nn; ++n) {
    if (!need[n]) continue;
    const coot_node& d = tree->nodes[n];
    if (d.op == COOT_N_LEAF) {
      val[n] = leaves[d.leaf];
      val[n].ld = mat_ld(leaves[d.leaf]);
      continue;
    }
    if (d.op == COOT_N_SUBMAT) {  // a view: no kernel
      coot_mat v = val[d.a];
      const int64_t vrs = v.rs > 1 ? v.rs : 1;
      v.data = (char*)v.data + (d.r0 * vrs + d.c0 * v.ld) * an.esz;
      v.n_rows = d.nr;
      v.n_cols = d.nc;
      val[n] = v;
      continue;
    }
    if (d.op == COOT_N_DIAG) {  // a strided view: no kernel
      coot_mat v = val[d.a];
      const int64_t vrs = v.rs > 1 ? v.rs : 1;
      const int64_t k = d.r0, kr = k < 0 ? -k : 0, kc = k > 0 ? k : 0;
      const int64_t len = (k >= 0) ? std::min(v.n_rows, v.n_cols - k) : std::min(v.n_rows + k, v.n_cols);
      v.data = (char*)v.data + (kr * vrs + kc * v.ld) * an.esz;
      v.rs = (int32_t)(vrs + v.ld);
      v.n_rows = std::max<int64_t>(len, 0);
      v.n_cols = 1;
      v.ld = std::max<int64_t>(v.n_rows, 1);
      val[n] = v;
      continue;
    }
    if (n == root && dot) continue;
    // one kernel: node n over its (materialised or viewed) operands
    coot_mat ops[2];
    int nops = 0;
    ops[nops++] = val[d.a];
    bool bin = (d.op >= COOT_N_PLUS && d.op <= COOT_N_DIV);
    if (bin) ops[nops++] = val[d.b];
    coot_node mini[3];
    memset(mini, 0, sizeof mini);
    mini[0].op = COOT_N_LEAF;
    mini[0].leaf = 0;
    mini[0].a = mini[0].b = -1;
    int nmini = 1;
    if (bin) {
      mini[1].op = COOT_N_LEAF;
      mini[1].leaf = 1;
      mini[1].a = mini[1].b = -1;
      nmini = 2;
    }
    coot_node& opn = mini[nmini];
    opn.op = d.op;
    opn.a = 0;
    opn.b = bin ? 1 : -1;
    opn.k = d.k;
    opn.r0 = d.r0;
    opn.c0 = d.c0;
    opn.nr = d.nr;
    opn.nc = d.nc;
    ++nmini;
    coot_tree mt{nmini, 0, mini};
    int64_t r = (d.op == COOT_N_TRANS) ? ops[0].n_cols : ops[0].n_rows;
    int64_t c = (d.op == COOT_N_TRANS) ? ops[0].n_rows : ops[0].n_cols;
    if (d.op == COOT_N_EACH_COL) c = d.nc;
    if (d.op == COOT_N_EACH_ROW) r = d.nr;
    coot_mat dst{};
    if (n == root && out && !dot) {
      dst = *out;
      dst.ld = mat_ld(*out);
    } else {
      void* t = nullptr;
      size_t bytes = (size_t)std::max<int64_t>(r * c, 1) * an.esz;
      cudaError_t e = cudaMallocAsync(&t, bytes, stream);
      if (e != cudaSuccess) {
        release();
        return cuda_error(e, "cudaMallocAsync (unfused temporary)");
      }
      temps.push_back(t);
      dst.data = t;
      dst.dtype = an.dtype;
      dst.n_rows = r;
      dst.n_cols = c;
      dst.ld = std::max<int64_t>(r, 1);
    }
    cg::Analysis man;
    coot_reduce none{COOT_R_NONE, -1, 0, 0};
    s = cg::analyse(&mt, ops, nops, &dst, none, &man);
    if (!s) s = run_fused(ctx, man, ops, &dst, nullptr, stream, false);
    if (s) {
      release();
      return s;
    }
    val[n] = dst;
  }
  // the reduction as its own kernel over the materialised root
  if (red.kind != COOT_R_NONE) {
    coot_node mini[3];
    memset(mini, 0, sizeof mini);
    coot_mat ops[2];
    int nops;
    coot_tree mt;
    if (dot) {
      const coot_node& d = tree->nodes[root];
      ops[0] = val[d.a];
      ops[1] = val[d.b];
      nops = 2;
      mini[0].op = COOT_N_LEAF;
      mini[0].leaf = 0;
      mini[0].a = mini[0].b = -1;
      mini[1].op = COOT_N_LEAF;
      mini[1].leaf = 1;
      mini[1].a = mini[1].b = -1;
      mini[2].op = COOT_N_SCHUR;
      mini[2].a = 0;
      mini[2].b = 1;
      mt = coot_tree{3, 0, mini};
      if (out) {  // the element-wise result still has to be written
        s = coot_eval_unfused(ctx, tree, leaves, n_leaves, out, coot_reduce{COOT_R_NONE, -1, 0, 0}, nullptr, stream_);
        if (s) {
          release();
          return s;
        }
      }
    } else {
      ops[0] = val[root];
      nops = 1;
      mini[0].op = COOT_N_LEAF;
      mini[0].leaf = 0;
      mini[0].a = mini[0].b = -1;
      mt = coot_tree{1, 0, mini};
    }
    cg::Analysis man;
    const coot_mat* ro = (red.kind == COOT_R_CUMSUM) ? out : nullptr;  // cumsum scans out in place
    s = cg::analyse(&mt, ops, nops, ro, red, &man);
    if (!s) s = run_fused(ctx, man, ops, ro, red_out, stream, false);
    if (s) {
      release();
      return s;
    }
  }
  const int rop = tree->nodes[root].op;
  if ((rop == COOT_N_LEAF || rop == COOT_N_SUBMAT || rop == COOT_N_DIAG) && out && red.kind != COOT_R_CUMSUM) {
    // a bare leaf or view: one copy kernel
    coot_node mini[1];
    memset(mini, 0, sizeof mini);
    mini[0].op = COOT_N_LEAF;
    mini[0].leaf = 0;
    mini[0].a = mini[0].b = -1;
    coot_tree mt{1, 0, mini};
    coot_mat op0 = val[root];
    cg::Analysis man;
    coot_reduce none{COOT_R_NONE, -1, 0, 0};
    s = cg::analyse(&mt, &op0, 1, out, none, &man);
    if (!s) s = run_fused(ctx, man, &op0, out, nullptr, stream, false);
    if (s) {
      release();
      return s;
    }
  }
  release();
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// GEMM with the tree fused onto the product
// ---------------------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return (EncodeTiledFn)f;
  }();
  return fn;
}

// TMA descriptor of an operand stored column-major (column stride ld
// elements), 128-byte swizzle, zeros outside; false when the driver rejects
// it.  K adjacent: a K x rows array read in boxes of 64 K values x box_rows
// rows; else a rows x K array read in boxes of 64 rows x 64 K values.
bool tma_map(unsigned long long* dst, const void* data, int dtype, bool kmaj, int64_t k, int64_t rows, int64_t ld,
             int box_rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)(kmaj ? k : rows), (cuuint64_t)(kmaj ? rows : k)};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)(kmaj ? coot::GEMM_TC_BK : 64),
                             (cuuint32_t)(kmaj ? box_rows : coot::GEMM_TC_BK)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, dtype == COOT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(data), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  static_assert(sizeof(CUtensorMap) == 16 * sizeof(unsigned long long), "CUtensorMap is 128 bytes");
  memcpy(dst, &map, sizeof map);
  return true;
}

}  // namespace

extern "C" coot_status coot_gemm_eval(coot_ctx* ctx, const coot_mat* A, int32_t trans_a, const coot_mat* B,
                                      int32_t trans_b, const coot_tree* epi, const coot_mat* extra, int32_t n_extra,
                                      const coot_mat* out, coot_stream stream_) {
  NvtxRange nvtx_range("cootgb gemm");
  if (!ctx || !A || !B || !out) return set_error(COOT_ERR_INVALID, "ctx, A, B or out is NULL");
  if (n_extra < 0 || n_extra > COOT_MAX_LEAVES - 1 || (n_extra > 0 && !extra))
    return set_error(COOT_ERR_INVALID, "n_extra %d outside 0..%d (or extra NULL)", n_extra, COOT_MAX_LEAVES - 1);
  if (A->dtype != B->dtype || A->dtype != out->dtype)
    return set_error(COOT_ERR_DTYPE, "A, B and out must share one dtype");
  if (A->dtype == COOT_I32) return set_error(COOT_ERR_UNSUPPORTED, "the fused GEMM takes BF16, FP16, FP32 or FP64");
  const bool simt = A->dtype == COOT_F32 || A->dtype == COOT_F64;  // CUDA-core kernel
  if (A->rs > 1 || B->rs > 1) return set_error(COOT_ERR_UNSUPPORTED, "GEMM operands need adjacent rows");
  const int64_t m = trans_a ? A->n_cols : A->n_rows, k = trans_a ? A->n_rows : A->n_cols;
  const int64_t kb = trans_b ? B->n_cols : B->n_rows, n = trans_b ? B->n_rows : B->n_cols;
  if (k != kb)
    return set_error(COOT_ERR_SHAPE, "op(A) is %lldx%lld, op(B) %lldx%lld", (long long)m, (long long)k,
                     (long long)kb, (long long)n);
  if ((m * k > 0 && !A->data) || (k * n > 0 && !B->data)) return set_error(COOT_ERR_INVALID, "A or B: NULL data");
  const int64_t lda = mat_ld(*A), ldb = mat_ld(*B);
  if ((A->n_cols > 1 && lda < A->n_rows) || (B->n_cols > 1 && ldb < B->n_rows))
    return set_error(COOT_ERR_INVALID, "A or B: ld smaller than the rows");
  // the epilogue tree: leaf 0 is the product, a placeholder with out's exact
  // layout (never read; out then aliases it only through an identical view)
  std::vector<coot_mat> lv(1 + n_extra);
  lv[0] = *out;
  for (int i = 0; i < n_extra; ++i) lv[1 + i] = extra[i];
  coot_node only{};
  only.op = COOT_N_LEAF;
  only.a = only.b = -1;
  const coot_tree single{1, 0, &only};
  const coot_tree* tree = epi ? epi : &single;
  cg::Analysis an;
  coot_status s = cg::analyse(tree, lv.data(), 1 + n_extra, out, coot_reduce{COOT_R_NONE, -1, 0, 0}, &an);
  if (s) return s;
  if (an.nr != m || an.nc != n) return set_error(COOT_ERR_SHAPE, "the epilogue is not m x n");
  if (an.any_trans) return set_error(COOT_ERR_UNSUPPORTED, "transposed reads in a GEMM epilogue");
  int ps = -1;
  for (size_t i = 0; i < an.slots.size(); ++i)
    if (an.slots[i].leaf == 0) {
      const cg::Slot& sl = an.slots[i];
      if (ps >= 0 || sl.gen || sl.off != 0 || (an.nc > 1 && sl.cs != mat_ld(*out)))
        return set_error(COOT_ERR_UNSUPPORTED, "the product must be read whole and untransposed, once");
      ps = (int)i;
    }
  if (ps < 0) return set_error(COOT_ERR_INVALID, "the epilogue does not read the product (leaf 0)");
  // out may not overlap the operands
  auto range = [](const coot_mat& X, int64_t r, int64_t c, uintptr_t* lo, uintptr_t* hi) {
    const int esz = (X.dtype == COOT_F64) ? 8 : ((X.dtype == COOT_BF16 || X.dtype == COOT_F16) ? 2 : 4);
    *lo = (uintptr_t)X.data;
    *hi = (r > 0 && c > 0) ? *lo + (uintptr_t)(((r - 1) + (c - 1) * mat_ld(X) + 1) * esz) : *lo;
  };
  uintptr_t olo, ohi, alo, ahi, blo, bhi;
  range(*out, m, n, &olo, &ohi);
  range(*A, A->n_rows, A->n_cols, &alo, &ahi);
  range(*B, B->n_rows, B->n_cols, &blo, &bhi);
  if ((olo < ahi && alo < ohi) || (olo < bhi && blo < ohi))
    return set_error(COOT_ERR_ALIAS, "out overlaps a GEMM operand");
  if (m == 0 || n == 0) return COOT_OK;
  an.gemm_ps = ps;
  an.gemm_ka = trans_a != 0;  // A stored k x m: K adjacent
  an.gemm_kb = trans_b == 0;  // B stored k x n: K adjacent
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaStream_t stream = (cudaStream_t)stream_;
  cg::Program pg = cg::make_program(an, cg::F_GEMM, false);
  if (!ctx->mods.count(pg.signature) && capturing(stream))
    return set_error(COOT_ERR_INVALID, "this GEMM's kernel is not compiled yet; run the call once before capturing");
  cg::Module* mod = nullptr;
  s = coot_get_module(ctx, pg, &mod);
  if (s) return s;
  s = ws_ensure(ctx, 1, 0, stream);
  if (s) return s;
  coot::GemmParams gp{};
  cg::Params& p = gp.p;
  for (size_t i = 0; i < an.slots.size(); ++i) {
    const cg::Slot& sl = an.slots[i];
    p.src[i] = ((int)i == ps) ? nullptr : (const char*)lv[sl.leaf].data + sl.off * an.esz;
    p.ld[i] = sl.cs;
    p.rs[i] = sl.rs;
  }
  for (size_t i = 0; i < an.scalars.size(); ++i) p.k[i] = scalar_bits(an.scalars[i], an.ct);
  p.out = out->data;
  p.out_ld = mat_ld(*out);
  p.out_rs = an.out_rs;
  p.err_flag = ctx->err_flag;
  gp.a = A->data;
  gp.b = B->data;
  gp.lda = lda;
  gp.ldb = ldb;
  gp.m = m;
  gp.n = n;
  gp.k = k;
  gp.vec = ((uintptr_t)A->data % 16 == 0 && (uintptr_t)B->data % 16 == 0 && (lda % 8 == 0 || A->n_cols <= 1) &&
            (ldb % 8 == 0 || B->n_cols <= 1))
               ? 1
               : 0;
  const int64_t tile = simt ? (A->dtype == COOT_F32 ? 128 : 64) : coot::GEMM_TILE;
  const dim3 grid((unsigned)ceil_div(m, tile), (unsigned)ceil_div(n, tile));
  if (ceil_div(n, tile) > 65535 || ceil_div(m, tile) >= ((int64_t)1 << 31))
    return set_error(COOT_ERR_UNSUPPORTED, "%lld x %lld is too large for one launch", (long long)m, (long long)n);
  // tcgen05 path: 16-byte aligned bases and column strides (TMA),
  // coordinates within int32
  const int64_t lim = (int64_t)1 << 31;
  bool tc = !simt && !(ctx->flags & COOT_CTX_NO_TCGEN05) && k > 0 && m < lim && n < lim && k < lim &&
            (uintptr_t)A->data % 16 == 0 && (uintptr_t)B->data % 16 == 0 && lda % 8 == 0 && ldb % 8 == 0;
  if (tc)
    tc = tma_map(gp.tma_a, A->data, A->dtype, an.gemm_ka, k, m, lda, coot::GEMM_TC_BM) &&
         tma_map(gp.tma_b, B->data, B->dtype, an.gemm_kb, k, n, ldb, coot::GEMM_TC_BN);
  cudaError_t e;
  const char* kname = simt ? "coot_gemm_simt" : (tc ? "coot_gemm_tc" : "coot_gemm");
  int block = 256;
  unsigned n_blocks = grid.x * grid.y;
  void* args[] = {&gp};
  if (tc) {
    gp.tiles_m = ceil_div(m, coot::GEMM_TC_BM);
    gp.tiles_n = ceil_div(n, coot::GEMM_TC_BN);
    if (gp.tiles_m * gp.tiles_n >= lim) return set_error(COOT_ERR_UNSUPPORTED, "too many output tiles");
    const void* kf = (const void*)mod->kernels[kname];
    if (!mod->gemm_tc_smem) {
      e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, coot::GEMM_TC_SMEM);
      if (e != cudaSuccess) return cuda_error(e, "coot_gemm_tc shared memory");
      mod->gemm_tc_smem = true;
    }
    block = coot::GEMM_TC_THREADS;  // persistent: at most one CTA per SM
    n_blocks = (unsigned)std::min<int64_t>(gp.tiles_m * gp.tiles_n, std::max(ctx->sms, 1));
    e = cudaLaunchKernel(kf, dim3(n_blocks), dim3(block), args, coot::GEMM_TC_SMEM, stream);
  } else {
    e = cudaLaunchKernel((const void*)mod->kernels[kname], grid, dim3(block), args, 0, stream);
  }
  if (e != cudaSuccess) return cuda_error(e, kname);
  coot_launch_info& li = ctx->last;
  memset(&li, 0, sizeof li);
  snprintf(li.kernel, sizeof li.kernel, "%s", kname);
  li.grid = (int)n_blocks;
  li.block = block;
  li.vec = gp.vec ? 8 : 1;
  li.unroll = 1;
  li.n_launches = 1;
  int64_t extra_bytes = 0;
  for (size_t i = 0; i < an.slots.size(); ++i)
    if ((int)i != ps) extra_bytes += an.slots[i].n_distinct * an.esz;
  li.algorithmic_bytes = (m * k + k * n + m * n) * an.esz + extra_bytes;
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
extern "C" coot_status coot_eval_adjoint(coot_ctx* ctx, const coot_tree* tree, const coot_mat* leaves,
                                         int32_t n_leaves, coot_reduce red, const void* upstream,
                                         const coot_mat* grads, coot_stream stream_) {
  NvtxRange nvtx_range("cootgb adjoint");
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!upstream || !grads) return set_error(COOT_ERR_INVALID, "upstream or grads is NULL");
  const bool ok_red = red.kind == COOT_R_ACCU || red.kind == COOT_R_DOT ||
                      ((red.kind == COOT_R_SUM || red.kind == COOT_R_MEAN) && red.dim == -1);
  if (!ok_red)
    return set_error(COOT_ERR_UNSUPPORTED, "the adjoint covers accu / sum / mean over all elements (and dot)");
  cg::Analysis an;
  coot_status s = cg::analyse(tree, leaves, n_leaves, nullptr, red, &an);
  if (s) return s;
  if (an.dtype != COOT_F32 && an.dtype != COOT_F64)
    return set_error(COOT_ERR_UNSUPPORTED, "the adjoint is implemented for F32 and F64 leaves");
  std::vector<int> uses(n_leaves, 0);
  for (const cg::Slot& sl : an.slots) {
    if (sl.trans || !sl.full)
      return set_error(COOT_ERR_UNSUPPORTED, "the adjoint needs every leaf read whole and untransposed");
    if (++uses[sl.leaf] > 1) return set_error(COOT_ERR_UNSUPPORTED, "leaf %d is read through two views", sl.leaf);
  }
  for (int i = 0; i < n_leaves; ++i) {
    if (!grads[i].data) continue;
    if (grads[i].dtype != an.dtype || grads[i].n_rows != leaves[i].n_rows || grads[i].n_cols != leaves[i].n_cols)
      return set_error(COOT_ERR_SHAPE, "grads[%d] must match leaf %d in shape and dtype", i, i);
  }
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  const int64_t count = an.nr * an.nc;
  if (count == 0) return COOT_OK;
  // iteration shape: one long column when every read and gradient is contiguous
  cg::Choice ch;
  ch.fam = cg::F_ADJ;
  bool contig = true, vec = true;
  for (size_t i = 0; i < an.slots.size(); ++i) {
    const coot_mat& L = leaves[an.slots[i].leaf];
    if (an.nc > 1 && mat_ld(L) != an.nr) contig = false;
    if ((uintptr_t)L.data % 16) vec = false;
    const coot_mat& G = grads[an.slots[i].leaf];
    if (G.data) {
      if (an.nc > 1 && mat_ld(G) != an.nr) contig = false;
      if ((uintptr_t)G.data % 16) vec = false;
    }
  }
  if (!contig) {
    for (size_t i = 0; i < an.slots.size(); ++i) {
      const coot_mat& L = leaves[an.slots[i].leaf];
      const coot_mat& G = grads[an.slots[i].leaf];
      if ((mat_ld(L) * an.esz) % 16) vec = false;
      if (G.data && (mat_ld(G) * an.esz) % 16) vec = false;
    }
  }
  ch.collapsed = contig;
  ch.vec_ok = vec;
  ch.it_rows = contig ? count : an.nr;
  ch.it_cols = contig ? 1 : an.nc;
  const bool bounds = (ctx->flags & COOT_CTX_DEBUG_BOUNDS) != 0;
  cg::Program pg = cg::make_program(an, cg::F_ADJ, false, bounds);
  if (!ctx->mods.count(pg.signature) && capturing(stream))
    return set_error(COOT_ERR_INVALID, "compile the adjoint before capturing");
  cg::Module* m = nullptr;
  if ((s = coot_get_module(ctx, pg, &m))) return s;
  Launch L;
  cg::Params& p = L.p;
  for (size_t i = 0; i < an.slots.size(); ++i) {
    const coot_mat& Lf = leaves[an.slots[i].leaf];
    p.src[i] = Lf.data;
    p.ld[i] = mat_ld(Lf);
    const coot_mat& G = grads[an.slots[i].leaf];
    p.grad[i] = G.data;
    p.grad_ld[i] = G.data ? mat_ld(G) : 0;
  }
  if (bounds) set_extents(an, leaves, nullptr, &p);
  for (size_t i = 0; i < an.scalars.size(); ++i) p.k[i] = scalar_bits(an.scalars[i], an.ct);
  p.upstream = upstream;
  p.grad_mult = (red.kind == COOT_R_MEAN) ? 1.0 / (double)count : 1.0;
  int kidx = default_variant(pg, ch);
  const cg::KernelSpec& ks = pg.kernels[kidx];
  int bps = occupancy(m, ks.name, 512);
  shape_launch(ctx, an, ch, m, ks, 512, bps, &L);
  if ((s = ws_ensure(ctx, 1, 0, stream))) return s;
  p.err_flag = ctx->err_flag;
  p.tickets = ctx->tickets;
  p.partials = ctx->partials;
  p.mu = ctx->mean_ptr;
  if ((s = launch_kernel(m, ks.name, L.grid, L.block, &p, stream))) return s;
  coot_launch_info& li = ctx->last;
  memset(&li, 0, sizeof li);
  snprintf(li.kernel, sizeof li.kernel, "%s", ks.name.c_str());
  li.grid = L.grid;
  li.block = L.block;
  li.vec = ks.vec;
  li.unroll = ks.unroll;
  li.n_launches = 1;
  int64_t b = 0;
  for (const cg::Slot& sl : an.slots) {
    b += count * an.esz;
    if (grads[sl.leaf].data) b += count * an.esz;
  }
  li.algorithmic_bytes = b;
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// batched evaluation
// ---------------------------------------------------------------------------
extern "C" coot_status coot_batch_create(coot_ctx* ctx, const coot_tree* tree, int64_t n_problems, int32_t n_leaves,
                                         const coot_mat* problems, const coot_mat* outs, coot_reduce red,
                                         coot_batch** out) {
  if (!ctx || !out || !problems) return set_error(COOT_ERR_INVALID, "ctx, problems or out is NULL");
  *out = nullptr;
  if (n_problems < 1) return set_error(COOT_ERR_INVALID, "n_problems must be >= 1");
  const bool ok_red = red.kind == COOT_R_NONE || red.kind == COOT_R_ACCU ||
                      ((red.kind == COOT_R_SUM || red.kind == COOT_R_MEAN) && red.dim == -1);
  if (!ok_red) return set_error(COOT_ERR_UNSUPPORTED, "batched reductions: accu / sum / mean over all elements");
  if (red.kind == COOT_R_NONE && !outs) return set_error(COOT_ERR_INVALID, "neither outs nor a reduction requested");
  cg::Analysis an0;
  coot_status s = cg::analyse(tree, problems, n_leaves, outs ? &outs[0] : nullptr, red, &an0);
  if (s) return set_error(s, "problem 0: %s", coot_last_error());
  std::vector<coot::BatchProblem> probs((size_t)n_problems);
  std::vector<long long> begin((size_t)n_problems + 1);
  long long tiles = 0;
  int64_t bytes = 0;
  for (int64_t q = 0; q < n_problems; ++q) {
    cg::Analysis an;
    const coot_mat* lv = &problems[q * n_leaves];
    s = cg::analyse(tree, lv, n_leaves, outs ? &outs[q] : nullptr, red, &an);
    if (s) return set_error(s, "problem %lld: %s", (long long)q, coot_last_error());
    if (an.dtype != an0.dtype || an.slots.size() != an0.slots.size() || an.trmask != an0.trmask)
      return set_error(COOT_ERR_INVALID, "problem %lld differs in dtype or leaf reads", (long long)q);
    if (an.gmask)
      return set_error(COOT_ERR_UNSUPPORTED, "problem %lld: row-broadcast, diagonal or row-strided reads and outputs "
                       "are not batched", (long long)q);
    if (an.nr >= INT32_MAX || an.nc >= INT32_MAX)
      return set_error(COOT_ERR_UNSUPPORTED, "problem %lld: %lld x %lld; batched problems have fewer than 2^31 - 1 "
                       "rows and columns", (long long)q, (long long)an.nr, (long long)an.nc);
    coot::BatchProblem& bp = probs[q];
    memset(&bp, 0, sizeof bp);
    for (size_t i = 0; i < an.slots.size(); ++i) {
      const cg::Slot& sl = an.slots[i];
      const coot_mat& L = lv[sl.leaf];
      bp.src[i] = (const char*)L.data + sl.off * an.esz;
      bp.ld[i] = sl.trans ? sl.rs : sl.cs;
      bytes += sl.n_distinct * an.esz;
    }
    if (outs) {
      bp.out = outs[q].data;
      bp.out_ld = mat_ld(outs[q]);
      bytes += an.nr * an.nc * an.esz;
    }
    bp.n_rows = an.nr;
    bp.n_cols = an.nc;
    int64_t ntr = std::max<int64_t>(1, ceil_div(an.nr, 32));
    int64_t ntc = std::max<int64_t>(1, ceil_div(an.nc, 32));
    bp.n_tile_rows = ntr;
    bp.tile_begin = tiles;
    begin[q] = tiles;
    tiles += ntr * ntc;
  }
  begin[n_problems] = tiles;
  if (red.kind != COOT_R_NONE) bytes += n_problems * rsize(an0.ct);
  // the kernel: the flat walk over work items unless COOT_BATCH_KERNEL=tile
  const char* kenv = getenv("COOT_BATCH_KERNEL");
  const bool flat = !(kenv && strcmp(kenv, "tile") == 0);
  if (!flat && tiles >= (1ll << 31)) return set_error(COOT_ERR_UNSUPPORTED, "%lld tiles: at most 2^31 - 1", tiles);
  // owning problem of every tile: one load per tile instead of a search
  std::vector<int> tile_prob(flat ? 0 : (size_t)tiles);
  if (!flat)
    for (int64_t q = 0; q < n_problems; ++q)
      for (long long t = begin[q]; t < begin[q + 1]; ++t) tile_prob[(size_t)t] = (int)q;
  // flat kernel: cut every problem into rectangles of whole columns (or, for
  // problems taller than an item, row chunks of one column) with
  // w * (h | 1) <= BE elements, in problem order
  std::vector<coot::BatchItem> items;
  if (flat) {
    int ntr = 0;
    for (int s = 0; s < 32; ++s) ntr += (an0.trmask >> s) & 1;
    // elements per item (COOT_BATCH_BE, 1024 .. 8192, for measurements) and
    // the register cap (COOT_BATCH_MINB resident blocks, 2 .. 6)
    int base = 8192;
    if (const char* be = getenv("COOT_BATCH_BE")) base = std::min(8192, std::max(1024, atoi(be)));
    if (const char* mb = getenv("COOT_BATCH_MINB")) an0.batch_minb = std::min(6, std::max(2, atoi(mb)));
    const int64_t BE = coot::batchf_elems(ntr, (an0.ct == cg::CT_F64) ? 8 : 4, base);
    an0.batch_be = (int)BE;
    const char* ienv = getenv("COOT_BATCH_ITEMS");
    const bool cols_items = !(ienv && strcmp(ienv, "tiles") == 0);
    items.reserve((size_t)n_problems * 2);
    for (int64_t q = 0; q < n_problems; ++q) {
      const int64_t r = probs[q].n_rows, c = probs[q].n_cols;
      const size_t first = items.size();
      auto push = [&](int64_t i0, int64_t j0, int64_t h, int64_t w) {
        coot::BatchItem it;
        memset(&it, 0, sizeof it);
        it.q = (int)q;
        it.i0 = (int)i0;
        it.j0 = (int)j0;
        it.h = (int)h;
        it.w = (int)w;
        it.first = (int)first;
        const int NB = coot::BATCHF_BLOCK;
        if (h > 0 && w > 0) {
          it.mh = (unsigned)(((1ull << 24) + (uint64_t)h - 1) / (uint64_t)h);
          it.mw = (unsigned)(((1ull << 24) + (uint64_t)w - 1) / (uint64_t)w);
          it.dih = (int)(NB % h);
          it.djh = (int)(NB / h);
          it.diw = (int)(NB % w);
          it.djw = (int)(NB / w);
        }
        items.push_back(it);
      };
      // item shape H x W: whole columns when they are short; otherwise runs
      // of at least 32 elements along both dimensions, so that the direct
      // reads (runs along columns) and the staged transposed reads (runs
      // along rows) both stay coalesced
      int64_t H, W;
      if (cols_items && (r | 1) <= BE) {  // whole columns whenever they fit
        H = r;
        W = std::max<int64_t>(1, BE / (r | 1));
      } else if (r <= 127) {
        H = r;
        W = std::max<int64_t>(1, BE / (r | 1));
      } else if (c <= 32) {
        W = c;
        H = BE / W;
        if (H >= r)
          H = ((r | 1) * W <= BE) ? r : r - 1;  // r - 1 is odd when r is even
        else if (H % 2 == 0)
          H -= 1;  // odd, so that every chunk keeps w * (h | 1) <= BE
      } else {
        H = 127;
        W = std::min<int64_t>(32, BE / 127);
      }
      if (r == 0 || c == 0) {
        push(0, 0, r, c);  // nothing to walk: writes the empty result
      } else {
        for (int64_t j0 = 0; j0 < c; j0 += W)
          for (int64_t i0 = 0; i0 < r; i0 += H) push(i0, j0, std::min(H, r - i0), std::min(W, c - j0));
      }
      for (size_t t = first; t < items.size(); ++t) items[t].nk = (int)(items.size() - first);
    }
    if (items.size() >= (size_t)INT32_MAX)
      return set_error(COOT_ERR_UNSUPPORTED, "%zu work items: at most 2^31 - 1", items.size());
  }

  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cg::Program pg = cg::make_program(an0, cg::F_BATCH, false);
  cg::Module* m = nullptr;
  if ((s = coot_get_module(ctx, pg, &m))) return s;
  if ((s = ws_ensure(ctx, 1, 0, nullptr))) return s;

  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_probs = 0;
  const size_t o_begin = align(o_probs + probs.size() * sizeof(coot::BatchProblem));
  const size_t o_map = align(o_begin + begin.size() * sizeof(long long));
  const size_t o_items = align(o_map + tile_prob.size() * sizeof(int));
  const size_t o_done = align(o_items + items.size() * sizeof(coot::BatchItem));
  const size_t o_queue = align(o_done + (size_t)n_problems * sizeof(unsigned));
  const size_t o_part = align(o_queue + 2 * sizeof(unsigned));
  const size_t total = align(o_part + (size_t)(flat ? (int64_t)items.size() : tiles) * 8);
  coot_batch* b = new coot_batch();
  cudaError_t e = cudaMalloc(&b->dev_mem, total);
  if (e != cudaSuccess) {
    delete b;
    return cuda_error(e, "batch cudaMalloc");
  }
  char* base = (char*)b->dev_mem;
  if ((e = cudaMemcpy(base + o_probs, probs.data(), probs.size() * sizeof(coot::BatchProblem),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(base + o_begin, begin.data(), begin.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(base + o_map, tile_prob.data(), tile_prob.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(base + o_items, items.data(), items.size() * sizeof(coot::BatchItem),
                      cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(base + o_done, 0, o_part - o_done)) != cudaSuccess) {
    cudaFree(b->dev_mem);
    delete b;
    return cuda_error(e, "batch upload");
  }
  b->ctx = ctx;
  b->mod = m;
  b->kname = flat ? "coot_batchf" : "coot_batch";
  b->n_problems = n_problems;
  b->has_red = red.kind != COOT_R_NONE;
  {
    // one warp per tile; as many warps per block as the transposed tiles'
    // shared memory allows within 48 KiB (the kernel computes the same)
    int ntr = 0;
    for (int s = 0; s < 32; ++s) ntr += (an0.trmask >> s) & 1;
    const int csize = (an0.ct == cg::CT_F64) ? 8 : 4;
    const int per = 32 * 33 * csize * std::max(ntr, 1);
    const int warps = (ntr == 0) ? 8 : std::max(1, std::min(8, 49152 / per));
    b->block = flat ? coot::BATCHF_THREADS : 32 * warps;
  }
  b->grid = ctx->sms * occupancy(m, b->kname, b->block);
  b->algorithmic_bytes = bytes;
  coot::BatchParams& bp = b->bp;
  memset(&bp, 0, sizeof bp);
  bp.probs = (const coot::BatchProblem*)(base + o_probs);
  bp.tile_begin = (const long long*)(base + o_begin);
  bp.tile_prob = (const int*)(base + o_map);
  bp.items = (const coot::BatchItem*)(base + o_items);
  bp.n_items = (long long)items.size();
  bp.n_problems = n_problems;
  bp.n_tiles = tiles;
  // a few tiles per queue pop: fewer atomics, still fine-grained balance
  bp.chunk = std::max<long long>(1, std::min<long long>(8, tiles / ((long long)b->grid * (b->block / 32) * 8)));
  for (size_t i = 0; i < an0.scalars.size(); ++i) bp.k[i] = scalar_bits(an0.scalars[i], an0.ct);
  bp.partials = base + o_part;
  bp.done = (unsigned*)(base + o_done);
  bp.queue = (unsigned*)(base + o_queue);
  bp.err_flag = ctx->err_flag;
  bp.has_out = outs ? 1 : 0;
  bp.mean = (red.kind == COOT_R_MEAN) ? 1 : 0;
  *out = b;
  return COOT_OK;
}

extern "C" coot_status coot_batch_run(coot_batch* b, void* red_out, coot_stream stream) {
  NvtxRange nvtx_range("cootgb batch");
  if (!b) return set_error(COOT_ERR_INVALID, "batch is NULL");
  if (b->has_red && !red_out) return set_error(COOT_ERR_INVALID, "red_out is NULL");
  std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
  DeviceGuard g(b->ctx->device);
  coot::BatchParams bp = b->bp;
  bp.red_out = red_out;
  coot_status s = launch_kernel(b->mod, b->kname, b->grid, b->block, &bp, (cudaStream_t)stream);
  if (s) return s;
  coot_launch_info& li = b->ctx->last;
  memset(&li, 0, sizeof li);
  snprintf(li.kernel, sizeof li.kernel, "%s", b->kname.c_str());
  li.grid = b->grid;
  li.block = b->block;
  li.vec = 1;
  li.unroll = 1;
  li.n_launches = 1;
  li.algorithmic_bytes = b->algorithmic_bytes;
  return COOT_OK;
}

extern "C" coot_status coot_batch_destroy(coot_batch* b) {
  if (!b) return COOT_OK;
  {
    DeviceGuard g(b->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(b->dev_mem);
    cudaGetLastError();
  }
  delete b;
  return COOT_OK;
}

extern "C" coot_status coot_eval_batched(coot_ctx* ctx, const coot_tree* tree, int64_t n_problems, int32_t n_leaves,
                                         const coot_mat* problems, const coot_mat* outs, coot_reduce red,
                                         void* red_out, coot_stream stream) {
  coot_batch* b = nullptr;
  coot_status s = coot_batch_create(ctx, tree, n_problems, n_leaves, problems, outs, red, &b);
  if (s) return s;
  s = coot_batch_run(b, red_out, stream);
  {
    DeviceGuard g(ctx->device);
    // release the plan's table in stream order
    cudaFreeAsync(b->dev_mem, (cudaStream_t)stream);
    b->dev_mem = nullptr;
    cudaGetLastError();
  }
  delete b;
  return s;
}

// ---------------------------------------------------------------------------
// CUDA graphs
// ---------------------------------------------------------------------------
extern "C" coot_status coot_graph_begin(coot_ctx* ctx, coot_stream stream) {
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  if (!stream) return set_error(COOT_ERR_INVALID, "capture needs a non-default stream");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
  return COOT_OK;
}

extern "C" coot_status coot_graph_end(coot_ctx* ctx, coot_stream stream, coot_graph** out) {
  if (!ctx || !out) return set_error(COOT_ERR_INVALID, "ctx or out is NULL");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  coot_graph* gr = new coot_graph();
  cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &gr->graph);
  if (e != cudaSuccess) {
    delete gr;
    return cuda_error(e, "cudaStreamEndCapture");
  }
  e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gr->graph);
    delete gr;
    return cuda_error(e, "cudaGraphInstantiate");
  }
  *out = gr;
  return COOT_OK;
}

extern "C" coot_status coot_graph_launch(coot_graph* gr, coot_stream stream) {
  if (!gr) return set_error(COOT_ERR_INVALID, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(gr->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
  return COOT_OK;
}

extern "C" coot_status coot_graph_destroy(coot_graph* gr) {
  if (!gr) return COOT_OK;
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  delete gr;
  return COOT_OK;
}

// ---------------------------------------------------------------------------
// host-side introspection
// ---------------------------------------------------------------------------
static coot_status analyse_for_host(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                    const coot_mat* out, coot_reduce red, cg::Analysis* an, cg::Program* pg) {
  coot_status s = cg::analyse(tree, leaves, n_leaves, out, red, an);
  if (s) return s;
  cg::Choice ch = cg::choose(*an, leaves, out);
  *pg = cg::make_program(*an, ch.fam, an->two_pass());
  return COOT_OK;
}

extern "C" coot_status coot_signature(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                      const coot_mat* out, coot_reduce red, char* buf, size_t len) {
  cg::Analysis an;
  cg::Program pg;
  coot_status s = analyse_for_host(tree, leaves, n_leaves, out, red, &an, &pg);
  if (s) return s;
  if (!buf || len == 0) return set_error(COOT_ERR_INVALID, "buf is NULL");
  if (pg.signature.size() + 1 > len) return set_error(COOT_ERR_INVALID, "buf too small (%zu needed)", pg.signature.size() + 1);
  memcpy(buf, pg.signature.c_str(), pg.signature.size() + 1);
  return COOT_OK;
}

extern "C" coot_status coot_codegen(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                    const coot_mat* out, coot_reduce red, char* buf, size_t len) {
  cg::Analysis an;
  cg::Program pg;
  coot_status s = analyse_for_host(tree, leaves, n_leaves, out, red, &an, &pg);
  if (s) return s;
  if (!buf || len == 0) return set_error(COOT_ERR_INVALID, "buf is NULL");
  if (pg.source.size() + 1 > len) return set_error(COOT_ERR_INVALID, "buf too small (%zu needed)", pg.source.size() + 1);
  memcpy(buf, pg.source.c_str(), pg.source.size() + 1);
  return COOT_OK;
}

extern "C" coot_status coot_compile(const coot_tree* tree, const coot_mat* leaves, int32_t n_leaves,
                                    const coot_mat* out, coot_reduce red, size_t* cubin_bytes) {
  cg::Analysis an;
  cg::Program pg;
  coot_status s = analyse_for_host(tree, leaves, n_leaves, out, red, &an, &pg);
  if (s) return s;
  std::vector<char> cubin;
  std::string log;
  s = cg::nvrtc_compile(pg.source, &cubin, &log);
  if (s) return s;
  if (cubin_bytes) *cubin_bytes = cubin.size();
  return COOT_OK;
}

extern "C" coot_status coot_check_device_flag(coot_ctx* ctx, coot_stream stream, uint32_t* flags) {
  if (!ctx) return set_error(COOT_ERR_INVALID, "ctx is NULL");
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
  unsigned f = 0;
  if ((e = cudaMemcpy(&f, ctx->err_flag, sizeof f, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_error(e, "read device flag");
  if (f && (e = cudaMemset(ctx->err_flag, 0, sizeof f)) != cudaSuccess) return cuda_error(e, "clear device flag");
  if (flags) *flags = f;
  if (f)
    return set_error(COOT_ERR_DEVICE_FLAG,
                     "device flag 0x%x (bit 0: INT32 division by zero; bit 1: a bounded wait timed out; bit 2: an "
                     "access outside a matrix)",
                     f);
  return COOT_OK;
}

extern "C" coot_status coot_last_launch(coot_ctx* ctx, coot_launch_info* info) {
  if (!ctx || !info) return set_error(COOT_ERR_INVALID, "ctx or info is NULL");
  *info = ctx->last;
  return COOT_OK;
}
