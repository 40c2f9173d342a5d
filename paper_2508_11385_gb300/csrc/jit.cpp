// jit.cpp -- per-tree kernel compilation and caching.
//
// The paper (Sec. 4) compiles its predefined kernel set for the device at
// start-up and caches the result, a one-time cost that its timings exclude
// (Sec. 5).  Here each distinct tree signature is compiled once by NVRTC for
// sm_103a; the cubin is kept in memory per context and on disk under
// $COOT_CACHE_DIR (default ~/.cache/cootgb).  A disk entry carries the
// signature and an FNV-1a checksum of its payload; a truncated or corrupted
// entry is ignored and recompiled.
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "coot_internal.h"

#include "_embedded.inc"  // k_headers[]: {name, text} of the device headers

namespace cg {

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

static std::vector<const char*> nvrtc_options() {
  std::vector<const char*> o = {"-arch=sm_103a", "-std=c++17", "-fmad=false", "-default-device", "-lineinfo",
                                "-DCOOT_JIT=1"};
  // fault injection for the error-path tests: an option NVRTC rejects
  const char* f = getenv("COOT_JIT_FAIL");
  if (f && *f && strcmp(f, "0") != 0) o.push_back("--definitely-not-an-option");
  return o;
}

uint64_t headers_hash() {
  static uint64_t h = 0;
  if (h) return h;
  uint64_t x = 1469598103934665603ull;
  for (int i = 0; i < k_n_headers; ++i) {
    x = fnv1a(k_headers[i].name, strlen(k_headers[i].name), x);
    x = fnv1a(k_headers[i].text, strlen(k_headers[i].text), x);
  }
  int maj = 0, min = 0;
  nvrtcVersion(&maj, &min);
  x = fnv1a(&maj, sizeof maj, x);
  x = fnv1a(&min, sizeof min, x);
  for (const char* opt : nvrtc_options()) x = fnv1a(opt, strlen(opt), x);
  h = x ? x : 1;
  return h;
}

coot_status nvrtc_compile(const std::string& source, std::vector<char>* cubin, std::string* log) {
  std::vector<const char*> names, texts;
  for (int i = 0; i < k_n_headers; ++i) {
    names.push_back(k_headers[i].name);
    texts.push_back(k_headers[i].text);
  }
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, source.c_str(), "coot_tree.cu", (int)names.size(), texts.data(),
                                     names.data());
  if (r != NVRTC_SUCCESS) return set_error(COOT_ERR_JIT, "nvrtcCreateProgram: %s", nvrtcGetErrorString(r));
  std::vector<const char*> opts = nvrtc_options();
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t lsz = 0;
  nvrtcGetProgramLogSize(prog, &lsz);
  std::string lg(lsz, '\0');
  if (lsz) nvrtcGetProgramLog(prog, &lg[0]);
  if (log) *log = lg;
  if (r != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    return set_error(COOT_ERR_JIT, "NVRTC compile failed (%s): %.1500s", nvrtcGetErrorString(r), lg.c_str());
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  cubin->resize(n);
  nvrtcGetCUBIN(prog, cubin->data());
  nvrtcDestroyProgram(&prog);
  return COOT_OK;
}

// ---- disk cache -------------------------------------------------------------
static const char kMagic[8] = {'C', 'O', 'O', 'T', 'C', 'B', '0', '1'};

static std::string cache_path(const std::string& dir, uint64_t key) {
  char name[64];
  snprintf(name, sizeof name, "/%016llx.cubin", (unsigned long long)key);
  return dir + name;
}

static void mkdirs(const std::string& dir) {
  std::string cur;
  for (size_t i = 0; i < dir.size(); ++i) {
    cur.push_back(dir[i]);
    if (dir[i] == '/' && cur.size() > 1) mkdir(cur.c_str(), 0755);
  }
  mkdir(dir.c_str(), 0755);
}

// entry = magic | u64 sig hash | u64 payload size | u64 payload fnv | payload
static bool disk_load(const std::string& path, uint64_t sig_hash, std::vector<char>* cubin) {
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return false;
  char mg[8];
  uint64_t hdr[3];
  bool ok = fread(mg, 1, 8, f) == 8 && memcmp(mg, kMagic, 8) == 0 && fread(hdr, sizeof(uint64_t), 3, f) == 3 &&
            hdr[0] == sig_hash && hdr[1] > 0 && hdr[1] < (1ull << 30);
  if (ok) {
    cubin->resize(hdr[1]);
    ok = fread(cubin->data(), 1, hdr[1], f) == hdr[1] && fnv1a(cubin->data(), hdr[1]) == hdr[2];
  }
  fclose(f);
  return ok;
}

static void disk_store(const std::string& dir, const std::string& path, uint64_t sig_hash,
                       const std::vector<char>& cubin) {
  mkdirs(dir);
  std::string tmp = path + ".tmp." + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  uint64_t hdr[3] = {sig_hash, (uint64_t)cubin.size(), fnv1a(cubin.data(), cubin.size())};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(uint64_t), 3, f) == 3 &&
            fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size();
  ok = (fclose(f) == 0) && ok;
  if (ok)
    rename(tmp.c_str(), path.c_str());  // atomic publish
  else
    unlink(tmp.c_str());
}

}  // namespace cg

// Get (compile / load) the module of a program; called with ctx->mu held.
coot_status coot_get_module(coot_ctx* ctx, const cg::Program& pg, cg::Module** out) {
  auto it = ctx->mods.find(pg.signature);
  if (it != ctx->mods.end()) {
    *out = it->second.get();
    return COOT_OK;
  }
  NvtxRange nvtx_range("cootgb jit (disk cache or NVRTC)");
  const uint64_t sig_hash = cg::fnv1a(pg.signature.data(), pg.signature.size(), cg::headers_hash());
  std::vector<char> cubin;
  bool from_disk = false;
  const bool use_disk = !(ctx->flags & COOT_CTX_NO_DISK_CACHE) && !ctx->cache_dir.empty();
  std::string path = use_disk ? cg::cache_path(ctx->cache_dir, sig_hash) : std::string();
  if (use_disk) from_disk = cg::disk_load(path, sig_hash, &cubin);
  if (!from_disk) {
    std::string log;
    coot_status s = cg::nvrtc_compile(pg.source, &cubin, &log);
    if (s) return s;
    if (use_disk) cg::disk_store(ctx->cache_dir, path, sig_hash, cubin);
  }
  std::unique_ptr<cg::Module> m(new cg::Module());
  m->cubin_bytes = cubin.size();
  cudaError_t e = cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(COOT_ERR_JIT, "cudaLibraryLoadData: %s", cudaGetErrorString(e));
  }
  for (const cg::KernelSpec& k : pg.kernels) {
    cudaKernel_t kh;
    e = cudaLibraryGetKernel(&kh, m->lib, k.name.c_str());
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(COOT_ERR_JIT, "cudaLibraryGetKernel(%s): %s", k.name.c_str(), cudaGetErrorString(e));
    }
    m->kernels[k.name] = kh;
    cudaFuncAttributes fa;
    memset(&fa, 0, sizeof fa);
    if (cudaFuncGetAttributes(&fa, (const void*)kh) != cudaSuccess) cudaGetLastError();
    m->attrs[k.name] = fa;
  }
  if (log_enabled(ctx))
    fprintf(stderr, "[cootgb] %s kernels (%zu B cubin) for %s\n", from_disk ? "loaded" : "compiled", cubin.size(),
            pg.signature.c_str());
  *out = m.get();
  ctx->mods[pg.signature] = std::move(m);
  return COOT_OK;
}
