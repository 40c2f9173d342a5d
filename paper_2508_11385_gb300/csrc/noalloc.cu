// noalloc.cu -- per-row sums of an FP32 matrix without allocating memory.
//
// Some callers cannot allocate device memory while they run: code that has
// handed all of its memory to its own pool or arena, code running inside a
// region where an allocation would synchronise the device or is forbidden
// outright, or a host framework that owns every byte it gives the library.
// For them, coot_sum_rows_f32_noalloc computes sum(X, 1) (or mean(X, 1)) of
// an FP32 matrix with the same per-row reduction kernel as coot_eval, but its
// scratch -- one ticket per block of rows and the column-split partials --
// lives in the fixed array below instead of a workspace that grows on
// demand.  The kernel is compiled into this library (no run-time
// compilation, no module loaded at call time).
//
// The array is COOT_NOALLOC_SCRATCH_BYTES (4 MiB) on every GPU that loads the
// library, held until the process exits.  Every call on a device shares it:
// calls whose work can overlap on the GPU (different streams, or threads
// without ordering) race on it; calls on one stream are ordered and safe.
//
// Its device address is looked up once per device (the first call on it) and
// kept for the life of the process, so the entry point must not be used on a
// device after cudaDeviceReset: the reset unloads the module that holds the
// array and the kept address would no longer be valid.
//
// Test hook: with COOT_NOALLOC_POISON_SCRATCH=1 in the environment, the set-up
// fills the whole array with the byte 0xA5 (a cudaMemset, not an allocation),
// which stands for tickets and partials left behind by an earlier call that
// failed part-way; every later call must still give correct sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "coot.h"
#include "dev/coot_kernels.cuh"

coot_status set_error(coot_status s, const char* fmt, ...);
coot_status cuda_error(cudaError_t e, const char* what);

namespace {

constexpr size_t kScratchBytes = COOT_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTicketBytes = 16384;  // 4096 row blocks
constexpr size_t kFlagBytes = 256;      // device error word
constexpr size_t kPartialOffset = kTicketBytes + kFlagBytes;
constexpr size_t kPartialBytes = kScratchBytes - kPartialOffset;
constexpr int kBlock = 256;

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: the address is obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char coot_noalloc_scratch[kScratchBytes];

extern "C" __global__ void __launch_bounds__(kBlock) coot_noalloc_row_v4(const __grid_constant__ coot::Params p) {
  coot::row_kernel<coot::Leaf<0>, float, 1, 0, coot::RED_SUM, 4, 2, false>(p);
}
extern "C" __global__ void __launch_bounds__(kBlock) coot_noalloc_row_v1(const __grid_constant__ coot::Params p) {
  coot::row_kernel<coot::Leaf<0>, float, 1, 0, coot::RED_SUM, 1, 4, false>(p);
}

std::mutex g_mu;
void* g_scratch[256];  // device address of the scratch, per device ordinal
int g_sms[256];
int g_occ[2][256];

// once per device, with that device current
coot_status setup(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch[dev]) return COOT_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, coot_noalloc_scratch);
  if (e != cudaSuccess || !ptr) return cuda_error(e, "cudaGetSymbolAddress(coot_noalloc_scratch)");
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_error(e, "cudaDeviceGetAttribute");
  int o4 = 0, o1 = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o4, coot_noalloc_row_v4, kBlock, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, coot_noalloc_row_v1, kBlock, 0)) != cudaSuccess)
    return cuda_error(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const char* poison = getenv("COOT_NOALLOC_POISON_SCRATCH");
  if (poison && poison[0] == '1') {
    if ((e = cudaMemset(ptr, 0xA5, kScratchBytes)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess)
      return cuda_error(e, "cudaMemset (poisoned scratch)");
  }
  g_sms[dev] = sms;
  g_occ[0][dev] = std::max(o4, 1);
  g_occ[1][dev] = std::max(o1, 1);
  g_scratch[dev] = ptr;
  return COOT_OK;
}

}  // namespace

extern "C" coot_status coot_sum_rows_f32_noalloc(const coot_mat* x, int32_t mean, float* out, coot_stream stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!x) return set_error(COOT_ERR_INVALID, "x is NULL");
  if (x->dtype != COOT_F32) return set_error(COOT_ERR_DTYPE, "coot_sum_rows_f32_noalloc takes an F32 matrix");
  const int64_t R = x->n_rows, C = x->n_cols;
  if (R < 0 || C < 0) return set_error(COOT_ERR_INVALID, "negative shape");
  // only adjacent rows (element (i,j) at data[i + j*ld]): the kernel reads V
  // consecutive elements per thread
  if (x->rs < 0) return set_error(COOT_ERR_INVALID, "negative row stride %d", (int)x->rs);
  if (x->rs > 1)
    return set_error(COOT_ERR_UNSUPPORTED,
                     "coot_sum_rows_f32_noalloc takes matrices with adjacent rows (rs 0 or 1), not rs = %d; use "
                     "coot_eval with R_SUM dim 1",
                     (int)x->rs);
  const int64_t ld = (C > 1) ? x->ld : std::max<int64_t>(x->ld, R);
  if (C > 1 && ld < R) return set_error(COOT_ERR_INVALID, "ld %lld < n_rows %lld", (long long)ld, (long long)R);
  if (R == 0) return COOT_OK;  // no outputs
  if (!out) return set_error(COOT_ERR_INVALID, "out is NULL");
  if (C > 0 && !x->data) return set_error(COOT_ERR_INVALID, "x->data is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return set_error(COOT_ERR_INVALID, "device ordinal %d", dev);
  // vector loads when every column start is 16-byte aligned
  const bool vec = ((uintptr_t)x->data % 16 == 0) && (C <= 1 || (ld * 4) % 16 == 0);
  const int64_t V = vec ? 4 : 1;
  const int64_t nrb = (R + kBlock * V - 1) / (kBlock * V);
  const int64_t max_rows = (int64_t)(kTicketBytes / sizeof(unsigned)) * kBlock * V;
  if (nrb > (int64_t)(kTicketBytes / sizeof(unsigned)))
    return set_error(COOT_ERR_UNSUPPORTED,
                     "n_rows %lld exceeds the no-allocation limit of %lld rows for this layout (the %zu-byte static "
                     "scratch holds %zu row-block tickets); use coot_eval with R_SUM dim 1",
                     (long long)R, (long long)max_rows, kScratchBytes, kTicketBytes / sizeof(unsigned));
  coot_status s = setup(dev);
  if (s) return s;
  if (C == 0) {  // empty rows: sums 0, means NaN (all-ones bytes)
    e = cudaMemsetAsync(out, mean ? 0xff : 0, (size_t)R * sizeof(float), stream);
    return e == cudaSuccess ? COOT_OK : cuda_error(e, "cudaMemsetAsync");
  }
  // column splits: fill the GPU, but keep the split partials inside the scratch
  const int64_t resident = (int64_t)g_sms[dev] * g_occ[vec ? 0 : 1][dev];
  int64_t nsp = std::max<int64_t>(1, std::min<int64_t>(C, resident / nrb));
  nsp = std::min<int64_t>(nsp, std::max<int64_t>(1, (int64_t)(kPartialBytes / ((size_t)R * 8))));
  const int64_t cps = (C + nsp - 1) / nsp;
  nsp = (C + cps - 1) / cps;
  char* base = (char*)g_scratch[dev];
  // tickets must start at zero: clear the ones this launch uses (a call that
  // failed part-way could have left some behind) and the error word
  if ((e = cudaMemsetAsync(base, 0, (size_t)nrb * sizeof(unsigned), stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + kTicketBytes, 0, sizeof(unsigned), stream)) != cudaSuccess)
    return cuda_error(e, "cudaMemsetAsync (scratch tickets)");
  coot::Params p;
  memset(&p, 0, sizeof p);
  p.src[0] = x->data;
  p.ld[0] = ld;
  p.n_rows = R;
  p.n_cols = C;
  p.n_row_blocks = nrb;
  p.n_splits = nsp;
  p.units_per_col = cps;
  p.count = R * C;
  p.div = mean ? (double)C : 1.0;
  p.red_out = out;
  p.tickets = (unsigned*)base;
  p.err_flag = (unsigned*)(base + kTicketBytes);
  p.partials = base + kPartialOffset;
  void* args[] = {&p};
  e = cudaLaunchKernel(vec ? (const void*)coot_noalloc_row_v4 : (const void*)coot_noalloc_row_v1,
                       dim3((unsigned)(nrb * nsp)), dim3(kBlock), args, 0, stream);
  if (e != cudaSuccess) return cuda_error(e, "coot_sum_rows_f32_noalloc launch");
  return COOT_OK;
}
