// probe.cu -- arithmetic and memory rates of the device, measured with small
// hand-written kernels timed by CUDA events (coot_probe_device).
//
// The rates are the denominators of the rooflines that are not HBM-bound:
// FP64 trees on a part whose FP64 pipe is a small fraction of its FP32 pipe
// (Sec. 4, first difference: GPUs are much faster in 32-bit than in 64-bit
// floating point), and the FP32 ALU bound of the float-float reductions.
//
// Arithmetic kernels: every thread runs 8 independent dependency chains of
// one operation on values held in registers, so the pipe, not latency, bounds
// the rate; the grid fills every SM at the kernel's occupancy.  The operands
// come from kernel arguments, so nothing folds at compile time, and a thread
// stores its chains only if their sum equals an argument that never matches,
// so nothing is dead code.  The exp kernels follow each exp with one fused
// multiply-add that keeps the argument inside [-1, 1] (reported as
// exp+FMA steps per second).  The memory kernels read (and copy) 16-byte
// vectors over buffers several times larger than L2, grid-stride; the same
// read and a write over 256 MiB of pinned host memory give the host link's
// rates as a kernel sees them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "coot.h"

coot_status set_error(coot_status s, const char* fmt, ...);
coot_status cuda_error(cudaError_t e, const char* what);

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

enum Op { OP_ADD = 0, OP_FMA = 1, OP_DIV = 2, OP_EXP = 3 };

template <class T> __device__ __forceinline__ T step(T x, T b, T m, Op op);
template <> __device__ __forceinline__ float step<float>(float x, float b, float m, Op op) {
  switch (op) {
    case OP_ADD: return __fadd_rn(x, b);
    case OP_FMA: return __fmaf_rn(x, m, b);
    case OP_DIV: return __fdiv_rn(b, x);  // x, b/x, x, ...: stays in range
    default: return __fmaf_rn(expf(x), m, b);
  }
}
template <> __device__ __forceinline__ double step<double>(double x, double b, double m, Op op) {
  switch (op) {
    case OP_ADD: return __dadd_rn(x, b);
    case OP_FMA: return __fma_rn(x, m, b);
    case OP_DIV: return __ddiv_rn(b, x);
    default: return __fma_rn(exp(x), m, b);
  }
}

template <class T, Op OP>
__global__ void __launch_bounds__(kBlock) probe_alu(T b, T m, T never, long long iters, T* sink) {
  T x[kChains];
  const T base = (T)(threadIdx.x & 63) * (T)(1.0 / 128.0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)0.25 + base + (T)c * (T)(1.0 / 64.0);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = step<T>(x[c], b, m, OP);
  }
  T s = x[0];
#pragma unroll
  for (int c = 1; c < kChains; ++c) s += x[c];
  if (s == never) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) probe_read(const float4* p, long long n4, float never, float* sink) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // four independent loads in flight per thread
  for (; i + 3 * stride < n4; i += 4 * stride) {
    float4 v0 = __ldg(p + i), v1 = __ldg(p + i + stride), v2 = __ldg(p + i + 2 * stride),
           v3 = __ldg(p + i + 3 * stride);
    acc.x += v0.x + v1.x + v2.x + v3.x;
    acc.y += v0.y + v1.y + v2.y + v3.y;
    acc.z += v0.z + v1.z + v2.z + v3.z;
    acc.w += v0.w + v1.w + v2.w + v3.w;
  }
  for (; i < n4; i += stride) {
    float4 v = __ldg(p + i);
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
  }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == never) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) probe_fill(float4* dst, long long n4, float v) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    dst[i] = make_float4(v, v, v, v);
}

__global__ void __launch_bounds__(kBlock) probe_copy(const float4* src, float4* dst, long long n4) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    float4 v0 = __ldg(src + i), v1 = __ldg(src + i + stride), v2 = __ldg(src + i + 2 * stride),
           v3 = __ldg(src + i + 3 * stride);
    dst[i] = v0;
    dst[i + stride] = v1;
    dst[i + 2 * stride] = v2;
    dst[i + 3 * stride] = v3;
  }
  for (; i < n4; i += stride) dst[i] = __ldg(src + i);
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&a);
    return e != cudaSuccess ? e : cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// best of `reps` timed launches (ms) of fn, after one untimed launch
template <class F> cudaError_t best_ms(Timer& t, int reps, F fn, float* out) {
  fn();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(t.a, 0);
    fn();
    cudaEventRecord(t.b, 0);
    if ((e = cudaEventSynchronize(t.b)) != cudaSuccess) return e;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    best = std::min(best, ms);
  }
  *out = best;
  return cudaGetLastError();
}

template <class T, Op OP>
cudaError_t alu_rate(Timer& t, int sms, long long iters, T b, T m, void* sink, double* rate) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_alu<T, OP>, kBlock, 0);
  if (e != cudaSuccess) return e;
  const int grid = sms * std::max(occ, 1);
  float ms = 0.f;
  e = best_ms(t, 3, [&] { probe_alu<T, OP><<<grid, kBlock>>>(b, m, (T)-12345.0, iters, (T*)sink); }, &ms);
  if (e != cudaSuccess) return e;
  *rate = (double)grid * kBlock * kChains * (double)iters / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

extern "C" coot_status coot_probe_device(int device, coot_probe_result* r) {
  if (!r) return set_error(COOT_ERR_INVALID, "result is NULL");
  memset(r, 0, sizeof *r);
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_error(e, "cudaSetDevice");
  int sms = 0, l2 = 0, clk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
  r->sms = sms;
  r->l2_bytes = l2;
  r->sm_clock_khz = clk;
  // memory: a read buffer of 8x the L2 (at least 1 GiB), copied half to half
  const size_t bytes = std::max<size_t>((size_t)1 << 30, ((size_t)l2 * 8 + 4095) & ~(size_t)4095);
  void* buf = nullptr;
  void* sink = nullptr;
  void* hbuf = nullptr;
  Timer t;
  coot_status st = COOT_OK;
  do {
    if ((e = t.init()) != cudaSuccess) { st = cuda_error(e, "cudaEventCreate"); break; }
    if ((e = cudaMalloc(&sink, (size_t)sms * 64 * kBlock * sizeof(double))) != cudaSuccess) {
      st = cuda_error(e, "cudaMalloc (probe sink)");
      break;
    }
    if ((e = alu_rate<float, OP_ADD>(t, sms, 1 << 16, 0.5f, 0.f, sink, &r->f32_add)) != cudaSuccess ||
        (e = alu_rate<float, OP_FMA>(t, sms, 1 << 16, 0.25f, 0.5f, sink, &r->f32_fma)) != cudaSuccess ||
        (e = alu_rate<float, OP_DIV>(t, sms, 1 << 12, 0.75f, 0.f, sink, &r->f32_div)) != cudaSuccess ||
        (e = alu_rate<float, OP_EXP>(t, sms, 1 << 12, -1.0f, 0.5f, sink, &r->f32_exp)) != cudaSuccess ||
        (e = alu_rate<double, OP_ADD>(t, sms, 1 << 11, 0.5, 0.0, sink, &r->f64_add)) != cudaSuccess ||
        (e = alu_rate<double, OP_FMA>(t, sms, 1 << 11, 0.25, 0.5, sink, &r->f64_fma)) != cudaSuccess ||
        (e = alu_rate<double, OP_DIV>(t, sms, 1 << 8, 0.75, 0.0, sink, &r->f64_div)) != cudaSuccess ||
        (e = alu_rate<double, OP_EXP>(t, sms, 1 << 7, -1.0, 0.5, sink, &r->f64_exp)) != cudaSuccess) {
      st = cuda_error(e, "arithmetic probe");
      break;
    }
    if ((e = cudaMalloc(&buf, bytes)) != cudaSuccess) { st = cuda_error(e, "cudaMalloc (probe buffer)"); break; }
    if ((e = cudaMemset(buf, 0, bytes)) != cudaSuccess) { st = cuda_error(e, "cudaMemset"); break; }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_read, kBlock, 0);
    const int grid = sms * std::max(occ, 1);
    const long long n4 = (long long)(bytes / 16);
    float ms = 0.f;
    if ((e = best_ms(t, 5, [&] { probe_read<<<grid, kBlock>>>((const float4*)buf, n4, -1.f, (float*)sink); },
                     &ms)) != cudaSuccess) {
      st = cuda_error(e, "read probe");
      break;
    }
    r->read_gbs = (double)bytes / (ms * 1e-3) / 1e9;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_copy, kBlock, 0);
    const int gridc = sms * std::max(occ, 1);
    const long long h4 = n4 / 2;
    if ((e = best_ms(t, 5, [&] { probe_copy<<<gridc, kBlock>>>((const float4*)buf, (float4*)buf + h4, h4); },
                     &ms)) != cudaSuccess) {
      st = cuda_error(e, "copy probe");
      break;
    }
    r->copy_gbs = (double)(2 * h4 * 16) / (ms * 1e-3) / 1e9;
    r->buffer_bytes = (int64_t)bytes;
    // the host link: kernels reading and writing pinned host memory (device
    // addresses of host memory under unified addressing)
    const size_t hbytes = (size_t)256 << 20;
    if ((e = cudaHostAlloc(&hbuf, hbytes, cudaHostAllocMapped)) != cudaSuccess) {
      st = cuda_error(e, "cudaHostAlloc (probe)");
      break;
    }
    void* hdev = nullptr;
    if ((e = cudaHostGetDevicePointer(&hdev, hbuf, 0)) != cudaSuccess) {
      st = cuda_error(e, "cudaHostGetDevicePointer");
      break;
    }
    memset(hbuf, 0, hbytes);
    const long long hn4 = (long long)(hbytes / 16);
    if ((e = best_ms(t, 3, [&] { probe_read<<<grid, kBlock>>>((const float4*)hdev, hn4, -1.f, (float*)sink); },
                     &ms)) != cudaSuccess) {
      st = cuda_error(e, "host read probe");
      break;
    }
    r->host_read_gbs = (double)hbytes / (ms * 1e-3) / 1e9;
    if ((e = best_ms(t, 3, [&] { probe_fill<<<gridc, kBlock>>>((float4*)hdev, hn4, 1.f); }, &ms)) != cudaSuccess) {
      st = cuda_error(e, "host write probe");
      break;
    }
    r->host_write_gbs = (double)hbytes / (ms * 1e-3) / 1e9;
  } while (0);
  if (hbuf) cudaFreeHost(hbuf);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  return st;
}
