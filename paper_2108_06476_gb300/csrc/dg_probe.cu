// dg_measure_peaks: the FP64 and FP32 vector FMA throughput of the current
// device, measured by a kernel of independent fused multiply-add chains and
// timed with CUDA events. The roofline of the flux-differencing kernels
// (bound by the FP64 or FP32 pipe, not by memory) divides by these measured
// rates instead of a nominal figure.
#include <cuda_runtime.h>
#include <stdio.h>

#include "dgsem.h"

namespace dg {
int set_last_error(int code, const char* msg);
}

namespace {

constexpr int kChains = 8;

// store targets of the probe kernels (never written in practice)
__device__ double g_probe_sink64[256 * 2048];
__device__ float g_probe_sink32[256 * 2048];

template <typename T>
T* sink_symbol();
template <>
double* sink_symbol<double>() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_probe_sink64) == cudaSuccess ? (double*)p : nullptr;
}
template <>
float* sink_symbol<float>() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_probe_sink32) == cudaSuccess ? (float*)p : nullptr;
}

// kChains independent FMA chains per thread; the result is stored only if it
// takes an impossible value, so the chains stay live without memory traffic
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = T(threadIdx.x) * T(1e-3) + T(j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == T(-12345.0)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int nsm, cudaStream_t st, double* tflops) {
  const int threads = 256, blocks = nsm * 8;
  if (blocks * threads > 256 * 2048)
    return dg::set_last_error(DG_ERR_ARG, "dg_measure_peaks: more SMs than the probe covers");
  T* out = sink_symbol<T>();  // never written (see the kernel); a valid target anyway
  if (!out) return dg::set_last_error(DG_ERR_CUDA, "dg_measure_peaks: symbol lookup failed");
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return dg::set_last_error(DG_ERR_CUDA, "dg_measure_peaks: event creation failed");
  int iters = 1 << 12;
  float ms = 0.0f;
  // grow the work until one launch takes at least 20 ms; the mean of 3
  for (;;) {
    fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(a, st);
    for (int r = 0; r < 3; ++r)
      fma_probe_kernel<T><<<blocks, threads, 0, st>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      return dg::set_last_error(DG_ERR_CUDA, "dg_measure_peaks: probe kernel failed");
    }
    cudaEventElapsedTime(&ms, a, b);
    ms /= 3.0f;
    if (ms >= 20.0f || iters >= (1 << 24)) break;
    iters *= 4;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return DG_OK;
}

}  // namespace

extern "C" int dg_measure_peaks(double* fp64_tflops, double* fp32_tflops, int* sm_count,
                                void* cuda_stream) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return dg::set_last_error(DG_ERR_CUDA, "dg_measure_peaks: device query failed");
  if (sm_count) *sm_count = nsm;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int rc = DG_OK;
  if (fp64_tflops) rc = probe<double>(nsm, st, fp64_tflops);
  if (rc == DG_OK && fp32_tflops) rc = probe<float>(nsm, st, fp32_tflops);
  return rc;
}

// ---- issue cost of one FP64 warp instruction ----
namespace {

__device__ long long g_probe_cycles[2];

// one dependent DFMA chain per thread of `active` lanes (the others leave at
// once); thread 0 of block 0 records the SM cycles of `iters` steps
__global__ void dfma_chain_kernel(int iters, int active, int slot) {
  if ((int)(threadIdx.x & 31) >= active) return;
  double x = 1.0 + 1e-9 * threadIdx.x;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) x = fma(x, 0.9999999, 1e-7);
  const long long t1 = clock64();
  if (blockIdx.x == 0 && threadIdx.x == 0) g_probe_cycles[slot] = x == -1.0 ? 0 : t1 - t0;
}

}  // namespace

extern "C" int dg_measure_fp64_issue(double* cycles_full_warp, double* cycles_one_lane,
                                     void* cuda_stream) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return dg::set_last_error(DG_ERR_CUDA, "dg_measure_fp64_issue: device query failed");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int iters = 4096;
  // one warp per SM: 32 active lanes, then one
  dfma_chain_kernel<<<nsm, 32, 0, st>>>(16, 32, 0);
  dfma_chain_kernel<<<nsm, 32, 0, st>>>(iters, 32, 0);
  dfma_chain_kernel<<<nsm, 32, 0, st>>>(iters, 1, 1);
  long long c[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyFromSymbolAsync(c, g_probe_cycles, sizeof(c), 0, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return dg::set_last_error(DG_ERR_CUDA, "dg_measure_fp64_issue: probe failed");
  if (cycles_full_warp) *cycles_full_warp = (double)c[0] / iters;
  if (cycles_one_lane) *cycles_one_lane = (double)c[1] / iters;
  return DG_OK;
}

// ---- self-check of the device arithmetic helpers ----
#include "dg_f32.cuh"

namespace {

__global__ void arith_kernel(int op, const double* __restrict__ x, double* __restrict__ y,
                             long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r = 0.0;
    switch (op) {
      case 0: r = dg::rcp(v); break;                          // FP64 reciprocal
      case 1: r = (double)dg::rcp((float)v); break;           // FP32 reciprocal
      case 2: r = (double)dg::d2f(v); break;                  // double -> float
      case 3: r = dg::f2d((float)v); break;                   // float -> double
      case 4: r = dg::sqrt_pos(v); break;                     // FP64 square root
      default: r = 0.0;
    }
    y[i] = r;
  }
}

}  // namespace

extern "C" int dg_selftest_arith(int op, const double* x, double* y, long long n,
                                 void* cuda_stream) {
  if (op < 0 || op > 4 || n < 0 || (n > 0 && (!x || !y)))
    return dg::set_last_error(DG_ERR_ARG, "dg_selftest_arith: bad argument");
  if (n == 0) return DG_OK;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  arith_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(op, x, y, n);
  if (cudaGetLastError() != cudaSuccess)
    return dg::set_last_error(DG_ERR_CUDA, "dg_selftest_arith: launch failed");
  return DG_OK;
}
