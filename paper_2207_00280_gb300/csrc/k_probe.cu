// k_probe.cu -- throughput probes of the FP64 and FP32 arithmetic units
// (include/iga_probe.h).  The integration kernels of the FP64 forms are bound by
// GB300's FP64 issue rate; these kernels measure that rate on the device the
// library runs on, so that the roofline of those kernels rests on a
// measurement rather than on a unit count.
//
// Each probe keeps independent dependency chains in flight per thread (DFMA,
// FFMA) or per warp (DMMA) so that latency is hidden and only the pipe's issue
// rate limits the kernel.  The chains converge to a fixed point (a = b a + c
// with 0 < b < 1), or grow slowly (the MMA accumulators), so no value overflows.
#include <cuda_runtime.h>

#include "iga.h"
#include "iga_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kMmaChains = 4;   // independent MMA accumulators per warp

// Written only if a chain reaches a value it cannot reach (negative).
__device__ double g_probe_sink;

__global__ void __launch_bounds__(kThreads) k_probe_dfma(int64_t iters) {
  const double b = 0.999999 - 1e-9 * (threadIdx.x & 7);
  const double c = 1e-7 * (1 + (threadIdx.x & 3));
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3 * (i + 1) + 1e-6 * threadIdx.x;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s < 0.0) g_probe_sink = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma(int64_t iters) {
  const float b = 0.9999f - 1e-6f * (threadIdx.x & 7);
  const float c = 1e-5f * (1 + (threadIdx.x & 3));
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3f * (i + 1) + 1e-5f * (threadIdx.x & 31);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s < 0.f) g_probe_sink = s;
}

// One m8n8k4 FP64 MMA per instruction: A 8x4 (one double per thread), B 4x8
// (one double per thread), C/D 8x8 (two doubles per thread).
__global__ void __launch_bounds__(kThreads) k_probe_dmma(int64_t iters) {
  const double a = 1e-4 * (1 + (threadIdx.x & 7));
  const double bb = 1e-4 * (1 + (threadIdx.x & 3));
  double d[kMmaChains][2];
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i) d[i][0] = d[i][1] = 0.0;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kMmaChains; ++i)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
          : "+d"(d[i][0]), "+d"(d[i][1])
          : "d"(a), "d"(bb));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kMmaChains; ++i) s += d[i][0] + d[i][1];
  if (s < 0.0) g_probe_sink = s;
}

}  // namespace

extern "C" int iga_probe_rate(int kind, int64_t iters, int ctas_per_sm, double* ms_out,
                              double* flops_out, void* cuda_stream) {
  if (!ms_out || !flops_out || iters < 1 || ctas_per_sm < 1 || ctas_per_sm > 8 ||
      kind < IGA_PROBE_DFMA || kind > IGA_PROBE_FFMA)
    return IGA_ERR_ARG;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IGA_ERR_CUDA;
  const int grid = n_sm * ctas_per_sm;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return IGA_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return IGA_ERR_CUDA;
  }
  cudaError_t e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    if (kind == IGA_PROBE_DFMA) k_probe_dfma<<<grid, kThreads, 0, st>>>(iters);
    else if (kind == IGA_PROBE_FFMA) k_probe_ffma<<<grid, kThreads, 0, st>>>(iters);
    else k_probe_dmma<<<grid, kThreads, 0, st>>>(iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return IGA_ERR_CUDA;
  const double threads = (double)grid * kThreads;
  if (kind == IGA_PROBE_DMMA)
    *flops_out = threads / 32.0 * kMmaChains * (double)iters * 512.0;
  else
    *flops_out = threads * kChains * (double)iters * 2.0;
  *ms_out = ms;
  return IGA_OK;
}
