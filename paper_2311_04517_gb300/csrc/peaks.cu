// Throughput probes for the rooflines of the CUDA-core kernels: the rates
// the FP32 / FP64 / ALU pipes and the L2 and HBM read paths reach on this
// GPU, measured with CUDA events.  The hot-path kernels are compared against
// these (the tensor-core and HBM-copy peaks come from separate
// measurements).  Each arithmetic probe runs 8 independent dependency
// chains per thread on a grid of 8 blocks of 256 threads per SM, written in
// inline PTX so that the compiler keeps every operation; the result feeds a
// store that never happens (its condition is false for the probe's inputs)
// so no chain is dead code.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hpclust.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma(int iters, float b, float *sink) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %1;" : "+f"(a[i]) : "f"(b));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == -1.0f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma2(int iters, float b, float *sink) {
  unsigned long long a[8];
  float2 b2 = make_float2(b, b);
  const unsigned long long bb = *reinterpret_cast<unsigned long long *>(&b2);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float2 v = make_float2((float)(threadIdx.x + i), (float)(threadIdx.x + i) + 0.5f);
    a[i] = *reinterpret_cast<unsigned long long *>(&v);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(a[i]) : "l"(bb));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 v = *reinterpret_cast<const float2 *>(&a[i]);
    s += v.x + v.y;
  }
  if (s == -1.0f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_dfma(int iters, double b, float *sink) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("fma.rn.f64 %0, %0, %1, %1;" : "+d"(a[i]) : "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == -1.0) sink[threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_fmin(int iters, float b, float *sink) {
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("min.f32 %0, %0, %1;" : "+f"(a[i]) : "f"(b));
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == -1.0f) sink[threadIdx.x] = s;
}

// Reads nv float4 words `reps` times, grid-stride, 16-byte loads that keep
// their L2 lines (a buffer that fits L2 stays there after the first pass).
__global__ void __launch_bounds__(PROBE_THREADS) probe_read(const float4 *p, int64_t nv, int reps,
                                                           float *sink) {
  float s = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * PROBE_THREADS;
  for (int r = 0; r < reps; ++r)
    for (int64_t i = (int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x; i < nv; i += stride) {
      const float4 v = __ldcg(p + i);
      s += v.x + v.y + v.z + v.w;
    }
  if (s == -1.0f) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int hpc_peak_probe(int32_t kind, int32_t device, void *stream, double *rate_out,
                              double *ms_out) {
  if (!rate_out || kind < HPC_PROBE_FFMA || kind > HPC_PROBE_HBM_READ) return HPC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HPC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = sms * PROBE_BLOCKS_PER_SM;
  float *sink = nullptr;
  void *buf = nullptr;
  if (cudaMalloc(&sink, PROBE_THREADS * sizeof(float)) != cudaSuccess) return HPC_ERR_NOMEM;
  // L2: 64 MiB (inside the 129 MB L2), 40 passes; HBM: 4 GiB, one pass
  const int64_t bytes = kind == HPC_PROBE_L2_READ ? (64ll << 20) : (4ll << 30);
  const int reps = kind == HPC_PROBE_L2_READ ? 40 : 1;
  if (kind >= HPC_PROBE_L2_READ) {
    if (cudaMalloc(&buf, (size_t)bytes) != cudaSuccess) {
      cudaFree(sink);
      return HPC_ERR_NOMEM;
    }
    cudaMemsetAsync(buf, 0, (size_t)bytes, st);
  }
  // operations per thread and launch: iters x 16 x 8 chains (x 2 lanes for f32x2)
  const int iters = kind == HPC_PROBE_DFMA ? 64 : 1024;
  auto launch = [&]() {
    switch (kind) {
      case HPC_PROBE_FFMA: probe_ffma<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.999f, sink); break;
      case HPC_PROBE_FFMA2: probe_ffma2<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.999f, sink); break;
      case HPC_PROBE_DFMA: probe_dfma<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.999, sink); break;
      case HPC_PROBE_FMIN: probe_fmin<<<grid, PROBE_THREADS, 0, st>>>(iters, 0.5f, sink); break;
      default:
        probe_read<<<grid, PROBE_THREADS, 0, st>>>(static_cast<const float4 *>(buf), bytes / 16,
                                                   reps, sink);
    }
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();  // warm-up (and, for L2, the pass that brings the buffer in)
  cudaEventRecord(e0, st);
  const int timed = 3;
  for (int t = 0; t < timed; ++t) launch();
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) return HPC_ERR_CUDA;
  ms /= (float)timed;
  const double threads = (double)grid * PROBE_THREADS;
  double work;
  switch (kind) {
    case HPC_PROBE_FFMA2: work = threads * iters * 16.0 * 8.0 * 2.0; break;
    case HPC_PROBE_L2_READ:
    case HPC_PROBE_HBM_READ: work = (double)bytes * reps; break;
    default: work = threads * iters * 16.0 * 8.0;
  }
  *rate_out = work / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return HPC_OK;
}
