// Sampling (Section 3: each worker draws a random sample S of size s from X;
// Algorithms 3-5, first step of the worker loop).  Row i of the sample is
// X[floor(r_i * n / 2^64)], r_i = draw i of stream (seed, worker, round, 0):
// one thread turns one Philox block into four row indices, then the rows are
// gathered with 16-byte accesses where the row width allows it.
#include "common.cuh"
#include "kernels.h"
#include "round.cuh"

namespace {

__global__ void sample_index_kernel(int64_t n, uint64_t seed, uint32_t worker, uint32_t round,
                                    int64_t s, int64_t *__restrict__ idx) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b * 4 >= s) return;
  uint64_t v[4];
  hpc_draw_block(seed, worker, round, HPC_TAG_SAMPLE, (uint64_t)b, v);
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int64_t i = b * 4 + w;
    if (i < s) idx[i] = (int64_t)hpc_scale_word(v[w], (uint64_t)n);
  }
}

// One thread per 16-byte chunk of a sample row (d % 4 == 0).
__global__ void gather4_kernel(const float4 *__restrict__ X, int d4, int64_t s,
                               const int64_t *__restrict__ idx, float4 *__restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s * d4) return;
  const int64_t i = e / d4;
  const int c = (int)(e - i * d4);
  S[e] = __ldg(X + idx[i] * d4 + c);
}

__global__ void gather1_kernel(const float *__restrict__ X, int d, int64_t s,
                               const int64_t *__restrict__ idx, float *__restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= s * d) return;
  const int64_t i = e / d;
  const int t = (int)(e - i * d);
  S[e] = __ldg(X + idx[i] * d + t);
}

// Batched form for one round: blockIdx.y is the worker.  A block draws the
// indices of 1024 consecutive sample rows (256 Philox blocks, one per
// thread) into shared memory, then copies those rows with coalesced loads.
constexpr int SB_THREADS = 256, SB_ROWS = 4 * SB_THREADS;

template <bool VEC4>
__global__ void __launch_bounds__(SB_THREADS) sample_batch_kernel(
    const float *__restrict__ X, int64_t n, int d, uint64_t seed, uint32_t round,
    const uint32_t *round_dev, const hpc_sample_task *__restrict__ tasks, hpc_base_args base) {
  __shared__ int64_t s_idx[SB_ROWS];
  if (base.wk && blockIdx.x == gridDim.x - 1) {  // the extra block: this worker's base
    hpc_base_select_block(base, (int)blockIdx.y);
    return;
  }
  if (round_dev) round = *round_dev;
  const hpc_sample_task t = tasks[blockIdx.y];
  const int64_t r0 = (int64_t)blockIdx.x * SB_ROWS;
  if (r0 >= t.s) return;
  const int rows = (int)min((int64_t)SB_ROWS, t.s - r0);
  {
    uint64_t v[4];
    hpc_draw_block(seed, t.worker, round, HPC_TAG_SAMPLE, (uint64_t)(r0 / 4) + threadIdx.x, v);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int i = threadIdx.x * 4 + w;
      if (i < rows) {
        const int64_t x = (int64_t)hpc_scale_word(v[w], (uint64_t)n);
        s_idx[i] = x;
        if (t.idx) t.idx[r0 + i] = x;
      }
    }
  }
  __syncthreads();
  if (VEC4) {
    // eight independent row loads in flight per thread before their stores
    const int d4 = d >> 2, tot = rows * d4;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    float4 *S4 = reinterpret_cast<float4 *>(t.S) + r0 * d4;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * SB_THREADS) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * SB_THREADS;
        if (e < tot) {
          const int i = e / d4, c = e - i * d4;
          v[u] = __ldg(X4 + s_idx[i] * d4 + c);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * SB_THREADS;
        if (e < tot) S4[e] = v[u];
      }
    }
  } else {
    float *S = t.S + r0 * d;
    for (int e = threadIdx.x; e < rows * d; e += SB_THREADS) {
      const int i = e / d, c = e - i * d;
      S[e] = __ldg(X + s_idx[i] * d + c);
    }
  }
}

}  // namespace

int hpc_sample_batch_launch(const hpc_launch &L, const float *X, int64_t n, int d, uint64_t seed,
                            uint32_t round, const uint32_t *round_dev, int W,
                            const hpc_sample_task *tasks_dev, int64_t smax,
                            const hpc_base_args &base) {
  if (W < 1 || smax < 1) return HPC_OK;
  if (W > 65535) return HPC_ERR_ARG;
  // one extra block per worker selects its base when base.wk is given
  const dim3 grid((unsigned)((smax + SB_ROWS - 1) / SB_ROWS + (base.wk ? 1 : 0)), (unsigned)W);
  if (d % 4 == 0)
    sample_batch_kernel<true><<<grid, SB_THREADS, 0, L.stream>>>(X, n, d, seed, round, round_dev,
                                                                 tasks_dev, base);
  else
    sample_batch_kernel<false><<<grid, SB_THREADS, 0, L.stream>>>(X, n, d, seed, round, round_dev,
                                                                  tasks_dev, base);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

int hpc_sample_launch(const hpc_launch &L, const float *X, int64_t n, int d, uint64_t seed,
                      uint32_t worker, uint32_t round, int64_t s, float *S, int64_t *idx) {
  if (s == 0) return HPC_OK;
  const int T = 256;
  const int64_t blocks_idx = ((s + 3) / 4 + T - 1) / T;
  sample_index_kernel<<<(unsigned)blocks_idx, T, 0, L.stream>>>(n, seed, worker, round, s, idx);
  if (d % 4 == 0) {
    const int64_t tot = s * (d / 4);
    gather4_kernel<<<(unsigned)((tot + T - 1) / T), T, 0, L.stream>>>(
        reinterpret_cast<const float4 *>(X), d / 4, s, idx, reinterpret_cast<float4 *>(S));
  } else {
    const int64_t tot = s * d;
    gather1_kernel<<<(unsigned)((tot + T - 1) / T), T, 0, L.stream>>>(X, d, s, idx, S);
  }
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}
