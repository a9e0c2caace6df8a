// Row arithmetic shared by the TF32 tensor-core searches: warp-uniform
// bounded waits, and the exact FP32 quantities of one row (its squared norm,
// its direct-form distance to a centroid) taken either from registers
// (d <= 32: the row is loaded once) or from global memory / L2 (larger d).
#pragma once

#include "assign.cuh"
#include "tc.cuh"

namespace {

__host__ __device__ constexpr bool hpc_row_in_regs(int D) { return D <= 32; }

// All lanes wait; the warp gives up together if any lane gives up.
__device__ __forceinline__ bool wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort,
                                          int *status, uint64_t limit) {
  const bool ok = hpc_mbar_wait(bar, parity, abort, status, limit);
  return __all_sync(0xffffffffu, ok);
}

// ---- exact row arithmetic from registers (D <= 32) or from L2 (D > 32) ----
template <int D>
struct RowRef {
  float x[hpc_row_in_regs(D) ? D : 1];
  const float *g;
};

template <int D>
__device__ __forceinline__ void row_chunk(const RowRef<D> &r, int t0, float (&v)[16]) {
  if constexpr (hpc_row_in_regs(D)) {
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = r.x[(t0 + t) % D];
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 q = __ldg(reinterpret_cast<const float4 *>(r.g + t0) + c);
      v[4 * c] = q.x;
      v[4 * c + 1] = q.y;
      v[4 * c + 2] = q.z;
      v[4 * c + 3] = q.w;
    }
  }
}

// ||x||^2
template <int D>
__device__ __forceinline__ float row_norm2(const RowRef<D> &r) {
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int t0 = 0; t0 < D; t0 += 16) {
    float v[16];
    row_chunk<D>(r, t0, v);
#pragma unroll
    for (int t = 0; t < 16; t += 2)
      s = hpc_fma2(make_float2(v[t], v[t + 1]), make_float2(v[t], v[t + 1]), s);
  }
  return s.x + s.y;
}

// direct form with two interleaved partial sums (the objective's distance)
template <int D>
__device__ __forceinline__ float row_direct(const RowRef<D> &r, const float *cm) {
  if constexpr (hpc_row_in_regs(D)) {
    return hpc_dist_direct_cm<D>(r.x, cm);
  } else {
    float2 acc = make_float2(0.0f, 0.0f);
    const float2 half = make_float2(0.5f, 0.5f);
#pragma unroll
    for (int t0 = 0; t0 < D; t0 += 16) {
      float v[16];
      row_chunk<D>(r, t0, v);
#pragma unroll
      for (int t = 0; t < 16; t += 2) {
        const float2 e =
            hpc_fma2(half, make_float2(cm[t0 + t], cm[t0 + t + 1]), make_float2(v[t], v[t + 1]));
        acc = hpc_fma2(e, e, acc);
      }
    }
    return acc.x + acc.y;
  }
}

// sequential direct form (relative error <= (D + 2) u)
template <int D>
__device__ __forceinline__ float row_dist32(const RowRef<D> &r, const float *cm) {
  if constexpr (hpc_row_in_regs(D)) {
    return hpc_dist32_cm<D>(r.x, cm);
  } else {
    float acc = 0.0f;
#pragma unroll
    for (int t0 = 0; t0 < D; t0 += 16) {
      float v[16];
      row_chunk<D>(r, t0, v);
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const float diff = __fmaf_rn(0.5f, cm[t0 + t], v[t]);
        acc = __fmaf_rn(diff, diff, acc);
      }
    }
    return acc;
  }
}

// ||x||^2 and the FP32 direct-form distance to centroid j1 of every row of
// a warp (rows row0 .. row0 + 31, lane l's row is row0 + l), each row read by
// the whole warp with coalesced loads: lane l takes dimensions
// [l D / 32, (l + 1) D / 32), then a butterfly sum.  Relative error of the
// distance: (D / 32 + 6) u, within the (D + 3) u the callers assume.
template <int D>
__device__ __forceinline__ void warp_norm_direct(const float *__restrict__ X, int64_t row0,
                                                 bool valid, int j1, const hpc_cent_smem &cs,
                                                 float &nx, float &dd) {
  constexpr int PER = D / 32;
  constexpr int CS = hpc_cstride(D);
  const int lane = threadIdx.x & 31;
  nx = 0.0f;
  dd = 0.0f;
#pragma unroll 4
  for (int src = 0; src < 32; ++src) {
    const int js = __shfl_sync(0xffffffffu, j1, src);
    const bool vs = __shfl_sync(0xffffffffu, (int)valid, src) != 0;
    float px = 0.0f, pd = 0.0f;
    if (vs) {
      const float *xr = X + (row0 + src) * D + lane * PER;
      const float *cm = cs.cm + js * CS + lane * PER;
      float xv[PER];
      if constexpr (PER == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(xr));
        xv[0] = q.x;
        xv[1] = q.y;
        xv[2] = q.z;
        xv[3] = q.w;
      } else {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(xr));
        xv[0] = q.x;
        xv[1] = q.y;
      }
#pragma unroll
      for (int t = 0; t < PER; ++t) {
        const float diff = __fmaf_rn(0.5f, cm[t], xv[t]);
        pd = __fmaf_rn(diff, diff, pd);
        px = __fmaf_rn(xv[t], xv[t], px);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      px += __shfl_xor_sync(0xffffffffu, px, o);
      pd += __shfl_xor_sync(0xffffffffu, pd, o);
    }
    if (lane == src) {
      nx = px;
      dd = pd;
    }
  }
}


}  // namespace
