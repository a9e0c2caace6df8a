// Nearest-centroid search shared by the Lloyd and objective kernels.
//
// Search: expanded form ||c||^2 - 2 x.c in FP32 (the ||x||^2 term is the same
// for every centroid of a row), packed FMA over pairs of dimensions, top-2
// per row kept in registers, centroids broadcast from shared memory.
//
// Exactness: |computed - true| <= E = (D + 4) u (||x|| + max||c||)^2 for
// every centroid (u = 2^-24, D the padded dimension), so a row whose top-2
// margin exceeds 2E has the true nearest centroid.  Rows at or under it are
// rescored by the whole warp: FP32 direct form against every centroid, with
// its relative bound (D + 3) u; rows still unresolved go to FP64 direct form
// in the same rounding as the double-precision reference, ties to the
// lowest index (Eq. 1; "assign each x to the nearest centroid",
// Algorithm 1).
#pragma once

#include "common.cuh"

#define HPC_U32 5.9604644775390625e-08f  // 2^-24

// Centroid block in shared memory: c[k][D] (zero padded beyond d) and
// cn[k] = ||c_j||^2, +inf for degenerate centroids so they never win.
struct hpc_cent_smem {
  float *c;
  float *cn;
  float cmax;  // max ||c_j|| over live centroids
  int live;    // number of live centroids
};

// Loads C (k x d, global) into shared memory; all threads participate.
template <int D>
__device__ void hpc_load_centroids(hpc_cent_smem &cs, const float *__restrict__ C,
                                   const uint8_t *__restrict__ deg, int k, int d,
                                   float *s_red /* >= 2 floats */) {
  for (int e = threadIdx.x; e < k * D; e += blockDim.x) {
    const int j = e / D, t = e - j * D;
    cs.c[e] = t < d ? C[(int64_t)j * d + t] : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_red[0] = 0.0f;
    s_red[1] = 0.0f;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const bool dead = deg != nullptr && deg[j] != 0;
    float nn = 0.0f;
#pragma unroll 8
    for (int t = 0; t < D; ++t) nn = fmaf(cs.c[j * D + t], cs.c[j * D + t], nn);
    cs.cn[j] = dead ? __int_as_float(0x7f800000) : nn;
    if (!dead) {
      atomicMax(reinterpret_cast<unsigned *>(&s_red[0]), __float_as_uint(nn));
      atomicAdd(reinterpret_cast<unsigned *>(&s_red[1]), 1u);
    }
  }
  __syncthreads();
  cs.cmax = sqrtf(s_red[0]);
  cs.live = (int)__float_as_uint(s_red[1]);
  __syncthreads();
}

// Top-2 search of R register rows over all centroids.
template <int D, int R>
__device__ __forceinline__ void hpc_top2(const float (&x)[R][D], const hpc_cent_smem &cs, int k,
                                         float (&d1)[R], int (&j1)[R], float (&d2)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    d1[r] = __int_as_float(0x7f800000);
    d2[r] = d1[r];
    j1[r] = -1;
  }
#pragma unroll 1
  for (int j = 0; j < k; ++j) {
    const float *cj = cs.c + j * D;
    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = make_float2(0.0f, 0.0f);
    if constexpr (D == 2) {
      const float2 cv = *reinterpret_cast<const float2 *>(cj);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = hpc_fma2(make_float2(x[r][0], x[r][1]), cv, acc[r]);
    } else {
#pragma unroll
      for (int t = 0; t < D; t += 4) {
        const float4 cv = *reinterpret_cast<const float4 *>(cj + t);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          acc[r] = hpc_fma2(make_float2(x[r][t], x[r][t + 1]), make_float2(cv.x, cv.y), acc[r]);
          acc[r] = hpc_fma2(make_float2(x[r][t + 2], x[r][t + 3]), make_float2(cv.z, cv.w), acc[r]);
        }
      }
    }
    const float cnj = cs.cn[j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float v = fmaf(-2.0f, acc[r].x + acc[r].y, cnj);
      d2[r] = fminf(d2[r], fmaxf(d1[r], v));
      j1[r] = v < d1[r] ? j : j1[r];
      d1[r] = fminf(d1[r], v);
    }
  }
}

// Lexicographic (value, index) minimum merge of two top-2 records.
__device__ __forceinline__ void hpc_merge_top2(float &a1, int &ja, float &a2, float b1, int jb,
                                               float b2) {
  if (b1 < a1 || (b1 == a1 && jb < ja)) {
    a2 = fminf(a1, b2);
    a1 = b1;
    ja = jb;
  } else {
    a2 = fminf(a2, b1);
  }
}

// Warp-cooperative exact assignment of one row (every lane calls it with
// the same row pointer).  Returns the label; lanes split the centroids.
template <int D>
__device__ __noinline__ int hpc_rescore_row(const float *__restrict__ xrow, int d,
                                            const hpc_cent_smem &cs, int k) {
  const int lane = threadIdx.x & 31;
  float x[D];
  hpc_load_row<D>(x, xrow, d);
  // Phase 1: FP32 direct form, relative error <= (D + 3) u of each value.
  float a1 = __int_as_float(0x7f800000), a2 = a1;
  int ja = 0x7fffffff;
  for (int j = lane; j < k; j += 32) {
    if (isinf(cs.cn[j])) continue;
    const float v = hpc_dist32_seq<D>(x, cs.c + j * D);
    if (v < a1) {
      a2 = a1;
      a1 = v;
      ja = j;
    } else {
      a2 = fminf(a2, v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
    const int jb = __shfl_xor_sync(0xffffffffu, ja, o);
    const float b2 = __shfl_xor_sync(0xffffffffu, a2, o);
    hpc_merge_top2(a1, ja, a2, b1, jb, b2);
  }
  const float bound = (float)(D + 3) * HPC_U32 * 1.001f * (a1 + a2);
  if (a2 - a1 > bound) return ja;
  // Phase 2: double precision, same operation order as the reference.
  double b = __longlong_as_double(0x7ff0000000000000ll);
  int jb = 0x7fffffff;
  for (int j = lane; j < k; j += 32) {
    if (isinf(cs.cn[j])) continue;
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
      const double diff = __dsub_rn((double)x[t], (double)cs.c[j * D + t]);
      acc = __dadd_rn(acc, __dmul_rn(diff, diff));
    }
    if (acc < b) {
      b = acc;
      jb = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, b, o);
    const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
    if (ob < b || (ob == b && oj < jb)) {
      b = ob;
      jb = oj;
    }
  }
  return jb;
}

// Assigns the R rows of this thread in row group `base` (rows
// base + r * THREADS + tid).  Every thread of the block must call it with
// the same base.  Returns the FP32 sum of the exact-form distances of the
// thread's valid rows; valid[r] / lab[r] / xr[r] describe each row.
template <int D, int R, int THREADS>
__device__ __forceinline__ float hpc_assign_group(const float *__restrict__ X, int64_t n, int d,
                                                  int64_t base, const hpc_cent_smem &cs, int k,
                                                  float (&x)[R][D], int (&lab)[R],
                                                  bool (&valid)[R], int *status) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = base + (int64_t)r * THREADS + tid;
    valid[r] = i < n;
    if (valid[r]) {
      hpc_load_row<D>(x[r], X + i * d, d);
    } else {
#pragma unroll
      for (int t = 0; t < D; ++t) x[r][t] = 0.0f;
    }
  }
  float d1[R], d2[R];
  hpc_top2<D, R>(x, cs, k, d1, lab, d2);
  // margin test
  bool flag[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float nx = 0.0f;
#pragma unroll
    for (int t = 0; t < D; ++t) nx = fmaf(x[r][t], x[r][t], nx);
    const float rad = sqrtf(nx) * 1.00001f + cs.cmax * 1.00001f;
    const float E = (float)(D + 4) * HPC_U32 * rad * rad;
    flag[r] = valid[r] && lab[r] >= 0 && !(d2[r] - d1[r] > 2.001f * E);
  }
  // warp-cooperative rescoring of flagged rows
#pragma unroll
  for (int r = 0; r < R; ++r) {
    unsigned m = __ballot_sync(0xffffffffu, flag[r]);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int64_t i = base + (int64_t)r * THREADS + (tid & ~31) + src;
      const int j = hpc_rescore_row<D>(X + i * d, d, cs, k);
      if ((tid & 31) == src) lab[r] = j;
    }
  }
  float fsum = 0.0f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!valid[r]) continue;
    if (lab[r] < 0) {  // NaN/inf row: no finite distance to any centroid
      hpc_status_set(status, HPC_ERR_NONFINITE);
      valid[r] = false;
      lab[r] = 0;
      continue;
    }
    const float dd = hpc_dist_direct<D>(x[r], cs.c + lab[r] * D);
    if (!isfinite(dd)) hpc_status_set(status, HPC_ERR_NONFINITE);
    fsum += dd;
  }
  return fsum;
}
