// Nearest-centroid search shared by the Lloyd and objective kernels.
//
// Search: expanded form ||c||^2 - 2 x.c in FP32 (the ||x||^2 term is the same
// for every centroid of a row).  Shared memory holds cm = -2c and the pairs
// (||c||^2, 0); each row's dot product runs as two interleaved packed-FMA
// chains (fma.rn.f32x2) seeded with (||c||^2, 0), two centroids per loop
// step for instruction-level parallelism, top-2 kept in registers.  For
// k <= 32 the top-2 runs on (value, index) keys: the index replaces the low
// five mantissa bits, so three float min/max operations update both.
//
// Exactness: with E = (D + 4) u (||x|| + max||c||)^2, u = 2^-24, D the padded
// dimension, every computed value lies within E of the exact one; keys add at
// most 2^(IB-23) |v| (IB = 5 or 7 index bits).  A row whose top-2 margin
// exceeds 2E + 2^(IB-22) (|k1| + |k2|)
// therefore has the true nearest centroid.  Rows at or under it are rescored
// by the whole warp: FP32 direct form against every centroid, with its
// relative bound (D + 3) u, and rows still unresolved in FP64 direct form in
// the same rounding as the double-precision reference, ties to the lowest
// index (Eq. 1; Algorithm 1's assignment step).
#pragma once

#include "common.cuh"

#define HPC_U32 5.9604644775390625e-08f  // 2^-24
#define HPC_DEAD 1.0e38f                 // norm given to degenerate / padding centroids

// Row stride (floats) of the centroid block: rows are padded by 16 bytes so
// that lanes gathering different centroids hit different banks.
__host__ __device__ constexpr int hpc_cstride(int D) { return D >= 4 ? D + 4 : D; }

// Centroid block in shared memory.
struct hpc_cent_smem {
  float *cm;    // kp rows of hpc_cstride(D) floats: -2 c (zero padded beyond d)
  float2 *cnz;  // kp: (||c||^2, 0), HPC_DEAD for degenerate and padding slots
  float cmax;   // max ||c_j|| over live centroids
  int live;     // number of live centroids
  int kp;       // k rounded up to even
};

__host__ __device__ __forceinline__ size_t hpc_cent_smem_bytes(int D, int k) {
  const int kp = (k + 1) & ~1;
  return (size_t)kp * hpc_cstride(D) * 4 + (size_t)kp * 8;
}

__device__ __forceinline__ void hpc_cent_bind(hpc_cent_smem &cs, unsigned char *base, int D, int k) {
  cs.kp = (k + 1) & ~1;
  cs.cm = reinterpret_cast<float *>(base);
  cs.cnz = reinterpret_cast<float2 *>(base + (size_t)cs.kp * hpc_cstride(D) * 4);
}

// Recomputes norms, cmax and the live count from cs.cm (all threads).
// `dead(j)` says whether slot j is degenerate.
template <int D, typename Dead>
__device__ void hpc_cent_finish(hpc_cent_smem &cs, int k, float *s_red, Dead dead) {
  if (threadIdx.x == 0) {
    s_red[0] = 0.0f;
    s_red[1] = 0.0f;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < cs.kp; j += blockDim.x) {
    if (j >= k || dead(j)) {
      cs.cnz[j] = make_float2(HPC_DEAD, 0.0f);
      continue;
    }
    float nn = 0.0f;
#pragma unroll 8
    for (int t = 0; t < D; ++t) {
      const float c = -0.5f * cs.cm[j * hpc_cstride(D) + t];
      nn = fmaf(c, c, nn);
    }
    cs.cnz[j] = make_float2(nn, 0.0f);
    atomicMax(reinterpret_cast<unsigned *>(&s_red[0]), __float_as_uint(nn));
    atomicAdd(reinterpret_cast<unsigned *>(&s_red[1]), 1u);
  }
  __syncthreads();
  cs.cmax = sqrtf(s_red[0]);
  cs.live = (int)__float_as_uint(s_red[1]);
  __syncthreads();
}

// Loads C (k x d, global) into shared memory; all threads participate.
template <int D>
__device__ void hpc_load_centroids(hpc_cent_smem &cs, const float *__restrict__ C,
                                   const uint8_t *__restrict__ deg, int k, int d, float *s_red) {
  constexpr int CS = hpc_cstride(D);
  for (int e = threadIdx.x; e < cs.kp * CS; e += blockDim.x) {
    const int j = e / CS, t = e - j * CS;
    cs.cm[e] = (j < k && t < d) ? -2.0f * C[(int64_t)j * d + t] : 0.0f;
  }
  __syncthreads();
  hpc_cent_finish<D>(cs, k, s_red, [&](int j) { return deg != nullptr && deg[j] != 0; });
}

__device__ __forceinline__ bool hpc_is_dead(const hpc_cent_smem &cs, int j) {
  return cs.cnz[j].x >= HPC_DEAD;
}

// Dot products of R register rows with two consecutive centroids: returns
// v = ||c||^2 - 2 x.c for both.
template <int D, int R>
__device__ __forceinline__ void hpc_pair_values(const float (&x)[R][D], const hpc_cent_smem &cs, int j,
                                                float (&va)[R], float (&vb)[R]) {
  const float *ca = cs.cm + j * hpc_cstride(D);
  const float *cb = ca + hpc_cstride(D);
  const float4 nz = *reinterpret_cast<const float4 *>(cs.cnz + j);  // (n_a, 0, n_b, 0)
  float2 aa[R], ab[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    aa[r] = make_float2(nz.x, nz.y);
    ab[r] = make_float2(nz.z, nz.w);
  }
  if constexpr (D == 2) {
    const float2 pa = *reinterpret_cast<const float2 *>(ca);
    const float2 pb = *reinterpret_cast<const float2 *>(cb);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      aa[r] = hpc_fma2(make_float2(x[r][0], x[r][1]), pa, aa[r]);
      ab[r] = hpc_fma2(make_float2(x[r][0], x[r][1]), pb, ab[r]);
    }
  } else {
#pragma unroll
    for (int t = 0; t < D; t += 4) {
      const float4 pa = *reinterpret_cast<const float4 *>(ca + t);
      const float4 pb = *reinterpret_cast<const float4 *>(cb + t);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 x01 = make_float2(x[r][t], x[r][t + 1]);
        const float2 x23 = make_float2(x[r][t + 2], x[r][t + 3]);
        aa[r] = hpc_fma2(x01, make_float2(pa.x, pa.y), aa[r]);
        ab[r] = hpc_fma2(x01, make_float2(pb.x, pb.y), ab[r]);
        aa[r] = hpc_fma2(x23, make_float2(pa.z, pa.w), aa[r]);
        ab[r] = hpc_fma2(x23, make_float2(pb.z, pb.w), ab[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    va[r] = aa[r].x + aa[r].y;
    vb[r] = ab[r].x + ab[r].y;
  }
}

__device__ __forceinline__ float hpc_min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Folds four (value, index) keys into the running top-2 (d1 <= d2): the
// smallest of the four and the second smallest, then the merge.
__device__ __forceinline__ void hpc_top2_fold4(float &d1, float &d2, float k0, float k1, float k2,
                                               float k3) {
  const float a = fminf(k0, k1), b = fmaxf(k0, k1);
  const float c = fminf(k2, k3), e = fmaxf(k2, k3);
  const float m = fminf(a, c), s = hpc_min3(b, e, fmaxf(a, c));
  d2 = hpc_min3(d2, s, fmaxf(d1, m));
  d1 = fminf(d1, m);
}

// Adds v to the unevaluated FP32 pair hi + lo with an error-free TwoSum
// (Knuth): hi + lo equals the running sum up to the rounding of the lo adds,
// about m 2^-48 of the sum after m nonnegative terms, with no FP64
// instruction (FP64 runs at a small fraction of the FP32 rate on GB300).
__device__ __forceinline__ void hpc_sum2_add(float &hi, float &lo, float v) {
  const float t = hi + v;
  const float bv = t - hi;
  lo += (hi - (t - bv)) + (v - bv);
  hi = t;
}

__device__ __forceinline__ float hpc_key(float v, int j) {
  return __int_as_float((__float_as_int(v) & ~31) | j);
}

// (value, index) key with the index in the low IB mantissa bits: the key is
// within 2^(IB-23) |v| of v.
template <int IB>
__device__ __forceinline__ float hpc_key_b(float v, int j) {
  return __int_as_float((__float_as_int(v) & ~((1 << IB) - 1)) | j);
}

// Top-2 search of R register rows over all centroids.  IB > 0 (k <= 2^IB):
// d1/d2 are (value, index) keys with the index in the low IB bits, and j1
// is read from d1's low bits; IB = 0: values and a tracked index.
template <int D, int R, int IB>
__device__ __forceinline__ void hpc_top2(const float (&x)[R][D], const hpc_cent_smem &cs,
                                         float (&d1)[R], int (&j1)[R], float (&d2)[R]) {
  constexpr bool PACKED = IB > 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    d1[r] = __int_as_float(0x7f7fffff);
    d2[r] = d1[r];
    j1[r] = 0;
  }
#pragma unroll 1
  for (int j = 0; j < cs.kp; j += 2) {
    float va[R], vb[R];
    hpc_pair_values<D, R>(x, cs, j, va, vb);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (PACKED) {
        const float ka = hpc_key_b<IB>(va[r], j), kb = hpc_key_b<IB>(vb[r], j + 1);
        d2[r] = fminf(d2[r], fmaxf(d1[r], ka));
        d1[r] = fminf(d1[r], ka);
        d2[r] = fminf(d2[r], fmaxf(d1[r], kb));
        d1[r] = fminf(d1[r], kb);
      } else {
        // pair tournament (lower index on ties), then merge into (d1, d2)
        const bool bl = vb[r] < va[r];
        const float lo = bl ? vb[r] : va[r];
        const float hi = bl ? va[r] : vb[r];
        const int jl = bl ? j + 1 : j;
        d2[r] = fminf(fminf(d2[r], hi), fmaxf(d1[r], lo));
        j1[r] = lo < d1[r] ? jl : j1[r];
        d1[r] = fminf(d1[r], lo);
      }
    }
  }
  if constexpr (PACKED) {
#pragma unroll
    for (int r = 0; r < R; ++r) j1[r] = min(__float_as_int(d1[r]) & ((1 << IB) - 1), cs.kp - 1);
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

// FP32 direct form x - c with c = -0.5 * cm (exact), one FMA per dimension
// in dimension order: the same rounding as the K-means++ weights.
template <int D>
__device__ __forceinline__ float hpc_dist32_cm(const float (&x)[D], const float *cm) {
  float acc = 0.0f;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const float diff = __fmaf_rn(0.5f, cm[t], x[t]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return acc;
}

// Direct-form squared distance to the chosen centroid with two interleaved
// partial sums; relative error <= (D/2 + 4) u.  Used for the objective.
template <int D>
__device__ __forceinline__ float hpc_dist_direct_cm(const float (&x)[D], const float *cm) {
  float2 acc = make_float2(0.0f, 0.0f);
  const float2 half = make_float2(0.5f, 0.5f);
#pragma unroll
  for (int t = 0; t + 1 < D; t += 2) {
    const float2 e = hpc_fma2(half, make_float2(cm[t], cm[t + 1]), make_float2(x[t], x[t + 1]));
    acc = hpc_fma2(e, e, acc);
  }
  return acc.x + acc.y;
}

// Warp-cooperative exact assignment of one row (every lane calls it with
// the same row pointer).  Returns the label; lanes split the centroids.
template <int D>
__device__ __noinline__ int hpc_rescore_row(const float *__restrict__ xrow, int d,
                                            const hpc_cent_smem &cs) {
  const int lane = threadIdx.x & 31;
  float x[D];
  hpc_load_row<D>(x, xrow, d);
  // Phase 1: FP32 direct form, relative error <= (D + 3) u of each value.
  float a1 = __int_as_float(0x7f800000), a2 = a1;
  int ja = 0x7fffffff;
  for (int j = lane; j < cs.kp; j += 32) {
    if (hpc_is_dead(cs, j)) continue;
    const float v = hpc_dist32_cm<D>(x, cs.cm + j * hpc_cstride(D));
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
  if (a2 - a1 > bound) return ja < cs.kp ? ja : 0;
  // Phase 2: double precision, same operation order as the reference.
  double b = __longlong_as_double(0x7ff0000000000000ll);
  int jb = 0x7fffffff;
  for (int j = lane; j < cs.kp; j += 32) {
    if (hpc_is_dead(cs, j)) continue;
    double acc = 0.0;
    for (int t = 0; t < d; ++t) {
      const double c = -0.5 * (double)cs.cm[j * hpc_cstride(D) + t];
      const double diff = __dsub_rn((double)x[t], c);
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
  return jb < cs.kp ? jb : 0;
}

// FP32 stage of the exact assignment of one row by one thread (the
// per-thread form of hpc_rescore_row's first phase): direct form against
// every live centroid with its relative bound (D + 3) u.  Returns the label,
// or -1 when the two best are not separated (the caller then settles the
// row in FP64, warp-cooperatively: FP64 runs at a small fraction of the
// FP32 rate, so one thread must not walk every centroid in it).
template <int D>
__device__ __noinline__ int hpc_exact_row32(const float (&x)[D], const hpc_cent_smem &cs) {
  float a1 = __int_as_float(0x7f800000), a2 = a1;
  int ja = 0;
  for (int j = 0; j < cs.kp; ++j) {
    if (hpc_is_dead(cs, j)) continue;
    const float v = hpc_dist32_cm<D>(x, cs.cm + j * hpc_cstride(D));
    if (v < a1) {
      a2 = a1;
      a1 = v;
      ja = j;
    } else {
      a2 = fminf(a2, v);
    }
  }
  const float bound = (float)(D + 3) * HPC_U32 * 1.001f * (a1 + a2);
  return a2 - a1 > bound ? ja : -1;
}

// Assigns the R rows of this thread in row group `base` (rows
// base + r * THREADS + tid).  Every thread of the block must call it with
// the same base.  Returns the FP32 sum of the direct-form distances of the
// thread's valid rows; valid[r] / lab[r] describe each row.
// (x receives the thread's rows, zero-padded, for callers that reuse them.)
template <int D, int R, int THREADS, int IB>
__device__ __forceinline__ float hpc_assign_group_x(const float *__restrict__ X, int64_t n, int d,
                                                    int64_t base, const hpc_cent_smem &cs,
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
  hpc_top2<D, R, IB>(x, cs, d1, lab, d2);
  float dd[R];
  bool flag[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    // a NaN/inf row never updates d1: its label is meaningless, use slot 0
    const bool found = d1[r] < HPC_DEAD * 0.5f;
    if (!found) lab[r] = 0;
    dd[r] = hpc_dist_direct_cm<D>(x[r], cs.cm + lab[r] * hpc_cstride(D));
    // ||x|| <= sqrt(dd) + ||c_j1|| <= sqrt(dd) + cmax
    const float rad = sqrtf(dd[r]) * 1.0001f + 2.0f * cs.cmax * 1.00001f;
    float bound = 2.001f * (float)(D + 4) * HPC_U32 * rad * rad;
    // keys: 2 * 2^(IB-23) (|k1| + |k2|)
    if (IB > 0) bound += 1.0001f * ldexpf(1.0f, IB - 22) * (fabsf(d1[r]) + fabsf(d2[r]));
    const bool ok = found && isfinite(dd[r]);
    flag[r] = valid[r] && ok && !(d2[r] - d1[r] > bound);
    if (valid[r] && !ok) {  // NaN/inf row or out-of-range distance
      hpc_status_set(status, HPC_ERR_NONFINITE);
      valid[r] = false;
    }
  }
  // warp-cooperative rescoring of flagged rows
#pragma unroll
  for (int r = 0; r < R; ++r) {
    unsigned m = __ballot_sync(0xffffffffu, flag[r]);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int64_t i = base + (int64_t)r * THREADS + (tid & ~31) + src;
      const int j = hpc_rescore_row<D>(X + i * d, d, cs);
      if ((tid & 31) == src && j != lab[r]) {
        lab[r] = j;
        dd[r] = hpc_dist_direct_cm<D>(x[r], cs.cm + j * hpc_cstride(D));
      }
    }
  }
  float fsum = 0.0f;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (valid[r]) fsum += dd[r];
  return fsum;
}

template <int D, int R, int THREADS, int IB>
__device__ __forceinline__ float hpc_assign_group(const float *__restrict__ X, int64_t n, int d,
                                                  int64_t base, const hpc_cent_smem &cs,
                                                  int (&lab)[R], bool (&valid)[R], int *status) {
  float x[R][D];
  return hpc_assign_group_x<D, R, THREADS, IB>(X, n, d, base, cs, x, lab, valid, status);
}

// Fixed-order sum of n doubles by the whole block (thread 0 gets the result).
__device__ __forceinline__ double hpc_block_sum_array(const double *p, int n, double *scratch32) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(p + i);
  return hpc_block_sum(v, scratch32);
}
