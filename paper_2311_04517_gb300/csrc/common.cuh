// Device helpers shared by the HPClust kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hpclust.h"

#define HPC_TAG_SAMPLE 0u
#define HPC_TAG_SEED 1u

// Upper limit of any device-side wait (grid barrier): an error status is
// written and the kernel returns instead of hanging.
#define HPC_WAIT_LIMIT_NS (4ull * 1000ull * 1000ull * 1000ull)

#define HPC_MAX_D 128
#define HPC_MAX_ITER 100000

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter-based, so every
// (seed, worker, round, tag, j) draw is computed independently by any thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hpc_philox4x64_10(uint64_t x[4], uint64_t k0,
                                                  uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
    const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
    const uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
  }
}

// Block b (four draws 4b..4b+3) of stream (seed, worker, round, tag).
__device__ __forceinline__ void hpc_draw_block(uint64_t seed, uint32_t worker,
                                               uint32_t round, uint32_t tag,
                                               uint64_t b, uint64_t out[4]) {
  out[0] = b;
  out[1] = round;
  out[2] = tag;
  out[3] = 0;
  hpc_philox4x64_10(out, seed, (uint64_t)worker);
}

__device__ __forceinline__ uint64_t hpc_draw(uint64_t seed, uint32_t worker,
                                             uint32_t round, uint32_t tag,
                                             uint64_t j) {
  uint64_t v[4];
  hpc_draw_block(seed, worker, round, tag, j >> 2, v);
  const uint32_t w = (uint32_t)(j & 3u);
  return w == 0 ? v[0] : w == 1 ? v[1] : w == 2 ? v[2] : v[3];
}

// floor(r * m / 2^64)
__device__ __forceinline__ uint64_t hpc_scale_word(uint64_t r, uint64_t m) {
  return __umul64hi(r, m);
}

// ---------------------------------------------------------------------------
// Barrier over the `nblocks` blocks of a group (the whole grid, or one
// task's blocks) of a cooperative launch, with a bounded wait.  Returns false
// (in every thread of the block) when the device status word carries an
// error, including a wait that ran past the limit; the caller then returns.
// The barrier words are zeroed before each launch.  `arrive` counts every
// arrival of the launch (generation g is complete at (g + 1) nblocks);
// `gen` is the generation, bit 31 set when the last block of a generation
// saw an error in the status word.
// ---------------------------------------------------------------------------
struct hpc_gridbar {
  unsigned int arrive;
  unsigned int gen;
};

__device__ __forceinline__ unsigned hpc_ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void hpc_st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// atomic add with acquire-release semantics at GPU scope; returns the old value
__device__ __forceinline__ unsigned hpc_atom_add_acq_rel(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ uint64_t hpc_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int hpc_status_get(const int *status) {
  return *(volatile const int *)status;
}

__device__ __forceinline__ void hpc_status_set(int *status, int code) {
  atomicCAS(status, 0, code);
}

static __device__ __noinline__ bool hpc_grid_sync(hpc_gridbar *bar, int *status, unsigned nblocks,
                                                  uint64_t limit_ns = HPC_WAIT_LIMIT_NS) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    // a block arrives at generation g only after it saw g released, and g
    // cannot advance before it arrives: this read is the current generation
    const unsigned g = hpc_ld_acquire(&bar->gen);
    // the fence makes the whole block's writes (ordered before this thread by
    // __syncthreads) visible at GPU scope, as a grid-wide sync does; the
    // acquire half of the count lets the last block see every other block's
    __threadfence();
    const unsigned prev = hpc_atom_add_acq_rel(&bar->arrive, 1u);
    if ((prev + 1u) % nblocks == 0u) {
      const bool err = hpc_status_get(status) != 0;
      hpc_st_release(&bar->gen, (g + 1u) | (err ? 0x80000000u : 0u));
      ok = err ? 0 : 1;
    } else {
      const uint64_t t0 = hpc_globaltimer();
      unsigned v;
      for (unsigned n = 1; (v = hpc_ld_acquire(&bar->gen)) == g; ++n) {
        if ((n & 31u) == 0u) {  // the status word and the clock, now and then
          if (hpc_status_get(status) != 0) {
            ok = 0;
            break;
          }
          if (hpc_globaltimer() - t0 > limit_ns) {
            hpc_status_set(status, HPC_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
        __nanosleep(32);
      }
      if (ok && (v & 0x80000000u)) ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Distances
// ---------------------------------------------------------------------------
// Squared distance in the rounding that K-means++ decisions are defined in:
// float difference, one fused multiply-add per dimension, dimension order.
template <int D>
__device__ __forceinline__ float hpc_dist32_seq(const float (&x)[D], const float *c) {
  float acc = 0.0f;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    const float diff = __fsub_rn(x[t], c[t]);
    acc = __fmaf_rn(diff, diff, acc);
  }
  return acc;
}

// Direct-form squared distance with two interleaved partial sums (even and
// odd dimensions) using packed FMA; used for the objective of the chosen
// centroid.  |error| <= (D/2 + 2) u * value.
template <int D>
__device__ __forceinline__ float hpc_dist_direct(const float (&x)[D], const float *c) {
  float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
  for (int t = 0; t + 1 < D; t += 2) {
    const float e0 = x[t] - c[t], e1 = x[t + 1] - c[t + 1];
    a0 = fmaf(e0, e0, a0);
    a1 = fmaf(e1, e1, a1);
  }
  if (D & 1) {
    const float e = x[D - 1] - c[D - 1];
    a0 = fmaf(e, e, a0);
  }
  return a0 + a1;
}

// Packed two-lane FMA (sm_100 family): r = a * b + c per lane.
__device__ __forceinline__ float2 hpc_fma2(float2 a, float2 b, float2 c) {
  unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
  unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
  unsigned long long rc = *reinterpret_cast<unsigned long long *>(&c);
  unsigned long long rd;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  return *reinterpret_cast<float2 *>(&rd);
}

// ---------------------------------------------------------------------------
// 64-bit fixed-point grid for exact, order-independent sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int hpc_bit_length(int64_t s) {
  return s <= 0 ? 0 : 64 - __clzll((unsigned long long)s);
}

// e with 2^(e-1) <= M < 2^e, for finite M > 0 (frexp exponent).
__device__ __forceinline__ int hpc_frexp_exp(float M) {
  int e;
  frexpf(M, &e);
  return e;
}

// floor(w * 2^F) for finite w >= 0, exact (w has a 24-bit significand).
__device__ __forceinline__ int64_t hpc_quant(float w, int F) {
  const uint32_t b = __float_as_uint(w);
  const uint32_t ebits = (b >> 23) & 0xFFu;
  if (b == 0u) return 0;
  uint64_t mant = b & 0x7FFFFFu;
  int exp2;
  if (ebits == 0) {
    exp2 = -149;  // subnormal: w = mant * 2^-149
  } else {
    mant |= 0x800000u;
    exp2 = (int)ebits - 150;  // w = mant * 2^(ebits-150)
  }
  const int sh = exp2 + F;
  if (sh >= 0) return (int64_t)(mant << sh);  // callers keep this below 2^62
  if (sh <= -64) return 0;
  return (int64_t)(mant >> (-sh));
}

// Bits of a non-negative float ordered like the value (for atomicMax).
__device__ __forceinline__ unsigned hpc_fbits(float v) { return __float_as_uint(v); }

// ---------------------------------------------------------------------------
// Misc
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hpc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long hpc_warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one unsigned 64-bit integer per thread (two's complement, so
// signed values add too; blockDim.x a multiple of 32, at most 1024).  Result
// valid in thread 0.  Integer: exact and independent of the order.
__device__ __forceinline__ unsigned long long hpc_block_sum_u64(unsigned long long v,
                                                                unsigned long long *scratch32) {
  v = hpc_warp_sum_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch32[wid] = v;
  __syncthreads();
  unsigned long long r = 0ull;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) r += scratch32[w];
  }
  return r;
}

// 2^e as a float or a double, built from its bits (no arithmetic):
// -126 <= e <= 127 for the float, -1022 <= e <= 1023 for the double.
__device__ __forceinline__ float hpc_pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double hpc_pow2d(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// q 2^-F / cnt rounded to float, for |q| < 2^62, 1 <= cnt < 2^32 and
// 0 <= F <= 126, without an FP64 instruction (FP64 runs at 1/64 of the FP32
// rate on GB300): q and cnt as unevaluated sums of two floats, one FP32
// division, and a correction from the first quotient's residual (exact by
// FMA).  The result is within one unit in the last place of the exact
// quotient (the FP64 path it replaces rounded twice as well).
__device__ __forceinline__ float hpc_mean_f32(long long q, unsigned cnt, int F) {
  if (q == 0) return 0.0f;
  const bool neg = q < 0;
  const unsigned long long a = neg ? (unsigned long long)(-q) : (unsigned long long)q;
  const int L = 64 - __clzll((long long)a);
  const int sh = L > 24 ? L - 24 : 0;
  const unsigned long long top = a >> sh;  // < 2^24: exact in a float
  const unsigned long long rem = a - (top << sh);
  const float qh = (float)(unsigned)top * hpc_pow2f(sh);
  const int Lr = rem ? 64 - __clzll((long long)rem) : 0;
  const int shr = Lr > 31 ? Lr - 31 : 0;
  const float ql = (float)(unsigned)(rem >> shr) * hpc_pow2f(shr);
  const float ch = (float)cnt;
  const float cl = cnt < (1u << 24) ? 0.0f : (float)(int)((long long)cnt - (long long)ch);
  const float m0 = __fdiv_rn(qh, ch);
  const float r = (fmaf(-m0, ch, qh) + ql) - m0 * cl;
  const float m = m0 + __fdiv_rn(r, ch);
  const float v = m * hpc_pow2f(-F);
  return neg ? -v : v;
}

// Fixed-order block sum of one double per thread (blockDim.x multiple of 32,
// at most 1024).  Result valid in thread 0.
__device__ __forceinline__ double hpc_block_sum(double v, double *scratch32) {
  v = hpc_warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) scratch32[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) r += scratch32[w];
  }
  return r;
}

// Row loader for a D-wide register row from a row of d <= D floats (zero
// padding beyond d).  Vector loads when d == D and the row is aligned.
template <int D>
__device__ __forceinline__ void hpc_load_row(float (&x)[D], const float *__restrict__ p, int d) {
  if (d == D && (D % 4) == 0) {
#pragma unroll
    for (int c = 0; c < D / 4; ++c) {
      const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + c);
      x[4 * c + 0] = v.x;
      x[4 * c + 1] = v.y;
      x[4 * c + 2] = v.z;
      x[4 * c + 3] = v.w;
    }
  } else if (d == D && D == 2) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    x[0] = v.x;
    x[1] = v.y;
  } else {
#pragma unroll
    for (int t = 0; t < D; ++t) x[t] = t < d ? __ldg(p + t) : 0.0f;
  }
}

template <int D>
__device__ __forceinline__ bool hpc_row_finite(const float (&x)[D]) {
  bool ok = true;
#pragma unroll
  for (int t = 0; t < D; ++t) ok &= isfinite(x[t]);
  return ok;
}

// Dimension padding used by the templated kernels.
static inline int hpc_pad_dim(int d) {
  if (d <= 2) return 2;
  if (d <= 4) return 4;
  if (d <= 8) return 8;
  if (d <= 16) return 16;
  if (d <= 32) return 32;
  if (d <= 64) return 64;
  return 128;
}
