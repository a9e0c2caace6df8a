// Full-data objective (Eq. 1) for rows of 16 or 32 floats, with the x.c
// contraction of the nearest-centroid search on the tensor cores in split
// TF32 and everything else exact.
//
// Search value of centroid j for row x: v_j = ||c_j||^2 + x.c'_j, c' = -2c
// (the ||x||^2 term is common to a row).  The dot products run as tcgen05
// TF32 MMAs with three terms per K step:
//   x.c' ~ x_h.c'_h + x_h.c'_l + x_l.c'_h
// x_h = x with its low 13 mantissa bits cleared (a TF32 value), x_l = x - x_h
// (exact in FP32, |x_l| < 2^-10 |x|, the tensor core keeps its TF32 part);
// c'_h = c' rounded to TF32, c'_l = (c' - c'_h) rounded to TF32.  All three
// products are exact; the dropped terms are below 1.8 * 2^-20 |x_t| |c'_t|
// per coordinate.  With FP32 accumulation over 3 D / 8 MMA steps, the FP32
// norms and the final add, every computed v_j lies within 2^-17.8
// (||x|| + max||c||)^2 of the exact one; the kernel uses
// E = 2^-16 (||x|| + max||c||)^2, four times that.  A row whose top-2 margin
// exceeds 2E (plus the 2^-17 (|k1| + |k2|) of the packed keys) has the exact
// nearest centroid.  For the others the two nearest candidates are computed
// exactly (FP32 direct form); every other centroid is at least
// ||x||^2 + d2 - E away, which settles nearly all of them; the rest are
// rescored by the warp (FP32 direct form against every centroid, then FP64
// in the oracle's order, ties to the lowest index).  The objective adds the
// FP32 direct-form distance to the chosen centroid, from the exact row: per
// thread as an FP32 TwoSum pair (about 2^-48 relative, no FP64 instruction
// per row), then per block in FP64.
//
// Data path per 128-row tile (thread t owns tile row t = TMEM lane t):
//   TMA (2-D tile, 64/128-byte swizzle) -> shared-memory ring of 4 tiles
//   -> registers (conflict-free thanks to the swizzle) -> x_h | x_l written
//   to TMEM with tcgen05.st (the MMA's A operand, no shared-memory round
//   trip) -> one thread issues the 3 D / 8 MMAs (B = c'_h, c'_l in shared
//   memory) -> tcgen05.ld of the NP accumulator columns -> top-2, margin
//   test, direct distance, labels.
// The accumulator is double-buffered, so the MMAs of tile i + 1 run while
// the epilogue of tile i does.  One CTA per SM runs up to four such
// warpgroup pipelines side by side, each with its own ring, barriers and
// TMEM columns.  Every wait is bounded; a wait that runs out records
// HPC_ERR_TIMEOUT, the warpgroup leaves its loop at its next barrier,
// drains its copies and MMAs, and the CTA frees TMEM and returns.
#include "assign.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace {

constexpr int TS_M = 128;
constexpr uint64_t TS_WAIT_NS = 2000000000ull;
constexpr uint64_t TS_DRAIN_NS = 500000000ull;

__host__ __device__ constexpr int ts_pow2_cols(int c) {
  return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

// One CTA per SM (the occupancy rules give tensor-memory kernels one) with
// NWG independent warpgroup pipelines; each owns COLS_WG TMEM columns: one or
// two A buffers (x_h | x_l, 2 D columns each) and NACC accumulators (NP
// columns each).  Two accumulators let the MMAs of tile i + 1 run during the
// epilogue of tile i; where two would leave a single warpgroup (NP = 128)
// each warpgroup keeps one and runs its tiles strictly one after another,
// and two warpgroups overlap each other instead.
template <int D, int NP>
struct TsCfg {
  static constexpr uint32_t RB = D * 4;                 // bytes per row: 64 or 128
  static constexpr uint32_t SWZ = RB == 128 ? 2u : 4u;  // descriptor swizzle code
  static constexpr uint32_t TILE = TS_M * RB;
  static constexpr uint32_t BPART = NP * RB;  // one B part (hi or lo)
  // a second A buffer when it fits in the same power-of-two column count
  static constexpr int NBUF_A2 = ts_pow2_cols(4 * D + 2 * NP) == ts_pow2_cols(2 * D + 2 * NP) ? 2 : 1;
  static constexpr int NACC = 512 / ts_pow2_cols(2 * D * NBUF_A2 + 2 * NP) >= 2 ? 2 : 1;
  static constexpr int NBUF_A =
      NACC == 2 ? NBUF_A2 : (ts_pow2_cols(4 * D + NP) == ts_pow2_cols(2 * D + NP) ? 2 : 1);
  static constexpr int COLS_WG = ts_pow2_cols(2 * D * NBUF_A + NACC * NP);
  static constexpr int NWG = 512 / COLS_WG > 4 ? 4 : 512 / COLS_WG;
  static constexpr int THREADS = 128 * NWG;
  static constexpr int COLS = COLS_WG * NWG;
  static constexpr int RING = D == 16 ? 4 : 3;  // TMA ring slots per warpgroup
  static constexpr int NBAR = RING + 3;          // full[RING], mdone[2], drain
  static constexpr size_t BOP = (size_t)NWG * RING * TILE;
  static constexpr size_t CENT = BOP + 2 * (size_t)BPART;
  __host__ __device__ static size_t norms(int k) {
    return CENT + ((hpc_cent_smem_bytes(D, k) + 15) & ~(size_t)15);
  }
  __host__ __device__ static size_t bars(int k) { return norms(k) + (size_t)NP * 4; }
  __host__ __device__ static size_t total(int k) { return bars(k) + (size_t)NWG * NBAR * 8 + 1024; }
};

struct TsArgs {
  int64_t n;
  int d, k;
  const float *X;
  const float *C;
  const uint8_t *deg;
  double *f_out;
  int32_t *labels;
  int *status;
  double *part;
  unsigned *done_count;
  int64_t *queue;  // per CTA: queue_cap rows settled after the main loop
  int queue_cap;
};

__device__ __forceinline__ float tf32_rna(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// D = A[tmem] . B[smem] (+ D): A read from tensor memory.
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 16 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Named-barrier AND over the 128 threads of warpgroup `wg` (barrier 1 + wg).
__device__ __forceinline__ bool wg_sync_and(bool v, int wg) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, %2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + wg)
      : "memory");
  return r != 0;
}

template <int D, int NP, int IB>
__global__ void __launch_bounds__(TsCfg<D, NP>::THREADS, 1)
    tcs_objective_kernel(const __grid_constant__ CUtensorMap tmap, TsArgs a) {
  using Cfg = TsCfg<D, NP>;
  constexpr int CS = hpc_cstride(D);
  constexpr int RING = Cfg::RING;
  constexpr bool XT = Cfg::NBUF_A == 2;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float s_red[2];
  __shared__ double s_dsum[32];
  __shared__ bool s_last;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort[Cfg::NWG];
  __shared__ int s_qn;

  unsigned char *base =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *bop = base + Cfg::BOP;
  hpc_cent_smem cs;
  hpc_cent_bind(cs, base + Cfg::CENT, D, a.k);
  float *cnv = reinterpret_cast<float *>(base + Cfg::norms(a.k));
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + Cfg::bars(a.k));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = tid >> 7, r = tid & 127;  // warpgroup, tile row of this thread
  unsigned char *ring = base + (size_t)wg * RING * Cfg::TILE;
  uint64_t *full = bars + wg * Cfg::NBAR;
  uint64_t *mdone = full + RING;  // 2
  uint64_t *drain = mdone + 2;
  volatile int *abort = &s_abort[wg];

  const int64_t n = a.n;
  const int64_t ntiles = (n + TS_M - 1) / TS_M;
  const int64_t lanes = (int64_t)gridDim.x * Cfg::NWG;  // tile sequences
  const int64_t seq = (int64_t)blockIdx.x * Cfg::NWG + wg;
  const int my = seq < ntiles ? (int)((ntiles - 1 - seq) / lanes + 1) : 0;

  // ---- set-up: exact centroid block, B = split c', barriers, TMEM ----
  hpc_load_centroids<D>(cs, a.C, a.deg, a.k, a.d, s_red);
  for (int j = tid; j < NP; j += Cfg::THREADS) cnv[j] = j < cs.kp ? cs.cnz[j].x : HPC_DEAD;
  for (int e = tid; e < NP * D; e += Cfg::THREADS) {
    const int j = e / D, t = e - j * D;
    const float c = j < cs.kp ? cs.cm[j * CS + t] : 0.0f;  // -2c, zero padded
    const float hi = tf32_rna(c);
    const uint32_t off = hpc_swz_offset((uint32_t)j, (uint32_t)t * 4u, Cfg::RB);
    *reinterpret_cast<float *>(bop + off) = hi;
    *reinterpret_cast<float *>(bop + Cfg::BPART + off) = tf32_rna(c - hi);
  }
  hpc_fence_proxy_async();
  if (tid == 0) {
    for (int b = 0; b < Cfg::NWG * Cfg::NBAR; ++b) hpc_mbar_init(&bars[b], 1);
    for (int w = 0; w < Cfg::NWG; ++w) s_abort[w] = 0;
    s_qn = 0;
    hpc_fence_barrier_init();
  }
  if (warp == 0) hpc_tmem_alloc(&s_tmem, Cfg::COLS);
  hpc_tc_fence_before();
  __syncthreads();
  hpc_tc_fence_after();
  const uint32_t tmem = s_tmem + (uint32_t)(wg * Cfg::COLS_WG);  // this warpgroup's columns
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t d_col = 2 * D * Cfg::NBUF_A;  // A buffer(s), then the accumulator(s)
  auto acc_col = [&](int i) { return d_col + (uint32_t)(Cfg::NACC == 2 ? (i & 1) * NP : 0); };
  // with two A buffers the epilogue reads its row back from TMEM
  // (x = x_h + x_l exactly); with one, the row waits in registers
  const bool run = cs.live > 0 && my > 0;
  if (cs.live == 0 && n > 0 && tid == 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);

  int issued = 0;  // tiles whose TMA load was issued (thread r == 0)
  auto tile_row0 = [&](int i) { return (seq + (int64_t)i * lanes) * TS_M; };
  auto issue = [&](int i) {
    const int s = i % RING;
    hpc_mbar_arrive_expect_tx(&full[s], Cfg::TILE);
    hpc_tma_load_2d(ring + (size_t)s * Cfg::TILE, &tmap, &full[s], 0, (int)tile_row0(i));
    issued = i + 1;
  };

  // Reads row r of tile i from the ring into xr; once the A buffer is free,
  // writes x_h | x_l there; once the whole
  // warpgroup has, issues the MMAs of tile i and refills the ring slot.
  // Warpgroup-uniform result (false: stop).
  auto stage = [&](int i, float (&xout)[XT ? 1 : D]) -> bool {
    const int s = i % RING;
    bool ok = hpc_mbar_wait(&full[s], (uint32_t)(i / RING) & 1u, abort, a.status, TS_WAIT_NS);
    const unsigned char *tile = ring + (size_t)s * Cfg::TILE;
    float xr[D];
#pragma unroll
    for (int c = 0; c < D / 4; ++c) {
      float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (ok)
        q = *reinterpret_cast<const float4 *>(
            tile + hpc_swz_offset((uint32_t)r, (uint32_t)c * 16u, Cfg::RB));
      xr[4 * c] = q.x;
      xr[4 * c + 1] = q.y;
      xr[4 * c + 2] = q.z;
      xr[4 * c + 3] = q.w;
    }
    // the A buffer is free once the MMAs that last read it are done: those of
    // tile i - 1 (one buffer) or i - 2 (two, already waited for by the
    // epilogue of tile i - 2)
    if (Cfg::NBUF_A == 1 && i > 0)
      ok = hpc_mbar_wait(&mdone[(i - 1) & 1], (uint32_t)((i - 1) >> 1) & 1u, abort, a.status,
                         TS_WAIT_NS) && ok;
    hpc_tc_fence_after();
    const uint32_t a_col = (uint32_t)((i % Cfg::NBUF_A) * 2 * D);
    const uint32_t acol = tmem + lane_base + a_col;
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      uint32_t h[16], l[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const float v = xr[16 * c + t];
        h[t] = __float_as_uint(v) & 0xFFFFE000u;
        l[t] = __float_as_uint(v - __uint_as_float(h[t]));
      }
      tmem_st16(acol + (uint32_t)(16 * c), h);
      tmem_st16(acol + (uint32_t)(D + 16 * c), l);
    }
    if constexpr (!XT) {
#pragma unroll
      for (int t = 0; t < D; ++t) xout[t] = xr[t];
    }
    tmem_st_wait();
    hpc_tc_fence_before();
    if (!wg_sync_and(ok && !*abort, wg)) return false;
    if (r == 0) {
      hpc_tc_fence_after();
      constexpr uint32_t idesc = hpc_umma_idesc(2u, 2u, NP, TS_M);
      const uint32_t B = hpc_smem_u32(bop);
      const uint32_t a0 = tmem + a_col;
      const uint32_t d0 = tmem + acc_col(i);
#pragma unroll
      for (int ks = 0; ks < D / 8; ++ks) {
        const uint64_t bh = hpc_umma_desc(B + (uint32_t)ks * 32u, 16u, 8u * Cfg::RB, Cfg::SWZ);
        const uint64_t bl =
            hpc_umma_desc(B + Cfg::BPART + (uint32_t)ks * 32u, 16u, 8u * Cfg::RB, Cfg::SWZ);
        mma_tf32_tmem_a(d0, a0 + (uint32_t)(8 * ks), bh, idesc, ks > 0 ? 1u : 0u);
        mma_tf32_tmem_a(d0, a0 + (uint32_t)(8 * ks), bl, idesc, 1u);
        mma_tf32_tmem_a(d0, a0 + (uint32_t)(D + 8 * ks), bh, idesc, 1u);
      }
      hpc_mma_commit(&mdone[i & 1]);
      if (i + RING < my) issue(i + RING);  // the warpgroup has read slot s
    }
    return true;
  };

  float fs_hi = 0.0f, fs_lo = 0.0f;  // objective partial of this thread's rows (TwoSum pair)
  if (run) {
    if (r == 0) {
      hpc_prefetch_tensormap(&tmap);
      for (int i = 0; i < RING && i < my; ++i) issue(i);
    }
    // epilogue of tile i, whose row this thread holds in x
    auto epilogue = [&](int i, const float (&xin)[XT ? 1 : D]) {
      const bool w = __all_sync(0xffffffffu, hpc_mbar_wait(&mdone[i & 1], (uint32_t)(i >> 1) & 1u,
                                                          abort, a.status, TS_WAIT_NS));
      if (w) {
        hpc_tc_fence_after();
        float x[D];
        if constexpr (XT) {
#pragma unroll
          for (int c = 0; c < (2 * D) / 32; ++c) {
            float hl[32];
            hpc_tmem_ld32(tmem + lane_base + (uint32_t)((i % Cfg::NBUF_A) * 2 * D + 32 * c), hl);
            if constexpr (D == 16) {
#pragma unroll
              for (int t = 0; t < 16; ++t) x[t] = hl[t] + hl[16 + t];
            } else {
#pragma unroll
              for (int t = 0; t < 32; ++t) {
                if (c == 0) x[t] = hl[t];
                else x[t] += hl[t];
              }
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) x[t] = xin[t];
        }
        const int64_t row = tile_row0(i) + r;
        bool valid = row < n;
        float d1 = __int_as_float(0x7f7fffff), d2 = d1, e1 = d1, e2 = d1;
        int j1 = 0, j2 = 0, je = 1, je2 = 1;
#pragma unroll
        for (int c = 0; c < NP / 32; ++c) {
          if (c * 32 >= cs.kp) break;  // same for the whole CTA
          float acc[32];
          hpc_tmem_ld32(tmem + lane_base + acc_col(i) + (uint32_t)(32 * c), acc);
          if constexpr (IB > 0) {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 4) {
              // columns past the live ones carry HPC_DEAD norms and never
              // win: scanning the whole chunk without a branch per group is
              // faster except at d = 32 with 32 columns, whose registers
              // are short
              if (D == 32 && NP == 32 && c * 32 + jj >= cs.kp) break;
              const float4 cn = *reinterpret_cast<const float4 *>(cnv + c * 32 + jj);
              const int j = c * 32 + jj;
              // alternate groups of four go to two independent top-2 chains
              // (d1, d2) and (e1, e2), merged below; one chain at d = 32
              // with 32 columns, whose registers are short
              const bool alt = (jj & 4) && !(D == 32 && NP == 32);
              float &t1 = alt ? e1 : d1, &t2 = alt ? e2 : d2;
              hpc_top2_fold4(t1, t2, hpc_key_b<IB>(cn.x + acc[jj], j),
                             hpc_key_b<IB>(cn.y + acc[jj + 1], j + 1),
                             hpc_key_b<IB>(cn.z + acc[jj + 2], j + 2),
                             hpc_key_b<IB>(cn.w + acc[jj + 3], j + 3));
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 2) {
              if (c * 32 + jj >= cs.kp) break;
              const float2 cn = *reinterpret_cast<const float2 *>(cnv + c * 32 + jj);
              const float v0 = cn.x + acc[jj], v1 = cn.y + acc[jj + 1];
              const int j = c * 32 + jj;
              if (v0 < d1) {
                d2 = d1;
                j2 = j1;
                d1 = v0;
                j1 = j;
              } else if (v0 < d2) {
                d2 = v0;
                j2 = j;
              }
              if (v1 < e1) {
                e2 = e1;
                je2 = je;
                e1 = v1;
                je = j + 1;
              } else if (v1 < e2) {
                e2 = v1;
                je2 = j + 1;
              }
            }
          }
        }
        if constexpr (IB > 0) {
          d2 = hpc_min3(d2, e2, fmaxf(d1, e1));
          d1 = fminf(d1, e1);
          j1 = min(__float_as_int(d1) & ((1 << IB) - 1), cs.kp - 1);
          j2 = min(__float_as_int(d2) & ((1 << IB) - 1), cs.kp - 1);
        } else {
          // merge the even / odd chains, lower index on equal values
          if (e1 < d1 || (e1 == d1 && je < j1)) {
            if (d1 < e2 || (d1 == e2 && j1 < je2)) {
              d2 = d1;
              j2 = j1;
            } else {
              d2 = e2;
              j2 = je2;
            }
            d1 = e1;
            j1 = je;
          } else if (e1 < d2 || (e1 == d2 && je < j2)) {
            d2 = e1;
            j2 = je;
          }
        }
        const bool found = d1 < HPC_DEAD * 0.5f;
        if (!found) j1 = 0;
        float dd = hpc_dist_direct_cm<D>(x, cs.cm + j1 * CS);
        // ||x|| <= sqrt(dd) + ||c_j1|| <= sqrt(dd) + cmax (approximate square
        // root, 2 ulp, covered by the 1.0001 factor)
        const float rad = dd * rsqrtf(dd + 1e-30f) * 1.0001f + 2.0f * cs.cmax * 1.00001f;
        float win = 2.0f * 1.52587890625e-05f * rad * rad;  // 2E, E = 2^-16 (||x|| + cmax)^2
        if (IB > 0) win += 1.0001f * ldexpf(1.0f, IB - 22) * (fabsf(d1) + fabsf(d2));  // keys
        const bool ok = found && isfinite(dd) && isfinite(win);
        if (valid && !ok) {
          hpc_status_set(a.status, HPC_ERR_NONFINITE);
          valid = false;
        }
        // near ties go to this CTA's queue and are settled after the loop,
        // one row per thread, so that no warp holds up its warpgroup
        bool near = valid && !(d2 - d1 > win);
        if (__any_sync(0xffffffffu, near)) {
          const unsigned qm = __ballot_sync(0xffffffffu, near);
          int q0 = 0;
          if (qm && lane == 0) q0 = atomicAdd(&s_qn, __popc(qm));
          q0 = __shfl_sync(0xffffffffu, q0, 0);
          const int q = q0 + __popc(qm & ((1u << lane) - 1u));
          if (near && q < a.queue_cap) {
            a.queue[(int64_t)blockIdx.x * a.queue_cap + q] = row;
            near = false;
            valid = false;  // its label and distance come from the queue pass
          }
        }
        bool rescore = false;
        if (__any_sync(0xffffffffu, near) && near) {  // queue full: settle it here
          // the two nearest by the tensor-core values, exactly; every other
          // centroid is at least ||x||^2 + d2 - E away
          const bool has2 = d2 < HPC_DEAD * 0.5f;
          const float ex2 =
              has2 ? hpc_dist_direct_cm<D>(x, cs.cm + j2 * CS) : __int_as_float(0x7f800000);
          float2 s2 = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int t = 0; t < D; t += 2)
            s2 = hpc_fma2(make_float2(x[t], x[t + 1]), make_float2(x[t], x[t + 1]), s2);
          const float nx = s2.x + s2.y;
          const float E = 0.5f * win;
          constexpr float rho = (float)(D + 4) * HPC_U32 * 1.001f;  // direct-form bound
          const float others = nx * (1.0f - (float)(D + 2) * HPC_U32 * 1.01f) + d2 - E -
                               4.0f * HPC_U32 * (nx + fabsf(d2) + E);
          const bool lo1 = dd < ex2 || (dd == ex2 && j1 < j2);
          const float lo = lo1 ? dd : ex2, hi = lo1 ? ex2 : dd;
          if (lo * (1.0f + rho) < others && hi * (1.0f - rho) > lo * (1.0f + rho)) {
            if (!lo1) {
              j1 = j2;
              dd = ex2;
            }
          } else {
            rescore = true;  // a third candidate, or a tie FP32 cannot split
          }
        }
        // the warp settles the remaining rows exactly (FP32, then FP64)
        unsigned m = __ballot_sync(0xffffffffu, rescore);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int64_t ri = tile_row0(i) + 32 * (warp & 3) + src;
          const int j = hpc_rescore_row<D>(a.X + ri * a.d, a.d, cs);
          if (lane == src && j != j1) {
            j1 = j;
            dd = hpc_dist_direct_cm<D>(x, cs.cm + j1 * CS);
          }
        }
        if (valid) {
          hpc_sum2_add(fs_hi, fs_lo, dd);
          if (a.labels) a.labels[row] = j1;
        }
      } else {
        *abort = 1;
      }
    };
    // row registers alternate between the two arrays (no copies)
    float xa[XT ? 1 : D], xb[XT ? 1 : D];
    if constexpr (Cfg::NACC == 2) {
      bool go = stage(0, xa);
      for (int i = 0; go && i < my; i += 2) {
        if (i + 1 < my) go = stage(i + 1, xb);
        epilogue(i, xa);
        if (!go || i + 1 >= my) break;
        if (i + 2 < my) go = stage(i + 2, xa);
        epilogue(i + 1, xb);
      }
    } else {
      // one accumulator: the MMAs of tile i + 1 are issued (inside stage, after
      // the warpgroup barrier) only once every thread has read tile i's
      for (int i = 0; i < my; ++i) {
        if (!stage(i, xa)) break;
        epilogue(i, xa);
      }
    }
  }

  // ---- queued near ties: exact assignment, one row per thread ----
  __syncthreads();
  {
    const int nq = min(s_qn, a.queue_cap);
    const int64_t *qb = a.queue + (int64_t)blockIdx.x * a.queue_cap;
    for (int q0 = warp * 32; q0 < nq; q0 += Cfg::THREADS) {  // warp-uniform trip count
      const int q = q0 + lane;
      const bool have = q < nq;
      const int64_t row = have ? qb[q] : 0;
      float xr[D];
      hpc_load_row<D>(xr, a.X + row * a.d, a.d);
      int j = have ? hpc_exact_row32<D>(xr, cs) : 0;
      // rows FP32 cannot settle: the warp rescores them in FP64
      unsigned m = __ballot_sync(0xffffffffu, have && j < 0);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int64_t ri = __shfl_sync(0xffffffffu, row, src);
        const int jr = hpc_rescore_row<D>(a.X + ri * a.d, a.d, cs);
        if (lane == src) j = jr;
      }
      if (have) {
        const float dd = hpc_dist_direct_cm<D>(xr, cs.cm + j * CS);
        hpc_sum2_add(fs_hi, fs_lo, dd);
        if (a.labels) a.labels[row] = j;
      }
    }
  }

  // ---- drain: no copy or MMA may still target this CTA's memory ----
  if (r == 0 && run) {
    int no_abort = 0;
    hpc_mma_commit(drain);
    hpc_mbar_wait(drain, 0, (volatile int *)&no_abort, a.status, TS_DRAIN_NS);
    // loads issued but never consumed (only after an early stop): the last
    // fill of every slot
    if (*abort)
      for (int u = issued > RING ? issued - RING : 0; u < issued; ++u)
        hpc_mbar_wait(&full[u % RING], (uint32_t)(u / RING) & 1u, (volatile int *)&no_abort,
                      a.status, TS_DRAIN_NS);
  }

  // ---- objective partial, last block reduces in a fixed order ----
  const double bsum = hpc_block_sum((double)fs_hi + (double)fs_lo, s_dsum);
  if (tid == 0) {
    a.part[blockIdx.x] = bsum;
    __threadfence();
    const unsigned prev = atomicAdd(a.done_count, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const double f = hpc_block_sum_array(a.part, (int)gridDim.x, s_dsum);
    if (tid == 0) {
      *a.f_out = (cs.live == 0 && n > 0) ? __longlong_as_double(0x7ff8000000000000ll) : f;
      *a.done_count = 0u;
    }
  }
  hpc_tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    hpc_tc_fence_after();
    hpc_tmem_dealloc(s_tmem, Cfg::COLS);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <int D, int NP, int IB>
int tcs_launch_t(const hpc_launch &Lc, const ObjArgsHost &h) {
  using Cfg = TsCfg<D, NP>;
  auto kern = tcs_objective_kernel<D, NP, IB>;
  const size_t smem = Cfg::total(h.k);
  if (smem > (size_t)Lc.smem_optin) return HPC_ERR_UNSUPPORTED;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return HPC_ERR_UNSUPPORTED;
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)D, (cuuint64_t)h.n};
  cuuint64_t gstride[1] = {(cuuint64_t)D * 4};
  cuuint32_t box[2] = {(cuuint32_t)D, (cuuint32_t)TS_M};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle swz = D == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(h.X), gdim, gstride, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HPC_ERR_CUDA;
  // one CTA per SM: its warpgroups hold all the tensor memory they need
  const int64_t ntiles = (h.n + TS_M - 1) / TS_M;
  int64_t G = Lc.num_sms;
  const int64_t want = (ntiles + Cfg::NWG - 1) / Cfg::NWG;
  if (G > want) G = want;
  if (G < 1) G = 1;
  if (G > h.max_blocks) G = h.max_blocks;
  TsArgs a;
  a.n = h.n;
  a.d = h.d;
  a.k = h.k;
  a.X = h.X;
  a.C = h.C;
  a.deg = h.deg;
  a.f_out = h.f_out;
  a.labels = h.labels;
  a.status = h.status;
  a.part = h.part;
  a.done_count = h.done_count;
  a.queue = h.queue;
  a.queue_cap = (int)h.queue_cap;
  if (!a.queue || a.queue_cap < 0 || G > h.queue_ctas) a.queue_cap = 0;
  kern<<<(unsigned)G, Cfg::THREADS, smem, Lc.stream>>>(map, a);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

template <int D>
int tcs_dispatch(const hpc_launch &L, const ObjArgsHost &h) {
  if (h.k <= 32) return tcs_launch_t<D, 32, 5>(L, h);
  if (h.k <= 64) return tcs_launch_t<D, 64, 7>(L, h);
  return tcs_launch_t<D, 128, 7>(L, h);
}

}  // namespace

bool hpc_tcs_objective_supported(int d, int k, int64_t n) {
  return n >= 1 && n < ((int64_t)1 << 31) - 2 * TS_M && (d == 16 || d == 32) && k >= 1 && k <= 128;
}

int hpc_tcs_objective_launch(const hpc_launch &L, const ObjArgsHost &h) {
  if (!hpc_tcs_objective_supported(h.d, h.k, h.n)) return HPC_ERR_UNSUPPORTED;
  return h.d == 16 ? tcs_dispatch<16>(L, h) : tcs_dispatch<32>(L, h);
}
