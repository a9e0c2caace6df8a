// Full-data objective (Eq. 1) for 128 < k <= 512 centroids with the x.c
// contraction on the tensor cores in TF32.
//
// Search values, error bound and exact resolution are those of the TF32
// search for k <= 128: v_j = ||c_j||^2 - 2 x.c_j with x.c' (c' = -2c) from
// tcgen05 TF32 MMAs (the row tile as TMA staged it is the A operand, B is
// c' in FP32, of which the MMA reads the TF32 part), every computed value
// within E = 2^-10 (||x|| + max||c||)^2
// of the exact one; a row whose top-2 margin exceeds 2E (plus the packed
// keys' 2^(IB-22) (|k1| + |k2|)) has the exact nearest centroid, otherwise
// its two candidates are computed exactly and every other centroid is at
// least ||x||^2 + d2 - E away; rows still open are rescored by their warp
// against every centroid (FP32 direct form, then FP64 in the oracle's order,
// ties to the lowest index).  The objective adds the FP32 direct-form
// distance to the chosen centroid (per thread as an FP32 TwoSum pair, per
// block in FP64).
//
// What changes with k: a tile's accumulator is 256 or 512 TMEM columns, so
// the four epilogue warpgroups split the COLUMNS of each tile instead of
// taking whole tiles: warpgroup e folds columns [e NP/4, (e+1) NP/4) of all
// 128 rows into a partial top-2 per row (packed (value, index) keys with 8
// or 9 index bits) and leaves it in a shared-memory exchange buffer; the
// warpgroup e = i mod 4 then merges the four partials of tile i's rows and
// finishes them (exact distances, margin test, labels; rows whose window
// may hold a third candidate rescan the tile's accumulators in TMEM and take
// the candidates inside the window exactly, so a tile's banks are released
// only after its finishing warpgroup has looked).  Four exchange buffers
// rotate with mbarriers (ready: all 16 warps wrote; done: the finishing
// warpgroup read).  TMEM holds two 256-column banks: k <= 256
// double-buffers whole tiles; k <= 512 gives each tile both banks and
// commits them separately, so that the MMAs of the next tile's first bank
// run while the second bank is folded.  B holds c' in full FP32, so the
// exact distances of the finishing step read their centroids from it
// (shared memory, through the swizzle); a copy of the exact centroid block
// in the layout the warp-cooperative FP64 rescoring reads (rows of d + 4
// floats, norms) lives in global memory, written once per call by a
// one-block set-up kernel.
//
// One persistent CTA per SM: warp 0 TMA producer, warp 1 TMEM owner and MMA
// issuer (one thread), warps 2..17 the epilogue.  Every mbarrier wait is
// bounded; one that runs out records HPC_ERR_TIMEOUT and every role stops;
// in-flight copies and MMAs are drained before TMEM is freed.
#include "assign.cuh"
#include "kernels.h"
#include "tc.cuh"
#include "tc_rows.cuh"

namespace {

constexpr int TW_M = 128;
constexpr int TW_EPI0 = 2;                     // first epilogue warp
constexpr int TW_THREADS = (TW_EPI0 + 16) * 32;  // producer, MMA, four warpgroups
constexpr int TW_NX = 4;                       // exchange buffers
constexpr int TW_MAX_RING = 12;
constexpr uint64_t TW_WAIT_NS = 2000000000ull;
constexpr uint64_t TW_DRAIN_NS = 500000000ull;

template <int D>
struct TwCfg {
  static constexpr int CK = D < 32 ? D : 32;  // floats per swizzled chunk row
  static constexpr int NCH = D / CK;          // chunks per tile
  static constexpr uint32_t RB = CK * 4;      // bytes per chunk row (64 or 128)
  static constexpr uint32_t SWZ = RB == 128 ? 2u : 4u;
  static constexpr uint32_t CHUNK_BYTES = TW_M * RB;
};

// TMEM banks of 256 columns: NP = 256 uses one per tile (two tiles in
// flight), NP = 512 both.
template <int NP>
struct TwBanks {
  static constexpr int PARTS = NP / 256;        // banks per tile
  static constexpr int CPW = NP / 4;            // columns per epilogue warpgroup
  static constexpr int READERS = 16 / PARTS;    // epilogue warps reading one bank
};

// Shared memory: ring | B (NCH x NP rows of RB bytes) | norms | exchange | barriers
template <int D, int NP>
struct TwSmem {
  using Cfg = TwCfg<D>;
  __host__ __device__ static size_t bop(int nsx) { return (size_t)nsx * Cfg::CHUNK_BYTES; }
  __host__ __device__ static size_t norms(int nsx) {
    return bop(nsx) + (size_t)Cfg::NCH * NP * Cfg::RB;
  }
  __host__ __device__ static size_t xch(int nsx) { return norms(nsx) + (size_t)NP * 4; }
  __host__ __device__ static size_t bars(int nsx) {
    return xch(nsx) + (size_t)TW_NX * 4 * TW_M * 8;
  }
  // xfull, xfree per ring slot; accf, acce per bank; ready, done per
  // exchange buffer; drain; + 1024 for aligning the base
  __host__ __device__ static size_t total(int nsx) {
    return bars(nsx) + (size_t)(2 * nsx + 4 + 2 * TW_NX + 1) * 8 + 16 + 1024;
  }
};

struct TwArgs {
  int64_t n;
  int d, k, nsx;
  const float *X;
  unsigned char *gcent;  // exact centroid block (hpc_cent_smem layout), global
  const float *gmeta;    // [0] max ||c||, [1] live count (as int bits)
  double *f_out;
  int32_t *labels;
  int *status;
  double *part;
  unsigned *done_count;
};

// Centroid j's 16 values of c' = -2c starting at dimension t0, from the
// swizzled B operand (chunk t0 / CK, row j, 16-byte units where the swizzle
// put them).
template <int D, int NP>
__device__ __forceinline__ void b_chunk16(const unsigned char *bop, int j, int t0, float (&c)[16]) {
  using Cfg = TwCfg<D>;
  const unsigned char *rowp = bop + (size_t)(t0 / Cfg::CK) * NP * Cfg::RB;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 q = *reinterpret_cast<const float4 *>(
        rowp + hpc_swz_offset((uint32_t)j, (uint32_t)((t0 % Cfg::CK) + 4 * u) * 4u, Cfg::RB));
    c[4 * u] = q.x;
    c[4 * u + 1] = q.y;
    c[4 * u + 2] = q.z;
    c[4 * u + 3] = q.w;
  }
}

// The objective's direct form (two interleaved partial sums, as row_direct)
// of the row and centroid j, with c' from shared memory.
template <int D, int NP>
__device__ __forceinline__ float b_direct(const RowRef<D> &r, const unsigned char *bop, int j) {
  float2 acc = make_float2(0.0f, 0.0f);
  const float2 half = make_float2(0.5f, 0.5f);
#pragma unroll
  for (int t0 = 0; t0 < D; t0 += 16) {
    float v[16], c[16];
    row_chunk<D>(r, t0, v);
    b_chunk16<D, NP>(bop, j, t0, c);
#pragma unroll
    for (int t = 0; t < 16; t += 2) {
      const float2 e = hpc_fma2(half, make_float2(c[t], c[t + 1]), make_float2(v[t], v[t + 1]));
      acc = hpc_fma2(e, e, acc);
    }
  }
  return acc.x + acc.y;
}

// The sequential direct form (as row_dist32, relative error <= (D + 2) u).
template <int D, int NP>
__device__ __forceinline__ float b_dist32(const RowRef<D> &r, const unsigned char *bop, int j) {
  float acc = 0.0f;
#pragma unroll
  for (int t0 = 0; t0 < D; t0 += 16) {
    float v[16], c[16];
    row_chunk<D>(r, t0, v);
    b_chunk16<D, NP>(bop, j, t0, c);
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const float diff = __fmaf_rn(0.5f, c[t], v[t]);
      acc = __fmaf_rn(diff, diff, acc);
    }
  }
  return acc;
}

// One block: the exact centroid block in global memory, and its max norm and
// live count.
template <int D>
__global__ void tw_prep_kernel(const float *__restrict__ C, const uint8_t *__restrict__ deg, int k,
                               int d, unsigned char *gcent, float *gmeta) {
  __shared__ float s_red[2];
  hpc_cent_smem cs;
  hpc_cent_bind(cs, gcent, D, k);
  hpc_load_centroids<D>(cs, C, deg, k, d, s_red);
  if (threadIdx.x == 0) {
    gmeta[0] = cs.cmax;
    gmeta[1] = __int_as_float(cs.live);
  }
}

template <int D, int NP, int IB>
__global__ void __launch_bounds__(TW_THREADS, 1)
    tw_objective_kernel(const __grid_constant__ CUtensorMap tmap, TwArgs a) {
  using Cfg = TwCfg<D>;
  using L = TwSmem<D, NP>;
  using Bk = TwBanks<NP>;
  constexpr int NCH = Cfg::NCH;
  constexpr int CS = hpc_cstride(D);
  constexpr int PARTS = Bk::PARTS, CPW = Bk::CPW;
  const int nsx = a.nsx;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_dsum[32];
  __shared__ bool s_last;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  unsigned char *base =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *ring = base;
  unsigned char *bop = base + L::bop(nsx);
  float *cnv = reinterpret_cast<float *>(base + L::norms(nsx));
  float2 *xch = reinterpret_cast<float2 *>(base + L::xch(nsx));  // [TW_NX][4][TW_M]
  uint64_t *xfull = reinterpret_cast<uint64_t *>(base + L::bars(nsx));
  uint64_t *xfree = xfull + nsx;
  uint64_t *accf = xfree + nsx;  // 2 banks
  uint64_t *acce = accf + 2;     // 2 banks
  uint64_t *xready = acce + 2;   // TW_NX
  uint64_t *xdone = xready + TW_NX;
  uint64_t *drain = xdone + TW_NX;
  volatile int *abort = &s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = a.n;
  const int64_t ntiles = (n + TW_M - 1) / TW_M;
  const int my_tiles =
      (int)(blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);

  // exact centroid block in global memory (set-up kernel), norms and B here
  hpc_cent_smem cs;
  hpc_cent_bind(cs, a.gcent, D, a.k);
  cs.cmax = a.gmeta[0];
  cs.live = __float_as_int(a.gmeta[1]);
  for (int j = threadIdx.x; j < NP; j += TW_THREADS) cnv[j] = j < cs.kp ? cs.cnz[j].x : HPC_DEAD;
  for (int e = threadIdx.x; e < NP * D; e += TW_THREADS) {
    const int j = e / D, t = e - j * D;
    const float c = j < cs.kp ? cs.cm[j * CS + t] : 0.0f;  // -2c, zero padded
    const uint32_t off = (uint32_t)(t / Cfg::CK) * NP * Cfg::RB +
                         hpc_swz_offset((uint32_t)j, (uint32_t)(t % Cfg::CK) * 4u, Cfg::RB);
    *reinterpret_cast<float *>(bop + off) = c;  // exact: the MMA reads its TF32 part
  }
  hpc_fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < nsx; ++s) {
      hpc_mbar_init(&xfull[s], 1);
      hpc_mbar_init(&xfree[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      hpc_mbar_init(&accf[b], 1);
      hpc_mbar_init(&acce[b], Bk::READERS + 4);  // the folding warps, then the finishing ones
    }
    for (int b = 0; b < TW_NX; ++b) {
      hpc_mbar_init(&xready[b], 16);
      hpc_mbar_init(&xdone[b], 4);
    }
    hpc_mbar_init(drain, 1);
    s_abort = 0;
    hpc_fence_barrier_init();
  }
  if (warp == 1) hpc_tmem_alloc(&s_tmem, 512);
  hpc_tc_fence_before();
  __syncthreads();
  hpc_tc_fence_after();
  const uint32_t tmem = s_tmem;
  const bool run = cs.live > 0;
  if (!run && n > 0 && threadIdx.x == 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);

  // bank of part p of tile i, and how many times it was used before
  auto bank = [&](int i, int p) { return PARTS == 2 ? p : (i & 1); };
  auto bank_use = [&](int i) { return PARTS == 2 ? i : (i >> 1); };

  float fs_hi = 0.0f, fs_lo = 0.0f;
  if (run && warp == 0) {
    // ---- TMA producer: chunk u = i * NCH + ch goes to ring slot u % nsx ----
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      hpc_prefetch_tensormap(&tmap);
      for (int i = 0; i < my_tiles && ok; ++i) {
        const int64_t tg = blockIdx.x + (int64_t)i * gridDim.x;
        for (int ch = 0; ch < NCH; ++ch) {
          const int u = i * NCH + ch, s = u % nsx, ph = u / nsx;
          if (ph > 0 && !hpc_mbar_wait(&xfree[s], (ph - 1) & 1, abort, a.status, TW_WAIT_NS)) {
            ok = false;
            break;
          }
          hpc_mbar_arrive_expect_tx(&xfull[s], Cfg::CHUNK_BYTES);
          hpc_tma_load_2d(ring + (size_t)s * Cfg::CHUNK_BYTES, &tmap, &xfull[s], ch * Cfg::CK,
                          (int)(tg * TW_M));
          issued = u + 1;
        }
      }
      int no_abort = 0;
      for (int u = issued > nsx ? issued - nsx : 0; u < issued; ++u)
        hpc_mbar_wait(&xfull[u % nsx], (u / nsx) & 1, (volatile int *)&no_abort, a.status,
                      TW_DRAIN_NS);
    }
    __syncwarp();
  } else if (run && warp == 1) {
    // ---- MMA issuer: per tile and bank, all chunks; a ring slot is freed
    // after the tile's last bank has read it ----
    if (lane == 0) {
      constexpr int N = NP < 256 ? NP : 256;
      constexpr uint32_t idesc = hpc_umma_idesc(2u, 2u, N, TW_M);
      const uint32_t sbo = 8u * Cfg::RB;
      const uint32_t B = hpc_smem_u32(bop);
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        for (int p = 0; p < PARTS && ok; ++p) {
          const int bk = bank(i, p), v = bank_use(i);
          if (v > 0 && !hpc_mbar_wait(&acce[bk], (v - 1) & 1, abort, a.status, TW_WAIT_NS)) {
            ok = false;
            break;
          }
          const uint32_t dt = tmem + (uint32_t)(bk * 256);
          for (int ch = 0; ch < NCH; ++ch) {
            const int u = i * NCH + ch, s = u % nsx, ph = u / nsx;
            if (p == 0 && !hpc_mbar_wait(&xfull[s], ph & 1, abort, a.status, TW_WAIT_NS)) {
              ok = false;
              break;
            }
            hpc_tc_fence_after();
            const uint32_t A = hpc_smem_u32(ring + (size_t)s * Cfg::CHUNK_BYTES);
#pragma unroll
            for (int ks = 0; ks < Cfg::CK / 8; ++ks) {
              const uint64_t ad = hpc_umma_desc(A + (uint32_t)ks * 32u, 16u, sbo, Cfg::SWZ);
              const uint64_t bd =
                  hpc_umma_desc(B + (uint32_t)ch * (uint32_t)NP * Cfg::RB +
                                    (uint32_t)(p * 256) * Cfg::RB + (uint32_t)ks * 32u,
                                16u, sbo, Cfg::SWZ);
              hpc_mma_tf32(dt, ad, bd, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
            }
            if (p == PARTS - 1) hpc_mma_commit(&xfree[s]);
          }
          if (ok) hpc_mma_commit(&accf[bk]);
        }
      }
      hpc_mma_commit(drain);
      int no_abort = 0;
      hpc_mbar_wait(drain, 0, (volatile int *)&no_abort, a.status, TW_DRAIN_NS);
    }
    __syncwarp();
  } else if (run) {
    // ---- epilogue: warpgroup eg folds its columns of every tile and
    // finishes the tiles i with i mod 4 == eg ----
    const int eg = (warp - TW_EPI0) / 4, q = warp & 3;
    const int r_in = 32 * q + lane;
    const int col0 = eg * CPW;       // first column of this warpgroup
    const int part = col0 / 256;     // its bank within the tile
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    for (int i = 0; i < my_tiles; ++i) {
      const int bk = bank(i, part), v = bank_use(i);
      const int xb = i % TW_NX, xu = i / TW_NX;
      bool ok = wait_warp(&accf[bk], v & 1, abort, a.status, TW_WAIT_NS);
      // partial top-2 of this warpgroup's columns: two chains, merged
      float d1 = __int_as_float(0x7f7fffff), d2 = d1, e1 = d1, e2 = d1;
      if (ok) {
        hpc_tc_fence_after();
#pragma unroll
        for (int c = 0; c < CPW / 32; ++c) {
          const int cb = col0 + 32 * c;
          if (cb >= cs.kp) break;  // same for the whole warp
          float acc[32];
          hpc_tmem_ld32(tmem + lane_base + (uint32_t)(bk * 256 + cb - part * 256), acc);
#pragma unroll
          for (int jj = 0; jj < 32; jj += 4) {
            if (cb + jj >= cs.kp) break;
            const float4 cn = *reinterpret_cast<const float4 *>(cnv + cb + jj);
            const int j = cb + jj;
            float &t1 = (jj & 4) ? e1 : d1, &t2 = (jj & 4) ? e2 : d2;
            hpc_top2_fold4(t1, t2, hpc_key_b<IB>(cn.x + acc[jj], j),
                           hpc_key_b<IB>(cn.y + acc[jj + 1], j + 1),
                           hpc_key_b<IB>(cn.z + acc[jj + 2], j + 2),
                           hpc_key_b<IB>(cn.w + acc[jj + 3], j + 3));
          }
        }
        d2 = hpc_min3(d2, e2, fmaxf(d1, e1));
        d1 = fminf(d1, e1);
      }
      hpc_tc_fence_before();
      __syncwarp();
      if (lane == 0) hpc_mbar_arrive(&acce[bk]);  // this warp's columns are in registers
      if (!ok) break;
      // hand the partial to the finishing warpgroup
      if (xu > 0 && !wait_warp(&xdone[xb], (xu - 1) & 1, abort, a.status, TW_WAIT_NS)) break;
      xch[(xb * 4 + eg) * TW_M + r_in] = make_float2(d1, d2);
      __syncwarp();
      if (lane == 0) hpc_mbar_arrive(&xready[xb]);
      if ((i & 3) != eg) continue;

      // ---- finishing tile i: rows r_in = 32 q + lane.  This warpgroup
      // holds the tile's TMEM bank(s) until it has rescanned the rows whose
      // window holds a third candidate ----
      if (!wait_warp(&xready[xb], xu & 1, abort, a.status, TW_WAIT_NS)) break;
      {
        const float2 p0 = xch[(xb * 4 + 0) * TW_M + r_in];
        d1 = p0.x;
        d2 = p0.y;
#pragma unroll
        for (int e = 1; e < 4; ++e) {
          const float2 pe = xch[(xb * 4 + e) * TW_M + r_in];
          d2 = hpc_min3(d2, pe.y, fmaxf(d1, pe.x));
          d1 = fminf(d1, pe.x);
        }
      }
      __syncwarp();
      if (lane == 0) hpc_mbar_arrive(&xdone[xb]);
      const int64_t tg = blockIdx.x + (int64_t)i * gridDim.x;
      const int64_t row = tg * TW_M + r_in;
      bool valid = row < n;
      int j1 = min(__float_as_int(d1) & ((1 << IB) - 1), cs.kp - 1);
      const int j2 = min(__float_as_int(d2) & ((1 << IB) - 1), cs.kp - 1);
      const bool found = d1 < HPC_DEAD * 0.5f;
      if (!found) j1 = 0;
      // the row's exact quantities, per thread (rows of 256 / 512 bytes come
      // from L2, where the tile's TMA load left them)
      RowRef<D> xr;
      xr.g = a.X + (valid ? row : 0) * a.d;
      if constexpr (hpc_row_in_regs(D)) {
        if (valid) {
          hpc_load_row<D>(xr.x, xr.g, a.d);
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) xr.x[t] = 0.0f;
        }
      }
      const float nx = valid ? row_norm2<D>(xr) : 0.0f;
      float dd = valid ? b_direct<D, NP>(xr, bop, j1) : 0.0f;
      const float rad = sqrtf(nx) * 1.0001f + cs.cmax * 1.0001f;
      float win = 2.0f * 9.765625e-04f * rad * rad;  // 2E, E = 2^-10 (||x|| + max||c||)^2
      win += 1.0001f * ldexpf(1.0f, IB - 22) * (fabsf(d1) + fabsf(d2));  // keys
      const bool okf = found && isfinite(nx) && isfinite(win);
      if (valid && !okf) {
        hpc_status_set(a.status, HPC_ERR_NONFINITE);
        valid = false;
      }
      constexpr float rho = (float)(D + 3) * HPC_U32 * 1.001f;  // FP32 direct-form bound
      bool need64 = false, need_window = false;
      if (valid && !(d2 - d1 > win)) {
        // the two nearest by the tensor-core values, exactly; every other
        // centroid is at least ||x||^2 + d2 - E away
        const float ex2 = b_direct<D, NP>(xr, bop, j2);
        const float E = 0.5f * win;
        const float others = nx * (1.0f - (float)(D + 2) * HPC_U32 * 1.01f) + d2 - E -
                             4.0f * HPC_U32 * (nx + fabsf(d2) + E);
        const bool lo1 = dd < ex2 || (dd == ex2 && j1 < j2);
        const float lo = lo1 ? dd : ex2, hi = lo1 ? ex2 : dd;
        if (lo * (1.0f + rho) < others) {
          if (hi * (1.0f - rho) > lo * (1.0f + rho)) {
            if (!lo1) {
              j1 = j2;
              dd = ex2;
            }
          } else {
            need64 = true;
          }
        } else {
          need_window = true;
        }
      }
      if (__any_sync(0xffffffffu, need_window)) {
        // a third centroid may win: every candidate whose tensor-core value
        // lies within the window, exactly
        hpc_tc_fence_after();
        const float thr = d1 + win;
        float b1 = __int_as_float(0x7f800000), b2 = b1;
        int bj = j1;
#pragma unroll 1
        for (int p = 0; p < PARTS; ++p) {
          const uint32_t cbase = tmem + lane_base + (uint32_t)(bank(i, p) * 256);
#pragma unroll 1
          for (int c = 0; c < 256 / 32; ++c) {
            const int cb = p * 256 + 32 * c;
            if (cb >= cs.kp || cb >= NP) break;
            float acc[32];
            hpc_tmem_ld32(cbase + (uint32_t)(32 * c), acc);
#pragma unroll 4
            for (int jj = 0; jj < 32; ++jj) {
              const int j = cb + jj;
              if (need_window && j < cs.kp && cnv[j] + acc[jj] <= thr) {
                const float e = b_dist32<D, NP>(xr, bop, j);
                if (e < b1) {
                  b2 = b1;
                  b1 = e;
                  bj = j;
                } else {
                  b2 = fminf(b2, e);
                }
              }
            }
          }
        }
        if (need_window) {
          if (b2 - b1 > rho * (b1 + b2)) {
            j1 = bj;
            dd = b_direct<D, NP>(xr, bop, j1);
          } else {
            need64 = true;
          }
        }
      }
      hpc_tc_fence_before();
      __syncwarp();
      if (lane == 0)
        for (int p = 0; p < PARTS; ++p) hpc_mbar_arrive(&acce[bank(i, p)]);
      // unresolved by FP32: the warp rescores in FP64 (ties to the lowest index)
      unsigned m = __ballot_sync(0xffffffffu, need64);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int64_t ri = tg * TW_M + 32 * q + src;
        const int j = hpc_rescore_row<D>(a.X + ri * a.d, a.d, cs);
        if (lane == src && j != j1) {
          j1 = j;
          dd = b_direct<D, NP>(xr, bop, j1);
        }
      }
      if (valid && !isfinite(dd)) {
        hpc_status_set(a.status, HPC_ERR_NONFINITE);
        valid = false;
      }
      if (valid) {
        hpc_sum2_add(fs_hi, fs_lo, dd);
        if (a.labels) a.labels[row] = j1;
      }
    }
  }

  // ---- objective partial, last block reduces in a fixed order ----
  const double bsum = hpc_block_sum((double)fs_hi + (double)fs_lo, s_dsum);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = bsum;
    __threadfence();
    const unsigned prev = atomicAdd(a.done_count, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    const double f = hpc_block_sum_array(a.part, (int)gridDim.x, s_dsum);
    if (threadIdx.x == 0) {
      *a.f_out = (!run && n > 0) ? __longlong_as_double(0x7ff8000000000000ll) : f;
      *a.done_count = 0u;
    }
  }
  hpc_tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    hpc_tc_fence_after();
    hpc_tmem_dealloc(tmem, 512);
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
int tw_launch_t(const hpc_launch &Lc, const ObjArgsHost &h) {
  using Cfg = TwCfg<D>;
  using L = TwSmem<D, NP>;
  auto kern = tw_objective_kernel<D, NP, IB>;
  if (!h.cent_scratch || h.cent_scratch_bytes < (int64_t)hpc_tc_wide_scratch_bytes(D, h.k))
    return HPC_ERR_UNSUPPORTED;
  int nsx = TW_MAX_RING;
  while (nsx > Cfg::NCH && L::total(nsx) > (size_t)Lc.smem_optin) --nsx;
  if (L::total(nsx) > (size_t)Lc.smem_optin) return HPC_ERR_UNSUPPORTED;
  // at least 120 KB, so that no second block (and its 512-column TMEM
  // allocation) can share an SM
  size_t smem = L::total(nsx);
  if (smem < 120 * 1024) smem = 120 * 1024;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return HPC_ERR_UNSUPPORTED;
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)h.d, (cuuint64_t)h.n};
  cuuint64_t gstride[1] = {(cuuint64_t)h.d * 4};
  cuuint32_t box[2] = {(cuuint32_t)Cfg::CK, (cuuint32_t)TW_M};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle swz =
      Cfg::RB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(h.X), gdim, gstride, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HPC_ERR_CUDA;
  unsigned char *gcent = h.cent_scratch;
  float *gmeta = reinterpret_cast<float *>(gcent + ((hpc_cent_smem_bytes(D, h.k) + 255) & ~(size_t)255));
  tw_prep_kernel<D><<<1, 256, 0, Lc.stream>>>(h.C, h.deg, h.k, h.d, gcent, gmeta);
  if (cudaGetLastError() != cudaSuccess) return HPC_ERR_CUDA;
  const int64_t ntiles = (h.n + TW_M - 1) / TW_M;
  int64_t G = Lc.num_sms;
  if (G > ntiles) G = ntiles;
  if (G < 1) G = 1;
  if (G > h.max_blocks) G = h.max_blocks;
  TwArgs a;
  a.n = h.n;
  a.d = h.d;
  a.k = h.k;
  a.nsx = nsx;
  a.X = h.X;
  a.gcent = gcent;
  a.gmeta = gmeta;
  a.f_out = h.f_out;
  a.labels = h.labels;
  a.status = h.status;
  a.part = h.part;
  a.done_count = h.done_count;
  kern<<<(unsigned)G, TW_THREADS, smem, Lc.stream>>>(map, a);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

}  // namespace

size_t hpc_tc_wide_scratch_bytes(int d, int k) {
  const int D = d <= 16 ? 16 : d <= 32 ? 32 : d <= 64 ? 64 : 128;
  return ((hpc_cent_smem_bytes(D, k) + 255) & ~(size_t)255) + 256;
}

bool hpc_tc_wide_supported(int d, int k, int64_t n) {
  if (n < 1 || k <= 128) return false;
  if (d == 16 || d == 32 || d == 64) return k <= 512;
  return d == 128 && k <= 256;
}

// (value, index) keys with 8 index bits for k <= 256, 9 for k <= 512 (the
// keys' error, at most 2^-14 relative, is far inside the TF32 window)
int hpc_tc_wide_launch(const hpc_launch &L, const ObjArgsHost &h) {
  if (!hpc_tc_wide_supported(h.d, h.k, h.n)) return HPC_ERR_UNSUPPORTED;
  const bool w512 = h.k > 256;
  switch (h.d) {
    case 16: return w512 ? tw_launch_t<16, 512, 9>(L, h) : tw_launch_t<16, 256, 8>(L, h);
    case 32: return w512 ? tw_launch_t<32, 512, 9>(L, h) : tw_launch_t<32, 256, 8>(L, h);
    case 64: return w512 ? tw_launch_t<64, 512, 9>(L, h) : tw_launch_t<64, 256, 8>(L, h);
    default: return tw_launch_t<128, 256, 8>(L, h);
  }
}
