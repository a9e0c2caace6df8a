// Nearest-centroid search with the x.c contraction on the tensor cores in
// split BF16, for rows of 64 or 128 floats and up to 512 (d = 64) or 256
// (d = 128) centroids: Lloyd's iterations on a sample (Algorithm 1, with the
// stop rule of Section 6.5) and the full-data objective (Eq. 1).
//
// Search value of centroid j for row x: v_j = ||c_j||^2 + x.c'_j, c' = -2c.
// Both operands are split into two BF16 parts, x = x_h + x_l + r_x and
// c' = c_h + c_l + r_c (x_h = bf16(x), x_l = bf16(x - x_h); |r| <= 2^-18 of
// the value), and the tensor cores form three exact BF16 products per K step
// in FP32: x_h.c_h + x_h.c_l + x_l.c_h.  The dropped terms x_l c_l, r_x c'
// and x r_c stay below 3.01 * 2^-18 |x_t| |c'_t| per coordinate, and FP32
// accumulation over the 3 d products adds at most 3 d 2^-23 of
// sum_t |x_t| |c'_t| <= ||x|| ||c'|| = 2 ||x|| ||c||; with
// (||x|| + max||c||)^2 >= 4 ||x|| ||c||, every computed v_j lies within
// 2^-15.8 (||x|| + max||c||)^2 of the exact one at d = 64 (2^-14.9 at
// d = 128).  The kernels use E = 2^-14 (||x|| + max||c||)^2.  A row whose
// top-2 margin exceeds 2E (plus the packed keys' 2^(IB-22) (|k1| + |k2|)) has
// the exact nearest centroid; otherwise its two candidates are computed
// exactly (FP32 direct form), every other centroid being at least
// ||x||^2 + v3 - E away (v3 the third smallest computed value: the epilogue
// keeps three per row), and rows that remain open are settled against every
// centroid (FP32 direct form, then FP64 in the oracle's operation order,
// ties to the lowest index) after the CTA's pass, by all its warps.
//
// Data path per 128-row tile (one persistent CTA per SM):
//   warp 0 (TMEM owner, MMA issuer, one thread): 3 d / 16 x 3 kind::f16
//     MMAs per 256-column bank against B = (c_h | c_l) resident in shared
//     memory, the A operand from one of two shared-memory stages; TMEM holds
//     two banks (two tiles in flight for up to 256 centroids, the two halves
//     of one tile for up to 512); asks the L2 for the rows of the tile four
//     tiles ahead (bulk prefetch);
//   warps 1-16 (four fold warpgroups): warpgroup e folds a quarter of a
//     tile's columns into the three smallest (value, index) keys per row
//     (7 to 9 index bits) and leaves them in a rotating exchange buffer;
//     each warp then converts eight rows of a later tile: coalesced 16-byte
//     loads of the FP32 rows (issued before the fold, so that their latency
//     hides behind it), split into x_h | x_l and written as the MMA's A
//     operand (K-major, 128-byte swizzle), so that the conversion is spread
//     over sixteen warps;
//   warps 17-24 (two finisher warpgroups): warpgroup f takes every second
//     tile, merges the four partial top-3 of each row and finishes the row
//     (exact distance, margin test, exact stages, objective, labels, and in
//     Lloyd the centroid sums), so that the fold warps, which release the
//     TMEM banks, never wait on a row's global loads.
//
// Lloyd's centroid sums are kept incrementally: every coordinate goes on the
// exact 64-bit fixed-point grid 2^-Fs of the CUDA-core kernel, the first
// assignment adds every row, and each later one adds only the rows whose
// label changed (to the new centroid) and takes them away from the old one;
// integer sums make that equal to summing every row again, in any order.
// An iteration: the pipeline over the CTA's tiles, a bounded barrier of the
// task's CTAs, the stop test and the new means (every CTA, identical), a
// second barrier (every CTA has read the sums before any adds to them
// again).  Every mbarrier wait is bounded (a wait that runs out records
// HPC_ERR_TIMEOUT and every role stops); in-flight MMAs are drained before
// TMEM is freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "assign.cuh"
#include "kernels.h"
#include "round.cuh"
#include "tc.cuh"
#include "tc_rows.cuh"

namespace {

constexpr int TB_M = 128;
constexpr int TB_MMAW = 0;                       // TMEM owner and MMA issuer
constexpr int TB_EPI0 = 1;                       // first fold warp (four warpgroups)
constexpr int TB_NFOLD = 16;                     // fold warps
constexpr int TB_FIN0 = TB_EPI0 + TB_NFOLD;      // first finisher warp (two warpgroups)
constexpr int TB_NFIN = 2;                       // finisher warpgroups
constexpr int TB_THREADS = (TB_FIN0 + 4 * TB_NFIN) * 32;  // 800
constexpr int TB_PREFETCH = 4;                   // tiles the L2 is asked for ahead
constexpr size_t TB_SMEM_MAX = 226 * 1024;       // dynamic shared memory of one CTA (static: < 1 KB)
constexpr uint64_t TB_WAIT_NS = 2000000000ull;
constexpr uint64_t TB_DRAIN_NS = 500000000ull;
constexpr float TB_E_REL = 6.103515625e-05f;     // 2^-14

template <int D, int NP>
struct TbCfg {
  static_assert(D == 64 || D == 128, "rows of 64 or 128 floats");
  static_assert(NP == 128 || NP == 256 || NP == 512, "128, 256 or 512 columns");
  static constexpr uint32_t ATILE = TB_M * D * 2;  // one BF16 part of a row tile
  static constexpr uint32_t BPART = NP * D * 2;    // one BF16 part of B
  static constexpr int PARTS = NP > 256 ? 2 : 1;   // TMEM banks per tile
  static constexpr int BANKW = NP > 256 ? 256 : NP;
  static constexpr int TCOLS = NP > 256 ? 512 : 2 * NP;
  static constexpr int CPW = NP / 4;               // columns per epilogue warpgroup
  static constexpr int READERS = NP > 256 ? 8 : 16;
  static constexpr int IB = NP == 512 ? 9 : NP == 256 ? 8 : 7;
  // what every layout holds besides the A stages and the exchange buffers:
  // B, norms, flags, barriers (at most 32), alignment slack
  static constexpr size_t FIXED = 2 * (size_t)BPART + (size_t)NP * 4 + 512 + 32 * 8 + 1024;
  static constexpr size_t XBUF = 4 * (size_t)TB_M * 12;  // one exchange buffer
  static constexpr int NSTAGE = FIXED + 4 * (size_t)ATILE + 2 * XBUF <= TB_SMEM_MAX ? 2 : 1;
  static constexpr int NX =
      FIXED + (size_t)NSTAGE * 2 * ATILE + 4 * XBUF <= TB_SMEM_MAX ? 4 : 2;
  static constexpr size_t AOP = 2 * (size_t)BPART;
  static constexpr size_t CN = AOP + (size_t)NSTAGE * 2 * ATILE;
  static constexpr size_t XCH = CN + (size_t)NP * 4;
  static constexpr size_t DEADF = XCH + (size_t)NX * XBUF;
  static constexpr size_t BARS = DEADF + 512;
  static constexpr int NBARS = 2 * NSTAGE + 4 + 2 * NX + 1;
  static_assert(NBARS <= 32, "barrier room");
  static constexpr size_t TOTAL = BARS + NBARS * 8 + 1024;
  static_assert(TOTAL <= TB_SMEM_MAX, "shared memory of one CTA");
};

// Shared-memory views of one CTA.
struct TbSm {
  unsigned char *bh, *bl, *a;
  float *cn;
  float *xch;  // [NX][4 warpgroups][TB_M rows][3 keys]
  uint8_t *dead;
  uint64_t *afull, *afree, *accf, *acce, *xready, *xdone, *drain;
  volatile int *abort;
  uint32_t tmem;
};

template <int D, int NP>
__device__ __forceinline__ TbSm tb_bind(unsigned char *base, volatile int *abort) {
  using Cfg = TbCfg<D, NP>;
  TbSm m;
  m.bh = base;
  m.bl = base + Cfg::BPART;
  m.a = base + Cfg::AOP;
  m.cn = reinterpret_cast<float *>(base + Cfg::CN);
  m.xch = reinterpret_cast<float *>(base + Cfg::XCH);
  m.dead = base + Cfg::DEADF;
  uint64_t *b = reinterpret_cast<uint64_t *>(base + Cfg::BARS);
  m.afull = b;
  m.afree = b + Cfg::NSTAGE;
  m.accf = m.afree + Cfg::NSTAGE;
  m.acce = m.accf + 2;
  m.xready = m.acce + 2;
  m.xdone = m.xready + Cfg::NX;
  m.drain = m.xdone + Cfg::NX;
  m.abort = abort;
  m.tmem = 0;
  return m;
}

template <int D, int NP>
__device__ __forceinline__ void tb_init_barriers(const TbSm &m) {
  using Cfg = TbCfg<D, NP>;
  for (int s = 0; s < Cfg::NSTAGE; ++s) {
    hpc_mbar_init(&m.afull[s], TB_NFOLD);
    hpc_mbar_init(&m.afree[s], 1);
  }
  for (int b = 0; b < 2; ++b) {
    hpc_mbar_init(&m.accf[b], 1);
    hpc_mbar_init(&m.acce[b], Cfg::READERS);
  }
  for (int b = 0; b < Cfg::NX; ++b) {
    hpc_mbar_init(&m.xready[b], 16);  // the fold warps
    hpc_mbar_init(&m.xdone[b], 4);    // the finisher warpgroup's warps
  }
  hpc_mbar_init(m.drain, 1);
  hpc_fence_barrier_init();
}

__device__ __forceinline__ uint32_t tb_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<uint32_t *>(&v);
}

// Byte offset of element t (a multiple of 2) of row r in a K-major BF16
// operand of `rows` rows: 64-element chunks of rows x 128 bytes, 128-byte
// swizzle inside each.
__device__ __forceinline__ uint32_t tb_koff(uint32_t r, uint32_t t, uint32_t rows) {
  return (t >> 6) * rows * 128u + hpc_swz_offset(r, (t & 63u) * 2u, 128u);
}

// The split c' = -2c = c_h + c_l of centroid row j's values v[] at dims
// t0 .. t0 + PER - 1 into B (shared memory), PER even.
template <int PER, int NP>
__device__ __forceinline__ void tb_store_b(const TbSm &m, int j, int t0, const float (&c)[PER]) {
#pragma unroll
  for (int u = 0; u < PER; u += 2) {
    const float a0 = -2.0f * c[u], a1 = -2.0f * c[u + 1];
    const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a0 - hf.x, a1 - hf.y);
    const uint32_t off = tb_koff((uint32_t)j, (uint32_t)(t0 + u), NP);
    *reinterpret_cast<uint32_t *>(m.bh + off) = tb_bits(h);
    *reinterpret_cast<uint32_t *>(m.bl + off) = tb_bits(l);
  }
}

// Row source of the pipeline: rows [0, nrows) of `rows` (stride D floats);
// the i-th tile of this CTA is tile0 + i * tstep.
struct TbRows {
  const float *rows;
  int64_t nrows;
  int64_t tile0, tstep;
  int ntiles;
};

// ---- row conversion (by the fold warps) ---------------------------------------
// Fold warp wf (0 .. 15) converts rows 8 wf .. 8 wf + 7 of a row tile: it
// loads them from global memory (the L2 holds them: the MMA thread asks for
// every tile TB_PREFETCH tiles ahead) and splits them into x_h | x_l (K-major,
// 128-byte swizzle) in the tile's A stage.  Rows past the end are zeros.
template <int D>
struct TbConv {
  static constexpr int F4 = D / 4;               // float4 per row
  static constexpr int PER = 8 * F4 / 32;        // float4 per lane per tile (4 or 8)
  static constexpr int LP = PER < 4 ? PER : 4;   // loaded ahead of the fold
};

template <int D, int U0, int U1>
__device__ __forceinline__ void tb_rows_load(const TbRows &R, int64_t row0, int wf, int lane,
                                             float4 (&v)[U1 - U0]) {
  constexpr int F4 = TbConv<D>::F4;
#pragma unroll
  for (int u = U0; u < U1; ++u) {
    const int e = u * 32 + lane;
    const int64_t row = row0 + 8 * wf + e / F4;
    v[u - U0] = row < R.nrows ? __ldg(reinterpret_cast<const float4 *>(R.rows + row * D) + e % F4)
                              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

template <int D, int U0, int U1>
__device__ __forceinline__ void tb_rows_store(unsigned char *ah, unsigned char *al, int wf, int lane,
                                              const float4 (&v)[U1 - U0]) {
  constexpr int F4 = TbConv<D>::F4;
#pragma unroll
  for (int u = U0; u < U1; ++u) {
    const int e = u * 32 + lane;
    const int r = 8 * wf + e / F4;
    const int t = 4 * (e % F4);
    const float4 x = v[u - U0];
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(x.x, x.y);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(x.z, x.w);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(x.x - f01.x, x.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(x.z - f23.x, x.w - f23.y);
    const uint32_t off = tb_koff((uint32_t)r, (uint32_t)t, TB_M);
    *reinterpret_cast<uint2 *>(ah + off) = make_uint2(tb_bits(h01), tb_bits(h23));
    *reinterpret_cast<uint2 *>(al + off) = make_uint2(tb_bits(l01), tb_bits(l23));
  }
}

// First row of the CTA's i-th tile.
__device__ __forceinline__ int64_t tb_tile_row0(const TbRows &R, int i) {
  return (R.tile0 + (int64_t)i * R.tstep) * TB_M;
}

// This warp's rows of tile i (sequence number g): waits until the MMA has
// released the stage, writes the first LP float4 per lane from v (loaded
// earlier) and the rest from memory, and marks the warp's part ready.
template <int D, int NP>
__device__ __forceinline__ bool tb_convert(const TbSm &m, const TbRows &R, int i, uint32_t g, int wf,
                                           const float4 (&v)[TbConv<D>::LP], int *status) {
  using Cfg = TbCfg<D, NP>;
  using Cv = TbConv<D>;
  const int lane = threadIdx.x & 31;
  const int st = (int)(g % Cfg::NSTAGE);
  const uint32_t use = g / Cfg::NSTAGE;
  if (use > 0 && !wait_warp(&m.afree[st], (use - 1) & 1u, m.abort, status, TB_WAIT_NS)) return false;
  unsigned char *ah = m.a + (size_t)st * 2 * Cfg::ATILE;
  unsigned char *al = ah + Cfg::ATILE;
  tb_rows_store<D, 0, Cv::LP>(ah, al, wf, lane, v);
  if constexpr (Cv::PER > Cv::LP) {
    float4 w[Cv::PER - Cv::LP];
    tb_rows_load<D, Cv::LP, Cv::PER>(R, tb_tile_row0(R, i), wf, lane, w);
    tb_rows_store<D, Cv::LP, Cv::PER>(ah, al, wf, lane, w);
  }
  hpc_fence_proxy_async();  // the stage's generic writes, visible to the tensor core
  __syncwarp();
  if (lane == 0) hpc_mbar_arrive(&m.afull[st]);
  return true;
}

// ---- MMA issuer (warp 0, one thread) ------------------------------------------
// Also asks the L2 for the rows of the tile TB_PREFETCH tiles ahead.
template <int D, int NP>
__device__ __forceinline__ void tb_mma(const TbSm &m, const TbRows &R, uint32_t gbase, int *status) {
  using Cfg = TbCfg<D, NP>;
  constexpr uint32_t idesc = hpc_umma_idesc(1u, 1u, Cfg::BANKW, TB_M);
  constexpr uint32_t SBO = 8u * 128u;
  const uint32_t BH = hpc_smem_u32(m.bh), BL = hpc_smem_u32(m.bl);
  auto prefetch = [&](int i) {
    if (i >= R.ntiles) return;
    const int64_t p0 = tb_tile_row0(R, i);
    const int64_t nr = min((int64_t)TB_M, R.nrows - p0);
    if (nr > 0) hpc_prefetch_l2_bulk(R.rows + p0 * D, (uint32_t)(nr * D * 4));
  };
  for (int i = Cfg::NSTAGE; i < TB_PREFETCH; ++i) prefetch(i);
  for (int i = 0; i < R.ntiles; ++i) {
    const uint32_t g = gbase + (uint32_t)i;
    prefetch(i + TB_PREFETCH);
    const int st = (int)(g % Cfg::NSTAGE);
    const uint32_t use = g / Cfg::NSTAGE;
    if (!hpc_mbar_wait(&m.afull[st], use & 1u, m.abort, status, TB_WAIT_NS)) break;
    hpc_tc_fence_after();
    const uint32_t AH = hpc_smem_u32(m.a + (size_t)st * 2 * Cfg::ATILE);
    const uint32_t AL = AH + Cfg::ATILE;
    bool ok = true;
    for (int p = 0; p < Cfg::PARTS; ++p) {
      const int bk = Cfg::PARTS == 2 ? p : (int)(g & 1u);
      const uint32_t v = Cfg::PARTS == 2 ? g : (g >> 1);
      if (v > 0 && !hpc_mbar_wait(&m.acce[bk], (v - 1) & 1u, m.abort, status, TB_WAIT_NS)) {
        ok = false;
        break;
      }
      hpc_tc_fence_after();
      const uint32_t dt = m.tmem + (uint32_t)(bk * Cfg::BANKW);
      const uint32_t boff = (uint32_t)(p * 256) * 128u;
#pragma unroll
      for (int ks = 0; ks < D / 16; ++ks) {
        const uint32_t ka = (uint32_t)(ks >> 2) * TB_M * 128u + (uint32_t)(ks & 3) * 32u;
        const uint32_t kb = (uint32_t)(ks >> 2) * NP * 128u + boff + (uint32_t)(ks & 3) * 32u;
        const uint64_t ah = hpc_umma_desc(AH + ka, 16u, SBO, 2u);
        const uint64_t al = hpc_umma_desc(AL + ka, 16u, SBO, 2u);
        const uint64_t bh = hpc_umma_desc(BH + kb, 16u, SBO, 2u);
        const uint64_t bl = hpc_umma_desc(BL + kb, 16u, SBO, 2u);
        hpc_mma_bf16(dt, ah, bh, idesc, ks > 0 ? 1u : 0u);
        hpc_mma_bf16(dt, ah, bl, idesc, 1u);
        hpc_mma_bf16(dt, al, bh, idesc, 1u);
      }
      hpc_mma_commit(&m.accf[bk]);
    }
    hpc_mma_commit(&m.afree[st]);
    if (!ok) break;
  }
}

// Drains the MMA issuer's work before TMEM is freed (one thread).
__device__ __forceinline__ void tb_drain(const TbSm &m, uint32_t drain_use, int *status) {
  int no_abort = 0;
  hpc_mma_commit(m.drain);
  hpc_mbar_wait(m.drain, drain_use & 1u, (volatile int *)&no_abort, status, TB_DRAIN_NS);
}

// Exact centroid block (hpc_cent_smem layout: -2c rows of hpc_cstride(D)
// floats, then (||c||^2, 0) pairs) in global memory.
template <int D>
__device__ __forceinline__ hpc_cent_smem tb_gcs(float *gcent, int k, float cmax, int live) {
  hpc_cent_smem cs;
  hpc_cent_bind(cs, reinterpret_cast<unsigned char *>(gcent), D, k);
  cs.cmax = cmax;
  cs.live = live;
  return cs;
}

// The three smallest of two sorted triples (t1 <= t2 <= t3 and r1 <= r2 <=
// r3), into t: the k-th smallest of the union is the smallest over the
// splits i + j = k of max(t_i, r_j).
__device__ __forceinline__ void tb_merge3(float &t1, float &t2, float &t3, float r1, float r2,
                                          float r3) {
  const float u3 = fminf(hpc_min3(t3, r3, fmaxf(t2, r1)), fmaxf(t1, r2));
  const float u2 = hpc_min3(t2, r2, fmaxf(t1, r1));
  t1 = fminf(t1, r1);
  t2 = u2;
  t3 = u3;
}

// Folds four (value, index) keys into the running three smallest: the four
// sorted by a 2 x 2 merge (the three smallest kept), then merged.
__device__ __forceinline__ void tb_fold4_top3(float &t1, float &t2, float &t3, float k0, float k1,
                                              float k2, float k3) {
  const float a = fminf(k0, k1), b = fmaxf(k0, k1), c = fminf(k2, k3), e = fmaxf(k2, k3);
  const float M = fmaxf(a, c), mb = fminf(b, e);
  tb_merge3(t1, t2, t3, fminf(a, c), fminf(M, mb), fmaxf(M, mb));
}

// ---- fold warps (warps 1-16) -------------------------------------------------
// Warpgroup e folds columns [e NP/4, (e+1) NP/4) of every tile into the
// three smallest (value, index) keys per row and leaves them in the tile's
// exchange buffer (the finishers merge the four).  Each fold warp also
// converts its eight rows of the tile NSTAGE tiles ahead into that tile's A
// stage (the first NSTAGE tiles before the loop): with two stages after the
// fold, so that the accumulator bank is released first; with one stage
// before it, so that the next tile's MMAs run during the fold.
template <int D, int NP>
__device__ __forceinline__ void tb_fold(const TbSm &m, const TbRows &R, uint32_t gbase, int kp,
                                        int *status) {
  using Cfg = TbCfg<D, NP>;
  using Cv = TbConv<D>;
  constexpr int IB = Cfg::IB;
  constexpr int NS = Cfg::NSTAGE;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wf = warp - TB_EPI0;
  const int e = wf >> 2, q = warp & 3;
  const int r_in = 32 * q + lane;
  const int col0 = e * Cfg::CPW;
  const int part = Cfg::PARTS == 2 ? col0 / 256 : 0;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  for (int i = 0; i < min(NS, R.ntiles); ++i) {
    float4 v[Cv::LP];
    tb_rows_load<D, 0, Cv::LP>(R, tb_tile_row0(R, i), wf, lane, v);
    if (!tb_convert<D, NP>(m, R, i, gbase + (uint32_t)i, wf, v, status)) return;
  }
  for (int i = 0; i < R.ntiles; ++i) {
    const uint32_t g = gbase + (uint32_t)i;
    const int bk = Cfg::PARTS == 2 ? part : (int)(g & 1u);
    const uint32_t v = Cfg::PARTS == 2 ? g : (g >> 1);
    const int xb = (int)(g % Cfg::NX);
    const uint32_t xu = g / Cfg::NX;
    const bool ahead = i + NS < R.ntiles;
    float4 rows_ahead[Cv::LP];
    if (ahead) tb_rows_load<D, 0, Cv::LP>(R, tb_tile_row0(R, i + NS), wf, lane, rows_ahead);
    bool ok = wait_warp(&m.accf[bk], v & 1u, m.abort, status, TB_WAIT_NS);
    if constexpr (NS == 1) {
      if (ok && ahead) ok = tb_convert<D, NP>(m, R, i + NS, g + NS, wf, rows_ahead, status);
    }
    // the three smallest keys of this warpgroup's columns, as two chains
    float d1 = __int_as_float(0x7f7fffff), d2 = d1, d3 = d1, e1 = d1, e2 = d1, e3 = d1;
    if (ok) {
      hpc_tc_fence_after();
      // keys carry the column's index within this warpgroup's range (a
      // constant of the unrolled code: one logic instruction a key); the
      // finishers add the range's first column
#pragma unroll
      for (int c = 0; c < Cfg::CPW / 16; ++c) {
        const int cb = col0 + 16 * c;
        if (cb >= kp) continue;  // the same for the whole warp
        float acc[16];
        hpc_tmem_ld16(m.tmem + lane_base + (uint32_t)(bk * Cfg::BANKW + cb - part * 256), acc);
#pragma unroll
        for (int jj = 0; jj < 16; jj += 8) {
          const float4 ca = *reinterpret_cast<const float4 *>(m.cn + cb + jj);
          const float4 cc = *reinterpret_cast<const float4 *>(m.cn + cb + jj + 4);
          const int j = 16 * c + jj;
          tb_fold4_top3(d1, d2, d3, hpc_key_b<IB>(ca.x + acc[jj], j),
                        hpc_key_b<IB>(ca.y + acc[jj + 1], j + 1),
                        hpc_key_b<IB>(ca.z + acc[jj + 2], j + 2),
                        hpc_key_b<IB>(ca.w + acc[jj + 3], j + 3));
          tb_fold4_top3(e1, e2, e3, hpc_key_b<IB>(cc.x + acc[jj + 4], j + 4),
                        hpc_key_b<IB>(cc.y + acc[jj + 5], j + 5),
                        hpc_key_b<IB>(cc.z + acc[jj + 6], j + 6),
                        hpc_key_b<IB>(cc.w + acc[jj + 7], j + 7));
        }
      }
      tb_merge3(d1, d2, d3, e1, e2, e3);
    }
    hpc_tc_fence_before();
    __syncwarp();
    if (lane == 0) hpc_mbar_arrive(&m.acce[bk]);  // this warp's columns are in registers
    if (!ok) break;
    if constexpr (NS > 1) {
      if (ahead && !tb_convert<D, NP>(m, R, i + NS, g + NS, wf, rows_ahead, status)) break;
    }
    if (xu > 0 && !wait_warp(&m.xdone[xb], (xu - 1) & 1u, m.abort, status, TB_WAIT_NS)) break;
    {
      float *xp = m.xch + ((size_t)(xb * 4 + e) * TB_M + r_in) * 3;
      xp[0] = d1;
      xp[1] = d2;
      xp[2] = d3;
    }
    __syncwarp();
    if (lane == 0) hpc_mbar_arrive(&m.xready[xb]);
  }
}

// ---- finishers (warps 17-24) ----------------------------------------------------
// Finisher warpgroup f takes the tiles g with g mod TB_NFIN == f: merges the
// four partial top-3 of each row, frees the exchange buffer, and calls
// `fin(row0w, row, valid, j1, j2, d1, d2, v3)` with the whole warp (lane l
// holds row 32 q + l of the tile).
template <int D, int NP, typename Fin>
__device__ __forceinline__ void tb_finish(const TbSm &m, const TbRows &R, uint32_t gbase, int kp,
                                          int *status, Fin fin) {
  using Cfg = TbCfg<D, NP>;
  constexpr int IB = Cfg::IB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int f = (warp - TB_FIN0) >> 2, q = warp & 3;
  const int r_in = 32 * q + lane;
  for (int i = 0; i < R.ntiles; ++i) {
    const uint32_t g = gbase + (uint32_t)i;
    if ((int)(g % TB_NFIN) != f) continue;
    const int xb = (int)(g % Cfg::NX);
    const uint32_t xu = g / Cfg::NX;
    if (!wait_warp(&m.xready[xb], xu & 1u, m.abort, status, TB_WAIT_NS)) break;
    // the three smallest keys of the tile's row: every centroid but the two
    // best has a key of at least the third (each warpgroup kept its three)
    float d1, d2, lo3;
    {
      const float *xp = m.xch + ((size_t)(xb * 4) * TB_M + r_in) * 3;
      d1 = xp[0];
      d2 = xp[1];
      lo3 = xp[2];
#pragma unroll
      for (int o = 1; o < 4; ++o) {  // warpgroup o's keys: its first column added
        const float *xo = xp + (size_t)o * TB_M * 3;
        const int c0 = o * Cfg::CPW;
        tb_merge3(d1, d2, lo3, __int_as_float(__float_as_int(xo[0]) | c0),
                  __int_as_float(__float_as_int(xo[1]) | c0), __int_as_float(__float_as_int(xo[2]) | c0));
      }
    }
    __syncwarp();
    if (lane == 0) hpc_mbar_arrive(&m.xdone[xb]);
    const int64_t row0 = (R.tile0 + (int64_t)i * R.tstep) * TB_M;
    const int64_t row = row0 + r_in;
    const bool valid = row < R.nrows;
    const int j1 = min(__float_as_int(d1) & ((1 << IB) - 1), kp - 1);
    const int j2 = min(__float_as_int(d2) & ((1 << IB) - 1), kp - 1);
    fin(row0 + 32 * q, row, valid, j1, j2, d1, d2, lo3);
  }
}

// The objective's FP32 direct-form distance from row x to the centroid whose
// -2c row is cm (two interleaved partial sums, relative error <= (D/2 + 4) u),
// one thread.  Centroid rows are read through L2 (__ldcg): the exact block is
// rewritten between Lloyd iterations.
template <int D>
__device__ __forceinline__ float tb_direct(const float *__restrict__ x, const float *cm) {
  float2 sd = make_float2(0.0f, 0.0f);
  const float2 half = make_float2(0.5f, 0.5f);
#pragma unroll 4
  for (int t = 0; t < D; t += 4) {
    const float4 xv = __ldg(reinterpret_cast<const float4 *>(x + t));
    const float4 cv = __ldcg(reinterpret_cast<const float4 *>(cm + t));
    const float2 e01 = hpc_fma2(half, make_float2(cv.x, cv.y), make_float2(xv.x, xv.y));
    const float2 e23 = hpc_fma2(half, make_float2(cv.z, cv.w), make_float2(xv.z, xv.w));
    sd = hpc_fma2(e01, e01, sd);
    sd = hpc_fma2(e23, e23, sd);
  }
  return sd.x + sd.y;
}

// Exact assignment of one row by the whole warp (every lane passes the same
// row).  FP32 direct form for every centroid: the warp's four 8-lane groups
// take centroids 4i + g, and lane l of a group the dimensions 4l + 32v ..
// 4l + 32v + 3, so that a group reads a centroid row in coalesced 128-byte
// pieces; U centroids per group are loaded before any is used.  The group's
// partial sums meet by shuffles (every lane of the group gets the same
// value: the butterfly adds the same pairs); summed in any order, the D
// nonnegative terms carry the relative bound (D + 3) u.  If the two best are
// not separated by it, FP64 in the oracle's operation order for the
// centroids whose FP32 value lies within the bound of the best (no other one
// can win), ties to the lowest index.  Every lane returns the same index.
// Counts the FP64 rows in *stats.
template <int D>
__device__ __forceinline__ float tb_group_dist(const float4 (&xv)[D / 32], const float4 (&cv)[D / 32]) {
  float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
  for (int v = 0; v < D / 32; ++v) {
    const float dx = __fmaf_rn(0.5f, cv[v].x, xv[v].x), dy = __fmaf_rn(0.5f, cv[v].y, xv[v].y);
    const float dz = __fmaf_rn(0.5f, cv[v].z, xv[v].z), dw = __fmaf_rn(0.5f, cv[v].w, xv[v].w);
    s0 = __fmaf_rn(dx, dx, s0);
    s1 = __fmaf_rn(dy, dy, s1);
    s0 = __fmaf_rn(dz, dz, s0);
    s1 = __fmaf_rn(dw, dw, s1);
  }
  float s = s0 + s1;
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 4);
  return s;
}

template <int D>
__device__ __forceinline__ int tb_rescore(const float *__restrict__ x, const hpc_cent_smem &cs,
                                          unsigned long long *stats) {
  constexpr int CS = hpc_cstride(D);
  constexpr int V = D / 32;           // float4 of a centroid row per lane
  constexpr int U = D == 64 ? 4 : 2;  // centroids per group in flight
  const int lane = threadIdx.x & 31, g = lane >> 3, sl = lane & 7;
  const int kp = cs.kp;
  float4 xv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) xv[v] = __ldg(reinterpret_cast<const float4 *>(x + 4 * sl + 32 * v));
  float a1 = __int_as_float(0x7f800000), a2 = a1;
  int ja = 0x7fffffff;
#pragma unroll 1
  for (int j0 = 0; j0 < kp; j0 += 4 * U) {
    float4 cv[U][V];
    float nz[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = min(j0 + 4 * u + g, kp - 1);
      const float *cm = cs.cm + (size_t)j * CS + 4 * sl;
#pragma unroll
      for (int v = 0; v < V; ++v) cv[u][v] = __ldcg(reinterpret_cast<const float4 *>(cm + 32 * v));
      nz[u] = __ldcg(&cs.cnz[j].x);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float s = tb_group_dist<D>(xv, cv[u]);
      const int j = j0 + 4 * u + g;
      if (j < kp && nz[u] < HPC_DEAD) {
        if (s < a1) {
          a2 = a1;
          a1 = s;
          ja = j;
        } else {
          a2 = fminf(a2, s);
        }
      }
    }
  }
#pragma unroll
  for (int o = 8; o < 32; o <<= 1) {
    const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
    const int jb = __shfl_xor_sync(0xffffffffu, ja, o);
    const float b2 = __shfl_xor_sync(0xffffffffu, a2, o);
    hpc_merge_top2(a1, ja, a2, b1, jb, b2);
  }
  constexpr float rho = (float)(D + 3) * HPC_U32 * 1.001f;
  if (a2 - a1 > rho * (a1 + a2)) return ja < kp ? ja : 0;
  if (stats && lane == 0) atomicAdd(stats + 3, 1ull);
  // every centroid whose exact value may be at most the best's: FP32 value
  // s_j with s_j / (1 + rho) <= a1 / (1 - rho)
  const float thr = a1 * ((1.0f + rho) / (1.0f - rho)) * 1.0001f;
  double b = __longlong_as_double(0x7ff0000000000000ll);
  int jb = 0x7fffffff;
#pragma unroll 1
  for (int j0 = 0; j0 < kp; j0 += 4) {
    const int j = min(j0 + g, kp - 1);
    const float *cm = cs.cm + (size_t)j * CS;
    float4 cv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) cv[v] = __ldcg(reinterpret_cast<const float4 *>(cm + 4 * sl + 32 * v));
    const float s = tb_group_dist<D>(xv, cv);
    if (j0 + g < kp && sl == 0 && __ldcg(&cs.cnz[j].x) < HPC_DEAD && s <= thr) {
      double acc64 = 0.0;
      for (int t = 0; t < D; ++t) {
        const double c = -0.5 * (double)__ldcg(cm + t);
        const double diff = __dsub_rn((double)__ldg(x + t), c);
        acc64 = __dadd_rn(acc64, __dmul_rn(diff, diff));
      }
      if (acc64 < b) {  // j increases along a lane: ties keep the lower index
        b = acc64;
        jb = j;
      }
    }
  }
#pragma unroll
  for (int o = 8; o < 32; o <<= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, b, o);
    const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
    if (ob < b || (ob == b && oj < jb)) {
      b = ob;
      jb = oj;
    }
  }
  jb = __shfl_sync(0xffffffffu, jb, 0);  // the first lanes of the groups held the FP64 values
  return jb < kp ? jb : ja < kp ? ja : 0;
}

// Rows whose settling needs every centroid, deferred to after the CTA's
// pipeline (where every warp takes part, so that their latency overlaps):
// `cap` row indices per CTA in global memory, *count in shared memory.
struct TbQueue {
  int64_t *rows;
  int cap;
  int *count;
};

enum { TB_DONE = 1, TB_BAD = 0, TB_QUEUED = 2 };

// FP32 direct-form distances (and, with NORM, squared norms) of the warp's
// rows whose lanes are set in `todo` (lane l: row row0w + l, centroid jl),
// by 8-lane groups over dimensions: each round, group g takes the g-th of
// the next four rows, lane i of the group reads dimensions 4i + 32v ..
// 4i + 32v + 3 of the row and of the centroid's -2c row (coalesced 128-byte
// pieces), the group adds its lanes' partial sums by shuffles, and the row's
// own lane picks them up.  Every lane calls it; lanes not in `todo` keep
// their nx, dd.  Relative bounds as for any order of the D nonnegative
// terms: (D + 3) u for the distance.
template <int D, bool NORM>
__device__ __forceinline__ void tb_group_direct(const float *__restrict__ rows, int64_t row0w,
                                                unsigned todo, int jl, const float *cm, float &nx,
                                                float &dd) {
  constexpr int CS = hpc_cstride(D);
  constexpr int V = D / 32;
  const int lane = threadIdx.x & 31, g = lane >> 3, sl = lane & 7;
  while (todo) {  // the same for the whole warp
    unsigned t = todo;
    for (int i = 0; i < g; ++i) t &= t - 1;
    const int src = t ? __ffs(t) - 1 : -1;  // this group's row (lane), if any
    const int j = __shfl_sync(0xffffffffu, jl, src < 0 ? 0 : src);
    float pn = 0.0f, pd = 0.0f;
    if (src >= 0) {
      const float *xr = rows + (row0w + src) * D + 4 * sl;
      const float *cr = cm + (size_t)j * CS + 4 * sl;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(xr + 32 * v));
        const float4 c = __ldcg(reinterpret_cast<const float4 *>(cr + 32 * v));
        if constexpr (NORM) {
          pn = __fmaf_rn(x.x, x.x, pn);
          pn = __fmaf_rn(x.y, x.y, pn);
          pn = __fmaf_rn(x.z, x.z, pn);
          pn = __fmaf_rn(x.w, x.w, pn);
        }
        const float e0 = __fmaf_rn(0.5f, c.x, x.x), e1 = __fmaf_rn(0.5f, c.y, x.y);
        const float e2 = __fmaf_rn(0.5f, c.z, x.z), e3 = __fmaf_rn(0.5f, c.w, x.w);
        pd = __fmaf_rn(e0, e0, pd);
        pd = __fmaf_rn(e1, e1, pd);
        pd = __fmaf_rn(e2, e2, pd);
        pd = __fmaf_rn(e3, e3, pd);
      }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      pd += __shfl_xor_sync(0xffffffffu, pd, o);
      if constexpr (NORM) pn += __shfl_xor_sync(0xffffffffu, pn, o);
    }
    // lane l's row went to group popc(todo below l) when that is under 4
    const int rank = __popc(todo & ((1u << lane) - 1u));
    const bool mine = ((todo >> lane) & 1u) && rank < 4;
    const float rd = __shfl_sync(0xffffffffu, pd, 8 * (rank < 4 ? rank : 0));
    const float rn = NORM ? __shfl_sync(0xffffffffu, pn, 8 * (rank < 4 ? rank : 0)) : 0.0f;
    if (mine) {
      dd = rd;
      if constexpr (NORM) nx = rn;
    }
    for (int i = 0; i < 4; ++i) todo &= todo - 1;
  }
}

// The exact stages of one row (whole warp; lane l's row is row0w + l).
// Returns TB_DONE with the exact nearest centroid in *j_out and its FP32
// direct-form distance in *dd_out, TB_QUEUED when the row went to the CTA's
// queue, TB_BAD for an invalid or non-finite row (status recorded).
template <int D, int IB>
__device__ __forceinline__ int tb_exact(const float *__restrict__ rows, int64_t row0w, int64_t row,
                                        bool valid, int j1, int j2, float d1, float d2, float lo3,
                                        const hpc_cent_smem &gcs, int *status,
                                        unsigned long long *stats, const TbQueue &queue,
                                        int *j_out, float *dd_out) {
  constexpr int CS = hpc_cstride(D);
  const int lane = threadIdx.x & 31;
  const bool found = d1 < HPC_DEAD * 0.5f;
  if (!found) j1 = 0;
  const float *xg = rows + (valid ? row : 0) * D;
  float nx = 0.0f, dd = 0.0f;
  tb_group_direct<D, true>(rows, row0w, __ballot_sync(0xffffffffu, valid), j1, gcs.cm, nx, dd);
  const float rad = sqrtf(nx) * 1.0001f + gcs.cmax * 1.0001f;
  float win = 2.0f * TB_E_REL * rad * rad;
  win += 1.0001f * ldexpf(1.0f, IB - 22) * (fabsf(d1) + fabsf(d2));  // keys
  bool ok = valid;
  if (valid && !(found && isfinite(nx) && isfinite(win))) {
    hpc_status_set(status, HPC_ERR_NONFINITE);
    ok = false;
  }
  constexpr float rho = (float)(D + 3) * HPC_U32 * 1.001f;  // FP32 direct-form bound
  bool full = false;
  const bool near = ok && !(d2 - d1 > win);
  // the two nearest by the tensor-core values, exactly; every other
  // centroid's tensor-core key is at least lo3, the third smallest, so its
  // distance is at least ||x||^2 + lo3 - E (less lo3's own key error)
  const bool has2 = near && d2 < HPC_DEAD * 0.5f && j2 != j1;
  float ex2 = __int_as_float(0x7f800000), unused = 0.0f;
  tb_group_direct<D, false>(rows, row0w, __ballot_sync(0xffffffffu, has2), j2, gcs.cm, unused, ex2);
  if (near) {
    const float E = 0.5f * win + 1.0001f * ldexpf(1.0f, IB - 23) * fabsf(lo3);
    const float others = lo3 >= HPC_DEAD * 0.5f
                             ? __int_as_float(0x7f800000)
                             : nx * (1.0f - (float)(D + 2) * HPC_U32 * 1.01f) + lo3 - E -
                                   4.0f * HPC_U32 * (nx + fabsf(lo3) + E);
    const bool lo1 = dd < ex2 || (dd == ex2 && j1 < j2);
    const float lo = lo1 ? dd : ex2, hi = lo1 ? ex2 : dd;
    if (lo * (1.0f + rho) < others && hi * (1.0f - rho) > lo * (1.0f + rho)) {
      if (!lo1) {
        j1 = j2;
        dd = ex2;
      }
    } else {
      full = true;  // a third candidate, or a tie FP32 cannot split
    }
  }
  unsigned mfull = __ballot_sync(0xffffffffu, full);
  bool queued = false;
  if (mfull && queue.rows) {
    int q0 = 0;
    if (lane == 0) q0 = atomicAdd(queue.count, __popc(mfull));
    q0 = __shfl_sync(0xffffffffu, q0, 0);
    const int q = q0 + __popc(mfull & ((1u << lane) - 1u));
    if (full && q < queue.cap) {
      queue.rows[q] = row;
      queued = true;
    }
    mfull = __ballot_sync(0xffffffffu, full && !queued);  // the queue was full for these
  }
  if (stats) {  // the same for the whole warp
    const unsigned bv = __ballot_sync(0xffffffffu, valid);
    const unsigned bn = __ballot_sync(0xffffffffu, near);
    const unsigned bf = __ballot_sync(0xffffffffu, full);
    if (lane == 0) {
      atomicAdd(stats + 0, (unsigned long long)__popc(bv));
      atomicAdd(stats + 1, (unsigned long long)__popc(bn));
      atomicAdd(stats + 2, (unsigned long long)__popc(bf));
    }
  }
  while (mfull) {
    const int src = __ffs(mfull) - 1;
    mfull &= mfull - 1;
    const int j = tb_rescore<D>(rows + (row0w + src) * D, gcs, stats);
    if (lane == src && j != j1) {
      j1 = j;
      dd = tb_direct<D>(xg, gcs.cm + (size_t)j1 * CS);
    }
  }
  if (ok && !queued && !isfinite(dd)) {
    hpc_status_set(status, HPC_ERR_NONFINITE);
    ok = false;
  }
  *j_out = j1;
  *dd_out = dd;
  return queued ? TB_QUEUED : ok ? TB_DONE : TB_BAD;
}

// Settles the rows of the CTA's queue after its pass, when no MMA or copy
// touches shared memory any more: the CTA stages the exact centroid block
// (-2c rows of hpc_cstride(D) floats and the (||c||^2, 0) pairs; the row
// padding puts the rows that 32 lanes read at once in different banks) in
// shared memory, below the flags and barriers, and each warp takes a row at a
// time: the row in the warp's shared-memory slot, lane l the centroids
// l, l + 32, ..., FP32 direct form in dimension order (relative bound
// (D + 3) u); if the two best are not separated by that bound, FP64 in the
// oracle's operation order for the centroids whose FP32 value lies within it
// of the best, ties to the lowest index.  `done(row, j, dd)` is then called
// by the whole warp (dd: the objective's FP32 direct-form distance).
template <int D, int NP, typename Done>
__device__ __forceinline__ void tb_settle_queue(const TbSm &m, const float *__restrict__ rows,
                                                const TbQueue &queue, const hpc_cent_smem &gcs,
                                                unsigned long long *stats, Done done) {
  using Cfg = TbCfg<D, NP>;
  constexpr int CS = hpc_cstride(D);
  constexpr int NPL = NP / 32;  // centroids per lane
  constexpr size_t CM_BYTES = (size_t)NP * CS * 4, NZ_BYTES = (size_t)NP * 8;
  static_assert(CM_BYTES + NZ_BYTES + (size_t)(TB_THREADS / 32) * D * 4 <= Cfg::DEADF,
                "the centroid block fits below the flags");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nq = min(*queue.count, queue.cap);
  if (nq == 0) return;  // the same for the whole CTA
  const int kp = gcs.kp;
  float *cm = reinterpret_cast<float *>(m.bh);
  float2 *cnz = reinterpret_cast<float2 *>(m.bh + CM_BYTES);
  float *xs = reinterpret_cast<float *>(m.bh + CM_BYTES + NZ_BYTES) + (size_t)warp * D;
  {
    const float4 *src = reinterpret_cast<const float4 *>(gcs.cm);
    float4 *dst = reinterpret_cast<float4 *>(cm);
    for (int e = threadIdx.x; e < kp * CS / 4; e += TB_THREADS) dst[e] = __ldcg(src + e);
    for (int j = threadIdx.x; j < kp; j += TB_THREADS) cnz[j] = __ldcg(gcs.cnz + j);
  }
  __syncthreads();
  constexpr float rho = (float)(D + 3) * HPC_U32 * 1.001f;
  for (int qi = warp; qi < nq; qi += TB_THREADS / 32) {
    const int64_t row = queue.rows[qi];
    const float *xg = rows + row * D;
    for (int t = lane * 4; t < D; t += 128)
      *reinterpret_cast<float4 *>(xs + t) = __ldg(reinterpret_cast<const float4 *>(xg + t));
    __syncwarp();
    float acc[NPL];
    uint32_t live = 0u;  // bit u: centroid lane + 32 u is live
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int j = lane + 32 * u;
      if (j < kp && cnz[j].x < HPC_DEAD) live |= 1u << u;
      acc[u] = 0.0f;
    }
#pragma unroll 2
    for (int t = 0; t < D; t += 4) {
      const float4 x = *reinterpret_cast<const float4 *>(xs + t);
#pragma unroll
      for (int u = 0; u < NPL; ++u) {
        const float4 c = *reinterpret_cast<const float4 *>(cm + (size_t)(lane + 32 * u) * CS + t);
        const float d0 = __fmaf_rn(0.5f, c.x, x.x), d1 = __fmaf_rn(0.5f, c.y, x.y);
        const float d2 = __fmaf_rn(0.5f, c.z, x.z), d3 = __fmaf_rn(0.5f, c.w, x.w);
        acc[u] = __fmaf_rn(d0, d0, acc[u]);
        acc[u] = __fmaf_rn(d1, d1, acc[u]);
        acc[u] = __fmaf_rn(d2, d2, acc[u]);
        acc[u] = __fmaf_rn(d3, d3, acc[u]);
      }
    }
    float a1 = __int_as_float(0x7f800000), a2 = a1;
    int ja = 0x7fffffff;
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      if (!((live >> u) & 1u)) continue;
      if (acc[u] < a1) {
        a2 = a1;
        a1 = acc[u];
        ja = lane + 32 * u;
      } else {
        a2 = fminf(a2, acc[u]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float b1 = __shfl_xor_sync(0xffffffffu, a1, o);
      const int jb = __shfl_xor_sync(0xffffffffu, ja, o);
      const float b2 = __shfl_xor_sync(0xffffffffu, a2, o);
      hpc_merge_top2(a1, ja, a2, b1, jb, b2);
    }
    int j = ja < kp ? ja : 0;
    if (!(a2 - a1 > rho * (a1 + a2))) {
      if (stats && lane == 0) atomicAdd(stats + 3, 1ull);
      // the centroids whose exact value may be at most the best's
      const float thr = a1 * ((1.0f + rho) / (1.0f - rho)) * 1.0001f;
      double b = __longlong_as_double(0x7ff0000000000000ll);
      int jb = 0x7fffffff;
#pragma unroll
      for (int u = 0; u < NPL; ++u) {
        if (!((live >> u) & 1u) || !(acc[u] <= thr)) continue;
        const float *cj = cm + (size_t)(lane + 32 * u) * CS;
        double acc64 = 0.0;
        for (int t = 0; t < D; ++t) {
          const double c = -0.5 * (double)cj[t];
          const double diff = __dsub_rn((double)xs[t], c);
          acc64 = __dadd_rn(acc64, __dmul_rn(diff, diff));
        }
        if (acc64 < b) {  // u increases: ties keep the lower index
          b = acc64;
          jb = lane + 32 * u;
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
      if (jb < kp) j = jb;
    }
    const float dd = tb_direct<D>(xg, gcs.cm + (size_t)j * CS);
    __syncwarp();  // the row slot is read before the next row is staged
    done(row, j, dd);
  }
}

// One pass of the pipeline over a CTA's tiles (all threads of the CTA call it).
template <int D, int NP, typename Fin>
__device__ __forceinline__ void tb_pass(const TbSm &m, const TbRows &R, uint32_t gbase, int kp, int *status,
                        Fin fin) {
  const int warp = threadIdx.x >> 5;
  if (warp == TB_MMAW) {
    if ((threadIdx.x & 31) == 0) tb_mma<D, NP>(m, R, gbase, status);
    __syncwarp();
  } else if (warp < TB_FIN0) {
    tb_fold<D, NP>(m, R, gbase, kp, status);
  } else {
    tb_finish<D, NP>(m, R, gbase, kp, status, fin);
  }
}

// B (split c'), the norms and the flags from centroid values given by
// `val(j, t0, c[])` (PER = D / 32 values of row j from dim t0), for rows
// j < k that are live; rows beyond k and dead rows get zeros and HPC_DEAD.
// Warp-per-row; returns through s_nmax / s_live (shared) the largest squared
// norm (bits) and the live count.  When `ex` is set (the task's first CTA)
// the exact block (gcent) is written too.
template <int D, int NP, typename Val>
__device__ __forceinline__ void tb_build_b(const TbSm &m, int k, float *gcent, bool ex, unsigned *s_nmax,
                           unsigned *s_live, Val val) {
  constexpr int PER = D / 32;
  constexpr int CS = hpc_cstride(D);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = TB_THREADS / 32;
  const int kp = (k + 1) & ~1;
  float2 *gcnz = reinterpret_cast<float2 *>(gcent + (size_t)kp * CS);
  for (int j = warp; j < NP; j += nw) {
    float c[PER];
    bool live = j < k && !m.dead[j];
    if (live) {
      live = val(j, lane * PER, c);  // false: the centroid just became empty
    }
    if (!live) {
#pragma unroll
      for (int u = 0; u < PER; ++u) c[u] = 0.0f;
    }
    tb_store_b<PER, NP>(m, j, lane * PER, c);
    float nn = 0.0f;
#pragma unroll
    for (int u = 0; u < PER; ++u) nn = fmaf(c[u], c[u], nn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (ex && live && j < kp) {
#pragma unroll
      for (int u = 0; u < PER; ++u) gcent[(size_t)j * CS + lane * PER + u] = -2.0f * c[u];
    }
    if (lane == 0) {
      m.cn[j] = live ? nn : HPC_DEAD;
      if (ex && j < kp) gcnz[j] = make_float2(live ? nn : HPC_DEAD, 0.0f);
      if (live) {
        atomicMax(s_nmax, __float_as_uint(nn));
        atomicAdd(s_live, 1u);
      }
    }
  }
  hpc_fence_proxy_async();  // B's generic writes, visible to the tensor core
}

// ---- Lloyd ----------------------------------------------------------------------
struct TclArgs {
  int W;
  hpc_lloyd_task single;
  const hpc_lloyd_task *tasks;
  const int *block_task;   // W > 1: each CTA's first task (-2: take one from the list)
  const int *follow;       // W > 1: the tasks CTAs take as they become free, largest first
  const int *nfollow;      // W > 1: their number (device)
  const int *next;         // W > 1: the task a set runs after this one (-1: none)
  unsigned *pop;           // W > 1: the list's next entry (zero at launch)
  int max_iter;
  double tol;
  int *status;
  uint32_t *round_advance;
  unsigned long long *stats;  // nullable: rows, near rows, fully rescored, FP64
  int64_t *queue;             // nullable: queue_cap rows per CTA (tb_settle_queue)
  int queue_cap;
};

template <int D, int NP>
__global__ void __launch_bounds__(TB_THREADS, 1) tcl_lloyd_kernel(TclArgs a) {
  using Cfg = TbCfg<D, NP>;
  constexpr int CS = hpc_cstride(D);
  constexpr int PER = D / 32;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_dsum[32];
  __shared__ double s_f;
  __shared__ int s_done, s_abort;
  __shared__ unsigned s_umax, s_cmax, s_nmax, s_live;
  __shared__ uint32_t s_tmem;
  __shared__ int s_qn;
  // the current task's descriptor: its fields are read from here where used
  // rather than held in registers through the task
  __shared__ hpc_lloyd_task s_tk;
  // per-task values read where used (thread 0 writes them): the fixed-point
  // grids of the sums (2^-Fs) and of the objective (oscale = 2^Fo), the
  // previous objective
  __shared__ int s_Fs;
  __shared__ float s_oscale;
  __shared__ double s_fprev;

  if (a.round_advance && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.round_advance, 1u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *base =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TbSm m = tb_bind<D, NP>(base, &s_abort);

  if (threadIdx.x == 0) {
    tb_init_barriers<D, NP>(m);
    s_abort = 0;
  }
  if (warp == TB_MMAW) hpc_tmem_alloc(&s_tmem, Cfg::TCOLS);
  hpc_tc_fence_before();
  __syncthreads();
  hpc_tc_fence_after();
  m.tmem = s_tmem;
  // the CTA's tasks, one after another: those of its set, each on all of
  // the set's CTAs, then any from the list, alone; the pipeline's tile
  // sequence runs on from task to task
  uint32_t gbase = 0, drains = 0;
  // the next task from the list (the same for the whole CTA), -1 when empty
  auto take = [&]() {
    if (threadIdx.x == 0) {
      const unsigned i = atomicAdd(a.pop, 1u);
      s_qn = i < (unsigned)*a.nfollow ? a.follow[i] : -1;
    }
    __syncthreads();
    const int t = s_qn;
    __syncthreads();
    return t;
  };
  int tix = a.W == 1 ? 0 : a.block_task[blockIdx.x];
  bool alone = false;  // a task from the list: this CTA alone
  if (tix == -2) {
    tix = take();
    alone = true;
  }
  while (tix >= 0) {
  if (threadIdx.x == 0) s_tk = a.W == 1 ? a.single : a.tasks[tix];
  __syncthreads();
  const hpc_lloyd_task &tk = s_tk;
  const int k = tk.k, kp = (k + 1) & ~1;
  const int64_t s = tk.s;
  const int G = alone ? 1 : tk.nblocks, lb = alone ? 0 : (int)blockIdx.x - tk.block0;
  if (threadIdx.x == 0) {
    s_umax = s_cmax = s_nmax = s_live = 0u;
    s_qn = 0;
    s_done = 0;
    s_fprev = 0.0;
  }
  for (int j = threadIdx.x; j < 512; j += TB_THREADS) m.dead[j] = (j >= k) || tk.deg[j] != 0;
  __syncthreads();

  // Phase 0: largest |x| of the sample (fixed-point grid, non-finite rows),
  // zero sums, B from the starting centroids
  const int64_t ntiles = (s + TB_M - 1) / TB_M;
  {
    unsigned mx = 0u;
    for (int64_t e = (int64_t)lb * TB_THREADS + threadIdx.x; e < s * D;
         e += (int64_t)G * TB_THREADS) {
      const unsigned b = __float_as_uint(tk.S[e]) & 0x7fffffffu;
      mx = b > mx ? b : mx;
    }
    atomicMax(&s_umax, mx);
    for (int64_t e = (int64_t)lb * TB_THREADS + threadIdx.x; e < (int64_t)k * D;
         e += (int64_t)G * TB_THREADS)
      tk.gsum[e] = 0ull;
    for (int j = lb * TB_THREADS + threadIdx.x; j < k; j += G * TB_THREADS) tk.gcount[j] = 0u;
  }
  __syncthreads();
  tb_build_b<D, NP>(m, k, tk.gcent, lb == 0, &s_nmax, &s_live, [&](int j, int t0, float(&c)[PER]) {
    unsigned mc = 0u;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      c[u] = tk.C[(int64_t)j * D + t0 + u];
      const unsigned b = __float_as_uint(c[u]) & 0x7fffffffu;
      mc = b > mc ? b : mc;
    }
    atomicMax(&s_cmax, mc);
    return true;
  });
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(tk.gmaxabs, s_umax);
  // the exact centroid block as the latest build left it (max norm and live
  // count from shared memory, so that nothing of it stays in registers
  // through the pass)
  auto gcs_now = [&]() {
    return tb_gcs<D>(tk.gcent, k, sqrtf(__uint_as_float(s_nmax)), (int)s_live);
  };
  const int live0 = (int)s_live;
  bool run = hpc_grid_sync(tk.bar, a.status, (unsigned)G);
  const unsigned mabs = run ? __ldcg(tk.gmaxabs) : 0u;
  if (run && (mabs >= 0x7f800000u || s_cmax >= 0x7f800000u)) {
    if (threadIdx.x == 0) hpc_status_set(a.status, HPC_ERR_NONFINITE);
    run = false;
  }
  if (run && live0 == 0) {
    if (threadIdx.x == 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);
    run = false;
  }
  if (threadIdx.x == 0) {
    int Fs = 126;
    if (mabs != 0u) Fs = min(126, 62 - hpc_bit_length(s) - hpc_frexp_exp(__uint_as_float(mabs)));
    int Fo = 126;
    const unsigned mm = max(mabs, s_cmax);
    if (mm != 0u && mm < 0x7f800000u)
      Fo = min(126, 59 - hpc_bit_length(s) - hpc_bit_length(D) - 2 * hpc_frexp_exp(__uint_as_float(mm)));
    Fo = max(Fo, -126);
    s_Fs = Fs;
    s_oscale = hpc_pow2f(Fo);
  }
  __syncthreads();

  TbRows R;
  R.rows = tk.S;
  R.nrows = s;
  R.tile0 = lb;
  R.tstep = G;
  R.ntiles = lb < ntiles ? (int)((ntiles - 1 - lb) / G + 1) : 0;
  for (int it = 0; run; ++it) {
    // Phase A: assignment of the CTA's rows, sums of the rows that moved
    float fs_hi = 0.0f, fs_lo = 0.0f;
    // a row that moved from centroid jo (-1: first assignment) to jn: the
    // whole warp adds its fixed-point coordinates to jn's sums and takes them
    // from jo's, lanes over dimensions
    auto move = [&](int64_t row, int jn, int jo) {
      const float *xp = tk.S + row * D + lane * PER;
      float xv[PER];
      if constexpr (PER == 4) {
        const float4 q4 = __ldg(reinterpret_cast<const float4 *>(xp));
        xv[0] = q4.x;
        xv[1] = q4.y;
        xv[2] = q4.z;
        xv[3] = q4.w;
      } else {
        const float2 q2 = __ldg(reinterpret_cast<const float2 *>(xp));
        xv[0] = q2.x;
        xv[1] = q2.y;
      }
      const float qscale = hpc_pow2f(s_Fs);
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const long long qv = __float2ll_rn(xv[u] * qscale);
        atomicAdd(&tk.gsum[(size_t)jn * D + lane * PER + u], (unsigned long long)qv);
        if (jo >= 0) atomicAdd(&tk.gsum[(size_t)jo * D + lane * PER + u], (unsigned long long)(-qv));
      }
      if (lane == 0) {
        atomicAdd(&tk.gcount[jn], 1u);
        if (jo >= 0) atomicSub(&tk.gcount[jo], 1u);
      }
    };
    TbQueue queue{a.queue + (size_t)blockIdx.x * a.queue_cap, a.queue_cap, &s_qn};
    if (!a.queue) queue.rows = nullptr;
    tb_pass<D, NP>(m, R, gbase, kp, a.status,
                   [&](int64_t row0w, int64_t row, bool valid, int j1, int j2, float d1, float d2,
                       float lo3) {
      int j = 0;
      float dd = 0.0f;
      const bool ok = tb_exact<D, Cfg::IB>(tk.S, row0w, row, valid, j1, j2, d1, d2, lo3,
                                           gcs_now(), a.status, a.stats, queue, &j, &dd) ==
                      TB_DONE;
      if (ok) hpc_sum2_add(fs_hi, fs_lo, dd);
      int old = -1;
      bool moved = false;
      if (ok) {
        old = it > 0 ? tk.plab[row] : -1;
        moved = old != j;
        tk.plab[row] = j;
      }
      unsigned mv = __ballot_sync(0xffffffffu, moved);
      while (mv) {
        const int src = __ffs(mv) - 1;
        mv &= mv - 1;
        move(row0w + src, __shfl_sync(0xffffffffu, j, src), __shfl_sync(0xffffffffu, old, src));
      }
      if (ok && tk.labels && tk.labels != tk.plab) tk.labels[row] = j;
    });
    __syncthreads();
    // the queued rows, every warp
    tb_settle_queue<D, NP>(m, tk.S, queue, gcs_now(), a.stats, [&](int64_t row, int j, float dd) {
      if (lane == 0) hpc_sum2_add(fs_hi, fs_lo, dd);
      const int old = it > 0 ? tk.plab[row] : -1;
      if (old != j) move(row, j, old);
      __syncwarp();
      if (lane == 0) {
        tk.plab[row] = j;
        if (tk.labels && tk.labels != tk.plab) tk.labels[row] = j;
      }
    });
    gbase += (uint32_t)R.ntiles;
    __syncthreads();
    if (s_abort) break;
    // the objective partial on the grid 2^-Fo, summed over the block in integers
    const float oscale = s_oscale;
    const unsigned long long bq = hpc_block_sum_u64(
        (unsigned long long)(__float2ll_rn(fs_hi * oscale) + __float2ll_rn(fs_lo * oscale)),
        reinterpret_cast<unsigned long long *>(s_dsum));
    const int buf = it % 3;
    if (threadIdx.x == 0 && bq != 0ull) atomicAdd(tk.gobj + buf, bq);
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) break;
    // Phase B: objective, stop test, new centroids (every CTA, identical)
    if (threadIdx.x == 0) {
      // 1 / oscale is an exact power of two
      const double fo = (double)(long long)__ldcg(tk.gobj + buf) / (double)s_oscale;
      const double f_prev = s_fprev;
      s_f = fo;
      s_fprev = fo;
      s_done = (it > 0 && (f_prev == 0.0 || (f_prev - fo) < a.tol * f_prev)) || it == a.max_iter;
      s_nmax = 0u;
      s_live = 0u;
      s_qn = 0;
    }
    __syncthreads();
    const double f = s_f;
    if (s_done) {
      if (lb == 0) {
        if (threadIdx.x == 0) {
          *tk.f_out = f;
          if (tk.iters_out) *tk.iters_out = it;
        }
        if (tk.fhat) hpc_incumbent_block(tk, D, f, it);
      }
      break;
    }
    tb_build_b<D, NP>(m, k, tk.gcent, lb == 0, &s_nmax, &s_live,
                      [&](int j, int t0, float(&c)[PER]) {
      const unsigned cnt = __ldcg(tk.gcount + j);
      if (cnt == 0u) {  // emptied: degenerate for the rest of the run
        __syncwarp();
        if (lane == 0) {
          m.dead[j] = 1;
          if (lb == 0) tk.deg[j] = 1;
        }
        return false;
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const long long q = (long long)__ldcg(tk.gsum + (size_t)j * D + t0 + u);
        c[u] = hpc_mean_f32(q, cnt, s_Fs);
        if (lb == 0) tk.C[(int64_t)j * D + t0 + u] = c[u];
      }
      return true;
    });
    if (lb == 0 && threadIdx.x == 0) tk.gobj[(it + 2) % 3] = 0ull;
    __syncthreads();
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) break;
  }
  __syncthreads();  // every thread is done with the task's shared state
  // a task that stopped on an error (status recorded) ends the CTA's list;
  // s_done is set only by a run that finished
  const bool finished = s_done != 0;
  // the set's next task (on all its CTAs), else one from the list, alone
  const int nxt = !finished || a.W == 1 || alone ? -1 : a.next[tix];
  tix = !finished || a.W == 1 ? -1 : nxt >= 0 ? nxt : take();
  alone = nxt < 0;
  }
  // drain: no MMA may still target this CTA's TMEM or shared memory
  __syncthreads();
  if (warp == TB_MMAW && lane == 0) tb_drain(m, drains++, a.status);
  hpc_tc_fence_before();
  __syncthreads();
  if (warp == TB_MMAW) {
    hpc_tc_fence_after();
    hpc_tmem_dealloc(m.tmem, Cfg::TCOLS);
  }
}

// ---- full-data objective ----------------------------------------------------------
struct TcbArgs {
  const float *X;
  int64_t n;
  int k;
  const float *C;
  const uint8_t *deg;
  float *gcent;
  const float *gmeta;  // [0] max ||c||, [1] live count (int bits)
  double *f_out;
  int32_t *labels;
  int *status;
  double *part;
  unsigned *done_count;
  unsigned long long *stats;  // nullable: rows, near rows, fully rescored, FP64
  int64_t *queue;             // nullable: queue_cap rows per CTA (tb_settle_queue)
  int queue_cap;
};

// One block: the exact centroid block and its max norm / live count.
template <int D>
__global__ void tcb_prep_kernel(const float *__restrict__ C, const uint8_t *__restrict__ deg, int k,
                                float *gcent, float *gmeta) {
  __shared__ float s_red[2];
  hpc_cent_smem cs;
  hpc_cent_bind(cs, reinterpret_cast<unsigned char *>(gcent), D, k);
  hpc_load_centroids<D>(cs, C, deg, k, D, s_red);
  if (threadIdx.x == 0) {
    gmeta[0] = cs.cmax;
    gmeta[1] = __int_as_float(cs.live);
  }
}

template <int D, int NP>
__global__ void __launch_bounds__(TB_THREADS, 1) tcb_objective_kernel(TcbArgs a) {
  using Cfg = TbCfg<D, NP>;
  constexpr int PER = D / 32;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_dsum[32];
  __shared__ bool s_last;
  __shared__ int s_abort;
  __shared__ unsigned s_nmax, s_live;
  __shared__ uint32_t s_tmem;
  __shared__ int s_qn;
  const int warp = threadIdx.x >> 5;
  unsigned char *base =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TbSm m = tb_bind<D, NP>(base, &s_abort);
  const int k = a.k, kp = (k + 1) & ~1;
  if (threadIdx.x == 0) {
    tb_init_barriers<D, NP>(m);
    s_abort = 0;
    s_nmax = s_live = 0u;
    s_qn = 0;
  }
  if (warp == TB_MMAW) hpc_tmem_alloc(&s_tmem, Cfg::TCOLS);
  for (int j = threadIdx.x; j < 512; j += TB_THREADS)
    m.dead[j] = (j >= k) || (a.deg != nullptr && a.deg[j] != 0);
  hpc_tc_fence_before();
  __syncthreads();
  hpc_tc_fence_after();
  m.tmem = s_tmem;
  tb_build_b<D, NP>(m, k, a.gcent, false, &s_nmax, &s_live, [&](int j, int t0, float(&c)[PER]) {
#pragma unroll
    for (int u = 0; u < PER; ++u) c[u] = a.C[(int64_t)j * D + t0 + u];
    return true;
  });
  __syncthreads();
  const hpc_cent_smem gcs = tb_gcs<D>(a.gcent, k, a.gmeta[0], __float_as_int(a.gmeta[1]));
  const bool run = gcs.live > 0;
  if (!run && a.n > 0 && threadIdx.x == 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);
  const int64_t ntiles = (a.n + TB_M - 1) / TB_M;
  TbRows R;
  R.rows = a.X;
  R.nrows = a.n;
  R.tile0 = blockIdx.x;
  R.tstep = gridDim.x;
  R.ntiles = run && (int64_t)blockIdx.x < ntiles
                 ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  float fs_hi = 0.0f, fs_lo = 0.0f;
  TbQueue queue{a.queue + (size_t)blockIdx.x * a.queue_cap, a.queue_cap, &s_qn};
  if (!a.queue) queue.rows = nullptr;
  tb_pass<D, NP>(m, R, 0u, kp, a.status,
                 [&](int64_t row0w, int64_t row, bool valid, int j1, int j2, float d1, float d2,
                     float lo3) {
    int j = 0;
    float dd = 0.0f;
    if (tb_exact<D, Cfg::IB>(a.X, row0w, row, valid, j1, j2, d1, d2, lo3, gcs, a.status,
                                      a.stats, queue, &j, &dd) == TB_DONE) {
      hpc_sum2_add(fs_hi, fs_lo, dd);
      if (a.labels) a.labels[row] = j;
    }
  });
  __syncthreads();
  tb_settle_queue<D, NP>(m, a.X, queue, gcs, a.stats, [&](int64_t row, int j, float dd) {
    if ((threadIdx.x & 31) == 0) {
      hpc_sum2_add(fs_hi, fs_lo, dd);
      if (a.labels) a.labels[row] = j;
    }
  });
  __syncthreads();
  if (warp == TB_MMAW && (threadIdx.x & 31) == 0 && R.ntiles > 0) tb_drain(m, 0u, a.status);
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
      *a.f_out = (!run && a.n > 0) ? __longlong_as_double(0x7ff8000000000000ll) : f;
      *a.done_count = 0u;
    }
  }
  hpc_tc_fence_before();
  __syncthreads();
  if (warp == TB_MMAW) {
    hpc_tc_fence_after();
    hpc_tmem_dealloc(m.tmem, Cfg::TCOLS);
  }
}

// ---- host side ----------------------------------------------------------------------
int tb_np(int k) { return k <= 128 ? 128 : k <= 256 ? 256 : 512; }

// The CTAs of a batched tensor-core Lloyd launch (one per SM).  A launch
// runs up to 128 workers on 152 CTAs, so the average worker is about 1.2
// CTAs of work, and a CTA serves one worker at a time: whole CTAs per worker
// (a group for the larger ones, the smaller ones one after another on a CTA
// each) left the launch at about 1.5 times the balanced time even with the
// update counts known.  So the workers are dealt into sets, each a
// contiguous range of CTAs that runs its workers one after another, every
// worker on all of the set's CTAs (its rows split evenly, its barriers over
// the set): the workers, largest first, go to the set with the least work
// so far (TCL_SET_CTAS CTAs a set on average), then the CTAs to the sets,
// one at a time to the set with the most work per CTA (at most as many as
// the tiles of its smallest worker).  Workers with fewer 128-row tiles than
// TCL_SET_CTAS could not use a set's CTAs: they wait in a list, largest
// first, and CTAs without a set, or done with theirs, take them one at a
// time and run them alone; the list keeps CTAs in proportion to its work
// (at least one, at most one per listed worker, all with no set).  The
// work of a worker is s k (u + 1), u its updates in its previous run (0
// before the first).  (Simulated with
// update counts like the large workload's, predicted from the previous
// round: 1.07-1.09 times the balanced time, against 1.7-1.8 for the groups
// and list.)  Computed by one thread, on the host for the plan and on the
// device before every launch (the previous run's updates are there).
// Writes block_task[0, total) (each CTA's first worker, -2: none, it takes
// from the list), next[0, W) (the worker its set runs after this one, -1
// after the last), nb[] and b0[] per worker (its set's CTAs; 1 and -1 for
// listed workers), and the list follow[0, nf); returns nf.
constexpr int TCL_PACK_MAX = 128;  // workers of one launch (a round's chunk)
constexpr int TCL_SET_CTAS = 16;   // CTAs of a set, on average

// a task's work: s k (u + 1), u its updates in the previous run (clamped)
__host__ __device__ inline double tcl_work(int64_t s, int k, int u) {
  const int uc = u > 0 ? (u < 1000 ? u : 1000) : 0;
  return (double)(s > 0 ? s : 1) * (double)k * (double)(uc + 1);
}

// One candidate plan: workers with fewer tiles than `tiny` in the list
// (largest first), the others dealt into sets over the CTAs the list leaves;
// returns its estimated makespan (a set: its work over its CTAs; the list:
// each worker, largest first, to the CTA free first).
struct TclCand {
  int nsets, nf;
  int64_t lc;
  double sum[TCL_PACK_MAX];
  int first[TCL_PACK_MAX], next[TCL_PACK_MAX], follow[TCL_PACK_MAX];
  int64_t g[TCL_PACK_MAX];
};

__host__ __device__ double tcl_candidate(int W, const int *order, const double *work,
                                         const int64_t *cap, int64_t total, int64_t tiny,
                                         TclCand &c) {
  int nsw = 0;
  double lwork = 0.0, all = 0.0;
  c.nf = 0;
  for (int i = 0; i < W; ++i) {
    const int w = order[i];
    all += work[w];
    c.next[w] = -1;
    if (cap[w] < tiny) {
      c.follow[c.nf++] = w;
      lwork += work[w];
    } else {
      ++nsw;
    }
  }
  c.lc = 0;
  if (c.nf > 0) {
    c.lc = (int64_t)floor((double)total * lwork / all + 0.5);
    if (c.lc < 1) c.lc = 1;
    if (c.lc > c.nf) c.lc = c.nf;
    if (nsw == 0) c.lc = total;  // no sets: every CTA takes from the list
    else if (c.lc > total - 1) c.lc = total - 1;
  }
  const int64_t tset = total - c.lc;  // the sets' CTAs
  int64_t ns = tset / TCL_SET_CTAS;
  if (ns < 1) ns = 1;
  if (ns > nsw) ns = nsw;
  c.nsets = (int)ns;  // 0 when every worker is listed
  int last[TCL_PACK_MAX];
  int64_t gmax[TCL_PACK_MAX];
  for (int j = 0; j < c.nsets; ++j) {
    c.sum[j] = 0.0;
    c.first[j] = last[j] = -1;
    gmax[j] = tset;
  }
  // the set workers, largest first, to the set with the least work (lowest
  // index on ties), appended to its sequence
  for (int i = 0; i < W; ++i) {
    const int w = order[i];
    if (cap[w] < tiny) continue;
    int b = 0;
    for (int j = 1; j < c.nsets; ++j)
      if (c.sum[j] < c.sum[b]) b = j;
    c.sum[b] += work[w];
    if (last[b] >= 0) c.next[last[b]] = w;
    else c.first[b] = w;
    last[b] = w;
    if (cap[w] < gmax[b]) gmax[b] = cap[w];
  }
  // CTAs: one each, then one at a time to the set with the most work per
  // CTA that may take another
  int64_t used = c.nsets;
  for (int j = 0; j < c.nsets; ++j) c.g[j] = 1;
  while (used < tset) {
    int b = -1;
    for (int j = 0; j < c.nsets; ++j)
      if (c.g[j] < gmax[j] && (b < 0 || c.sum[j] / (double)c.g[j] > c.sum[b] / (double)c.g[b]))
        b = j;
    if (b < 0) break;
    ++c.g[b];
    ++used;
  }
  // the estimate: every CTA's time; the list onto the CTA free first
  double t[TCL_PACK_MAX + 1];  // the sets' CTAs (one value a set), then one for the rest
  int64_t cnt[TCL_PACK_MAX + 1];
  int nt = 0;
  double mk = 0.0;
  for (int j = 0; j < c.nsets; ++j) {
    t[nt] = c.sum[j] / (double)c.g[j];
    cnt[nt++] = c.g[j];
    mk = t[nt - 1] > mk ? t[nt - 1] : mk;
  }
  if (total > used) {
    t[nt] = 0.0;
    cnt[nt++] = total - used;
  }
  // CTAs of equal free time are interchangeable: take one from the group
  // free first, it moves on by the worker's work
  double extra[TCL_PACK_MAX];  // CTAs that took list workers: their free time
  int ne = 0;
  for (int i = 0; i < c.nf; ++i) {
    int bt = -1, be = -1;
    for (int q = 0; q < nt; ++q)
      if (cnt[q] > 0 && (bt < 0 || t[q] < t[bt])) bt = q;
    for (int q = 0; q < ne; ++q)
      if (be < 0 || extra[q] < extra[be]) be = q;
    const double w = work[c.follow[i]];
    if (be >= 0 && (bt < 0 || extra[be] <= t[bt])) {
      extra[be] += w;
      mk = extra[be] > mk ? extra[be] : mk;
    } else if (bt >= 0) {
      --cnt[bt];
      extra[ne] = t[bt] + w;
      mk = extra[ne] > mk ? extra[ne] : mk;
      ++ne;
    }
  }
  return mk;
}

__host__ __device__ int tcl_pack_core(int W, const double *work, const int64_t *cap, int64_t total,
                                      int *block_task, int *follow, int *next, int *nb, int *b0,
                                      TclCand *cand) {
  int order[TCL_PACK_MAX];
  for (int w = 0; w < W; ++w) {  // largest first, lower index on ties (insertion)
    int i = w;
    while (i > 0 && work[order[i - 1]] < work[w]) {
      order[i] = order[i - 1];
      --i;
    }
    order[i] = w;
  }
  // every worker in sets, or the workers too small to use a set's CTAs (on
  // average) in the list: the plan with the smaller estimated makespan
  // (cand: room for two candidates, the caller's)
  const double ma = tcl_candidate(W, order, work, cap, total, 0, cand[0]);
  bool tiny = false;
  for (int w = 0; w < W; ++w) tiny = tiny || cap[w] < TCL_SET_CTAS;
  const TclCand *c = &cand[0];
  if (tiny && tcl_candidate(W, order, work, cap, total, TCL_SET_CTAS, cand[1]) < ma) c = &cand[1];
  for (int w = 0; w < W; ++w) {
    next[w] = c->next[w];
    nb[w] = 1;
    b0[w] = -1;  // listed workers run alone wherever they are taken
  }
  for (int i = 0; i < c->nf; ++i) follow[i] = c->follow[i];
  int64_t grid = 0;
  for (int j = 0; j < c->nsets; ++j) {
    for (int64_t i = 0; i < c->g[j]; ++i) block_task[grid + i] = c->first[j];
    for (int w = c->first[j]; w >= 0; w = c->next[w]) {
      b0[w] = (int)grid;
      nb[w] = (int)c->g[j];
    }
    grid += c->g[j];
  }
  for (; grid < total; ++grid) block_task[grid] = -2;
  return c->nf;
}

// The device side: the tasks' work from the previous round's updates, the
// plan written into the launch's tables (block_task; after it the list, from
// block_task[max_blocks], the next links, from block_task[max_blocks +
// TCL_PACK_MAX], and the list's length in block_task[2 max_blocks - 1]; the
// tasks' sets).
__global__ void tcl_repack_kernel(hpc_lloyd_task *tasks, int *block_task, int W, int64_t total,
                                  int64_t max_blocks, int64_t task_blocks) {
  // one thread; its arrays in shared memory rather than its stack
  __shared__ TclCand cand[2];
  __shared__ double work[TCL_PACK_MAX];
  __shared__ int64_t cap[TCL_PACK_MAX];
  __shared__ int nb[TCL_PACK_MAX], b0[TCL_PACK_MAX];
  if (threadIdx.x != 0) return;
  for (int w = 0; w < W; ++w) {
    const int64_t sw = tasks[w].s > 0 ? tasks[w].s : 1;
    work[w] = tcl_work(sw, tasks[w].k, tasks[w].uprev ? *tasks[w].uprev : 0);
    const int64_t c = (sw + TB_M - 1) / TB_M;
    cap[w] = c < task_blocks ? c : task_blocks;
  }
  const int nf = tcl_pack_core(W, work, cap, total, block_task, block_task + max_blocks,
                               block_task + max_blocks + TCL_PACK_MAX, nb, b0, cand);
  block_task[2 * max_blocks - 1] = nf;
  for (int w = 0; w < W; ++w) {
    tasks[w].block0 = b0[w];
    tasks[w].nblocks = nb[w];
  }
}

void tcl_pack(LloydLaunch &h, int64_t total) {
  double work[TCL_PACK_MAX];
  int64_t cap[TCL_PACK_MAX];
  int nb[TCL_PACK_MAX], b0[TCL_PACK_MAX];
  for (int w = 0; w < h.W; ++w) {
    const int64_t sw = std::max<int64_t>(1, h.tasks[w].s);
    work[w] = tcl_work(sw, h.tasks[w].k, 0);
    cap[w] = std::min<int64_t>((sw + TB_M - 1) / TB_M, h.task_blocks);
  }
  std::vector<TclCand> cand(2);
  h.nfollow = tcl_pack_core(h.W, work, cap, total, h.block_task_host, h.block_task_host + h.max_blocks,
                            h.block_task_host + h.max_blocks + TCL_PACK_MAX, nb, b0, cand.data());
  h.block_task_host[2 * h.max_blocks - 1] = h.nfollow;
  for (int w = 0; w < h.W; ++w) {
    h.tasks[w].block0 = b0[w];
    h.tasks[w].nblocks = nb[w];
  }
  h.grid = total;
}

template <int D, int NP>
int tcl_plan_t(const hpc_launch &L, LloydLaunch &h) {
  using Cfg = TbCfg<D, NP>;
  auto kern = tcl_lloyd_kernel<D, NP>;
  const size_t smem = Cfg::TOTAL;
  if (smem > (size_t)L.smem_optin) return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HPC_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TB_THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return HPC_ERR_UNSUPPORTED;
  // one CTA per SM: it holds the tensor memory its pipeline needs
  int64_t total = L.num_sms;
  if (total > h.max_blocks) total = h.max_blocks;
  int64_t want = 0;
  for (int w = 0; w < h.W; ++w) want += (h.tasks[w].s + TB_M - 1) / TB_M;
  if (total > want) total = want;
  if (h.W > HPC_MAX_TASKS) return HPC_ERR_UNSUPPORTED;
  h.nfollow = 0;
  if (h.W == 1) {
    h.tasks[0].block0 = 0;
    h.tasks[0].nblocks = (int)total;
    h.grid = total;
  } else {
    if (!h.pop || h.W > TCL_PACK_MAX || h.max_blocks < 2 * TCL_PACK_MAX + 2)
      return HPC_ERR_UNSUPPORTED;
    tcl_pack(h, total);
  }
  h.smem = smem;
  h.smem_sums = 0;
  h.xstage = 0;
  h.form = HPC_SEARCH_SPLIT_BF16;
  return HPC_OK;
}

template <int D, int NP>
int tcl_run_t(const hpc_launch &L, const LloydLaunch &h) {
  auto kern = tcl_lloyd_kernel<D, NP>;
  TclArgs a;
  a.W = h.W;
  a.single = h.tasks[0];
  a.tasks = h.tasks_dev;
  a.block_task = h.block_task_dev;
  a.follow = h.W > 1 ? h.block_task_dev + h.max_blocks : nullptr;
  a.nfollow = h.W > 1 ? h.block_task_dev + 2 * h.max_blocks - 1 : nullptr;
  a.next = h.W > 1 ? h.block_task_dev + h.max_blocks + TCL_PACK_MAX : nullptr;
  a.pop = h.pop;
  if (h.W > 1) {  // the plan for this round, from the previous round's updates
    tcl_repack_kernel<<<1, 32, 0, L.stream>>>(const_cast<hpc_lloyd_task *>(h.tasks_dev),
                                              const_cast<int *>(h.block_task_dev), h.W, h.grid,
                                              h.max_blocks, h.task_blocks);
    if (cudaGetLastError() != cudaSuccess) return HPC_ERR_CUDA;
  }
  a.max_iter = h.max_iter;
  a.tol = h.tol;
  a.status = h.status;
  a.round_advance = h.round_advance;
  a.stats = h.stats;
  a.queue = h.queue;
  a.queue_cap = (int)h.queue_cap;
  if (!a.queue || h.queue_cap < 1 || h.grid > h.queue_ctas) {
    a.queue = nullptr;
    a.queue_cap = 0;
  }
  void *args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)h.grid),
                                                    dim3(TB_THREADS), args, h.smem, L.stream);
  return e == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

template <int D, int NP>
int tcb_objective_t(const hpc_launch &L, const ObjArgsHost &h) {
  using Cfg = TbCfg<D, NP>;
  auto kern = tcb_objective_kernel<D, NP>;
  const size_t smem = Cfg::TOTAL;
  if (smem > (size_t)L.smem_optin) return HPC_ERR_UNSUPPORTED;
  const size_t gbytes = hpc_tcl_gcent_bytes(D, h.k);
  if (!h.cent_scratch || h.cent_scratch_bytes < (int64_t)(gbytes + 256)) return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return HPC_ERR_CUDA;
  float *gcent = reinterpret_cast<float *>(h.cent_scratch);
  float *gmeta = reinterpret_cast<float *>(h.cent_scratch + gbytes);
  tcb_prep_kernel<D><<<1, 256, 0, L.stream>>>(h.C, h.deg, h.k, gcent, gmeta);
  if (cudaGetLastError() != cudaSuccess) return HPC_ERR_CUDA;
  const int64_t ntiles = (h.n + TB_M - 1) / TB_M;
  int64_t G = L.num_sms;
  if (G > ntiles) G = ntiles;
  if (G < 1) G = 1;
  if (G > h.max_blocks) G = h.max_blocks;
  TcbArgs a;
  a.X = h.X;
  a.n = h.n;
  a.k = h.k;
  a.C = h.C;
  a.deg = h.deg;
  a.gcent = gcent;
  a.gmeta = gmeta;
  a.f_out = h.f_out;
  a.labels = h.labels;
  a.status = h.status;
  a.part = h.part;
  a.done_count = h.done_count;
  a.stats = h.stats;
  a.queue = h.queue;
  a.queue_cap = (int)h.queue_cap;
  if (!a.queue || h.queue_cap < 1 || G > h.queue_ctas) {
    a.queue = nullptr;
    a.queue_cap = 0;
  }
  kern<<<(unsigned)G, TB_THREADS, smem, L.stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

}  // namespace

bool hpc_tcl_supported(int d, int kmax) {
  return (d == 64 && kmax >= 1 && kmax <= 512) || (d == 128 && kmax >= 1 && kmax <= 256);
}

size_t hpc_tcl_gcent_bytes(int d, int k) {
  const int kp = (k + 1) & ~1;
  const int D = d <= 64 ? 64 : 128;
  return (((size_t)kp * hpc_cstride(D) * 4 + (size_t)kp * 8) + 255) & ~(size_t)255;
}

int hpc_tcl_cta_plan(int W, const int64_t *s, const int32_t *k, const int32_t *u, int64_t ctas,
                     int32_t *cta_task, int32_t *list, int32_t *nlist, int32_t *next,
                     int32_t *nblocks) {
  if (W < 1 || W > TCL_PACK_MAX || ctas < 1) return HPC_ERR_ARG;
  double work[TCL_PACK_MAX];
  int64_t cap[TCL_PACK_MAX];
  int b0[TCL_PACK_MAX];
  for (int w = 0; w < W; ++w) {
    if (s[w] < 1 || k[w] < 1) return HPC_ERR_ARG;
    work[w] = tcl_work(s[w], k[w], u ? u[w] : 0);
    cap[w] = (s[w] + TB_M - 1) / TB_M;
  }
  std::vector<TclCand> cand(2);
  *nlist = tcl_pack_core(W, work, cap, ctas, cta_task, list, next, nblocks, b0, cand.data());
  return HPC_OK;
}

int hpc_tcl_plan(const hpc_launch &L, LloydLaunch &h) {
  if (!hpc_tcl_supported(h.d, h.kmax)) return HPC_ERR_UNSUPPORTED;
  const int np = tb_np(h.kmax);
  if (h.d == 64) {
    if (np == 128) return tcl_plan_t<64, 128>(L, h);
    if (np == 256) return tcl_plan_t<64, 256>(L, h);
    return tcl_plan_t<64, 512>(L, h);
  }
  if (np == 128) return tcl_plan_t<128, 128>(L, h);
  return tcl_plan_t<128, 256>(L, h);
}

int hpc_tcl_run(const hpc_launch &L, const LloydLaunch &h) {
  const int np = tb_np(h.kmax);
  if (h.d == 64) {
    if (np == 128) return tcl_run_t<64, 128>(L, h);
    if (np == 256) return tcl_run_t<64, 256>(L, h);
    return tcl_run_t<64, 512>(L, h);
  }
  if (np == 128) return tcl_run_t<128, 128>(L, h);
  return tcl_run_t<128, 256>(L, h);
}

int hpc_tcb_objective_launch(const hpc_launch &L, const ObjArgsHost &h) {
  if (!hpc_tcl_supported(h.d, h.k) || h.n < 1) return HPC_ERR_UNSUPPORTED;
  const int np = tb_np(h.k);
  if (h.d == 64) {
    if (np == 128) return tcb_objective_t<64, 128>(L, h);
    if (np == 256) return tcb_objective_t<64, 256>(L, h);
    return tcb_objective_t<64, 512>(L, h);
  }
  if (np == 128) return tcb_objective_t<128, 128>(L, h);
  return tcb_objective_t<128, 256>(L, h);
}
