// Full-data objective (Eq. 1) with the x.c contraction on the tensor cores.
//
// The search is the nearest-centroid argmin of ||c||^2 - 2 x.c.  Its dot
// products run as tcgen05 TF32 MMAs (8-wide K steps): the A operand is the
// FP32 row tile exactly as TMA staged it (the tensor core reads its TF32
// part), B holds c' = -2c cut to TF32 (10 explicit mantissa bits), FP32
// accumulation in TMEM.  Each factor is within 2^-10 of its value, so every
// computed ||c||^2 - 2 x.c lies within E = 2^-10 (||x|| + max||c||)^2 of the
// exact one (2^-9 sum_t |x_t c'_t| <= 2^-10 (||x|| + ||c||)^2, plus FP32
// accumulation far below it).  A row whose top-2 margin exceeds 2E has the
// exact nearest centroid.  Otherwise its two nearest candidates are
// computed exactly (FP32 direct form, relative error <= (D + 3) u); every
// other centroid is at least ||x||^2 + d2 - E away, which settles almost
// all rows; the rest take every candidate within the window exactly, and
// rows still unresolved are rescored by the warp in FP64 (ties to the lowest
// index).  The objective adds the FP32 direct-form distance to the chosen
// centroid, from the exact row, in FP64.
//
// The bound is wide (2^-10 relative to ||x|| ||c||), so this search suits
// data whose cluster margins are large next to it: large d, where the SIMT
// form runs out of registers.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0       TMA producer: 128-row x 32-float (or 16-float) chunks of
//                the row tiles into a ring sized to the shared memory left
//   warp 1       TMEM owner and MMA issuer (one thread); each chunk's commit
//                frees its ring slot as soon as the MMAs have read it
//   warps 2..17  four epilogue warpgroups: TMEM -> registers, top-2, margin
//                test, exact rescoring, direct distance, labels
// Every mbarrier wait is bounded; a wait that runs out records
// HPC_ERR_TIMEOUT, every role stops, in-flight copies and MMAs are drained,
// TMEM is freed and the kernel returns.
#include "assign.cuh"
#include "kernels.h"
#include "tc.cuh"
#include "tc_rows.cuh"

namespace {

constexpr int TC_M = 128;
constexpr int TC_NEPI = 4;  // epilogue warpgroups
constexpr int TC_EPI0 = 2;  // first epilogue warp
constexpr int TC_WARPS = TC_EPI0 + 4 * TC_NEPI;
constexpr int TC_THREADS = TC_WARPS * 32;
constexpr int TC_MAX_RING = 16;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;
constexpr uint64_t TC_DRAIN_NS = 500000000ull;

template <int D>
struct TcCfg {
  static constexpr int CK = D < 32 ? D : 32;  // floats per swizzled chunk row
  static constexpr int NCH = D / CK;          // chunks per tile
  static constexpr uint32_t RB = CK * 4;      // bytes per chunk row (64 or 128)
  static constexpr uint32_t SWZ = RB == 128 ? 2u : 4u;
  static constexpr uint32_t CHUNK_BYTES = TC_M * RB;
  static constexpr bool XREG = D <= 32;  // the epilogue keeps the row in registers
};

// TMEM accumulator slots of NP columns (at most 512 columns in all)
template <int NP>
struct TcSlots {
  static constexpr int N = NP <= 32 ? 8 : 4;
  static constexpr int COLS = N * NP;
};

// Shared-memory layout: ring, B operand, exact centroid block, norms, barriers.
template <int D, int NP>
struct TcSmem {
  __host__ __device__ static size_t bop(int nsx) { return (size_t)nsx * TcCfg<D>::CHUNK_BYTES; }
  __host__ __device__ static size_t cent(int nsx) {
    return bop(nsx) + (size_t)TcCfg<D>::NCH * NP * TcCfg<D>::RB;
  }
  __host__ __device__ static size_t norms(int nsx, int k) {
    return cent(nsx) + ((hpc_cent_smem_bytes(D, k) + 15) & ~(size_t)15);
  }
  __host__ __device__ static size_t bars(int nsx, int k) { return norms(nsx, k) + (size_t)NP * 4; }
  // + 1024 for aligning the base
  __host__ __device__ static size_t total(int nsx, int k) {
    return bars(nsx, k) + (size_t)(2 * nsx + 2 * TcSlots<NP>::N + 1) * 8 + 16 + 1024;
  }
};

struct TcArgs {
  int64_t n;
  int d, k, nsx;
  const float *X;
  const float *C;
  const uint8_t *deg;
  double *f_out;
  int32_t *labels;
  int *status;
  double *part;
  unsigned *done_count;
};

template <int D, int NP, int IB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_objective_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  using Cfg = TcCfg<D>;
  using L = TcSmem<D, NP>;
  constexpr int NSL = TcSlots<NP>::N;
  constexpr int NCH = Cfg::NCH;
  constexpr int CS = hpc_cstride(D);
  const int nsx = a.nsx;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float s_red[2];
  __shared__ double s_dsum[32];
  __shared__ bool s_last;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  unsigned char *base =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *ring = base;               // row-tile chunks as TMA stages them
  unsigned char *bop = base + L::bop(nsx);  // B operand: TF32 c'
  hpc_cent_smem cs;
  hpc_cent_bind(cs, base + L::cent(nsx), D, a.k);
  float *cnv = reinterpret_cast<float *>(base + L::norms(nsx, a.k));  // NP norms
  uint64_t *xfull = reinterpret_cast<uint64_t *>(base + L::bars(nsx, a.k));
  uint64_t *xfree = xfull + nsx;
  uint64_t *accf = xfree + nsx;
  uint64_t *acce = accf + NSL;
  uint64_t *drain = acce + NSL;
  volatile int *abort = &s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = a.n;
  const int64_t ntiles = (n + TC_M - 1) / TC_M;
  const int my_tiles =
      (int)(blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);

  // ---- set-up: exact centroids, MMA operand B, barriers, TMEM ----
  hpc_load_centroids<D>(cs, a.C, a.deg, a.k, a.d, s_red);
  for (int j = threadIdx.x; j < NP; j += TC_THREADS) cnv[j] = j < cs.kp ? cs.cnz[j].x : HPC_DEAD;
  for (int e = threadIdx.x; e < NP * D; e += TC_THREADS) {
    const int j = e / D, t = e - j * D;
    const float c = j < cs.kp ? cs.cm[j * CS + t] : 0.0f;  // -2c, zero padded
    const uint32_t off = (uint32_t)(t / Cfg::CK) * NP * Cfg::RB +
                         hpc_swz_offset((uint32_t)j, (uint32_t)(t % Cfg::CK) * 4u, Cfg::RB);
    *reinterpret_cast<float *>(bop + off) = __uint_as_float(__float_as_uint(c) & 0xFFFFE000u);
  }
  hpc_fence_proxy_async();
  if (threadIdx.x == 0) {
    for (int s = 0; s < nsx; ++s) {
      hpc_mbar_init(&xfull[s], 1);
      hpc_mbar_init(&xfree[s], 1);
    }
    for (int s = 0; s < NSL; ++s) {
      hpc_mbar_init(&accf[s], 1);
      hpc_mbar_init(&acce[s], 128);
    }
    hpc_mbar_init(drain, 1);
    s_abort = 0;
    hpc_fence_barrier_init();
  }
  if (warp == 1) hpc_tmem_alloc(&s_tmem, TcSlots<NP>::COLS);
  hpc_tc_fence_before();
  __syncthreads();
  hpc_tc_fence_after();
  const uint32_t tmem = s_tmem;
  const bool run = cs.live > 0;
  if (!run && n > 0 && threadIdx.x == 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);

  double fsum = 0.0;
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
          if (ph > 0 && !hpc_mbar_wait(&xfree[s], (ph - 1) & 1, abort, a.status, TC_WAIT_NS)) {
            ok = false;
            break;
          }
          hpc_mbar_arrive_expect_tx(&xfull[s], Cfg::CHUNK_BYTES);
          hpc_tma_load_2d(ring + (size_t)s * Cfg::CHUNK_BYTES, &tmap, &xfull[s], ch * Cfg::CK,
                          (int)(tg * TC_M));
          issued = u + 1;
        }
      }
      // every copy issued must have landed before the block can exit
      int no_abort = 0;
      for (int u = issued > nsx ? issued - nsx : 0; u < issued; ++u)
        hpc_mbar_wait(&xfull[u % nsx], (u / nsx) & 1, (volatile int *)&no_abort, a.status,
                      TC_DRAIN_NS);
    }
    __syncwarp();
  } else if (run && warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      constexpr uint32_t idesc = hpc_umma_idesc(2u, 2u, NP, TC_M);
      const uint32_t sbo = 8u * Cfg::RB;
      const uint32_t B = hpc_smem_u32(bop);
      bool ok = true;
      for (int i = 0; i < my_tiles && ok; ++i) {
        const int sl = i % NSL, v = i / NSL;
        if (v > 0 && !hpc_mbar_wait(&acce[sl], (v - 1) & 1, abort, a.status, TC_WAIT_NS)) break;
        const uint32_t dt = tmem + (uint32_t)(sl * NP);
        for (int ch = 0; ch < NCH; ++ch) {
          const int u = i * NCH + ch, s = u % nsx, ph = u / nsx;
          if (!hpc_mbar_wait(&xfull[s], ph & 1, abort, a.status, TC_WAIT_NS)) {
            ok = false;
            break;
          }
          hpc_tc_fence_after();
          const uint32_t A = hpc_smem_u32(ring + (size_t)s * Cfg::CHUNK_BYTES);
#pragma unroll
          for (int ks = 0; ks < Cfg::CK / 8; ++ks) {
            const uint64_t ad = hpc_umma_desc(A + (uint32_t)ks * 32u, 16u, sbo, Cfg::SWZ);
            const uint64_t bd = hpc_umma_desc(
                B + (uint32_t)ch * (uint32_t)NP * Cfg::RB + (uint32_t)ks * 32u, 16u, sbo, Cfg::SWZ);
            hpc_mma_tf32(dt, ad, bd, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
          }
          hpc_mma_commit(&xfree[s]);  // the slot may be refilled once these MMAs are done
        }
        if (ok) hpc_mma_commit(&accf[sl]);
      }
      // no MMA may still run when TMEM is freed
      hpc_mma_commit(drain);
      int no_abort = 0;
      hpc_mbar_wait(drain, 0, (volatile int *)&no_abort, a.status, TC_DRAIN_NS);
    }
    __syncwarp();
  } else if (run) {
    // ---- epilogue warpgroups ----
    const int eg = (warp - TC_EPI0) / 4, q = warp & 3;
    const int r_in = 32 * q + lane;
    for (int i = eg; i < my_tiles; i += TC_NEPI) {
      const int sl = i % NSL, v = i / NSL;
      const int64_t tg = blockIdx.x + (int64_t)i * gridDim.x;
      const int64_t row = tg * TC_M + r_in;
      bool valid = row < n;
      RowRef<D> xr;
      xr.g = a.X + (valid ? row : 0) * a.d;
      if constexpr (Cfg::XREG) {  // fetched (L2) while the MMA runs
        if (valid) {
          hpc_load_row<D>(xr.x, xr.g, a.d);
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t) xr.x[t] = 0.0f;
        }
      }
      if (!wait_warp(&accf[sl], v & 1, abort, a.status, TC_WAIT_NS)) break;
      hpc_tc_fence_after();
      // top-2 over the NP columns as two independent chains (even / odd
      // columns), merged at the end
      float d1 = __int_as_float(0x7f7fffff), d2 = d1, e1 = d1, e2 = d1;
      int j1 = 0, j2 = 0, je = 1, je2 = 1;
#pragma unroll
      for (int c = 0; c < NP / 32; ++c) {
        if (c * 32 >= cs.kp) break;
        float acc[32];
        hpc_tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(sl * NP + c * 32), acc);
#pragma unroll
        for (int jj = 0; jj < 32; jj += 4) {
          if (c * 32 + jj >= cs.kp) break;  // past the last centroid (same for the whole warp)
          const float4 cn = *reinterpret_cast<const float4 *>(cnv + c * 32 + jj);
          const float v0 = cn.x + acc[jj], v1 = cn.y + acc[jj + 1];
          const float v2 = cn.z + acc[jj + 2], v3 = cn.w + acc[jj + 3];
          const int j = c * 32 + jj;
          if constexpr (IB > 0) {
            hpc_top2_fold4(d1, d2, hpc_key_b<IB>(v0, j), hpc_key_b<IB>(v1, j + 1),
                           hpc_key_b<IB>(v2, j + 2), hpc_key_b<IB>(v3, j + 3));
          } else {
#define HPC_TOP2_STEP(V, J, A1, B1, A2, B2) \
  if (V < A1) {                             \
    A2 = A1;                                \
    B2 = B1;                                \
    A1 = V;                                 \
    B1 = J;                                 \
  } else if (V < A2) {                      \
    A2 = V;                                 \
    B2 = J;                                 \
  }
            HPC_TOP2_STEP(v0, j, d1, j1, d2, j2)
            HPC_TOP2_STEP(v1, j + 1, e1, je, e2, je2)
            HPC_TOP2_STEP(v2, j + 2, d1, j1, d2, j2)
            HPC_TOP2_STEP(v3, j + 3, e1, je, e2, je2)
#undef HPC_TOP2_STEP
          }
        }
      }
      if constexpr (IB > 0) {
        const float lo = fminf(d1, e1);
        d2 = fminf(fmaxf(d1, e1), fminf(d2, e2));
        d1 = lo;
        j1 = min(__float_as_int(d1) & ((1 << IB) - 1), cs.kp - 1);
        j2 = min(__float_as_int(d2) & ((1 << IB) - 1), cs.kp - 1);
      } else {
        // merge (d1 j1, d2 j2) with (e1 je, e2 je2); lower index on equal values
        float m1, m2;
        int i1, i2;
        if (e1 < d1 || (e1 == d1 && je < j1)) {
          m1 = e1;
          i1 = je;
          if (d1 < e2 || (d1 == e2 && j1 < je2)) {
            m2 = d1;
            i2 = j1;
          } else {
            m2 = e2;
            i2 = je2;
          }
        } else {
          m1 = d1;
          i1 = j1;
          if (e1 < d2 || (e1 == d2 && je < j2)) {
            m2 = e1;
            i2 = je;
          } else {
            m2 = d2;
            i2 = j2;
          }
        }
        d1 = m1;
        j1 = i1;
        d2 = m2;
        j2 = i2;
      }
      const bool found = d1 < HPC_DEAD * 0.5f;
      if (!found) j1 = 0;
      // every value is within E of the exact ||c||^2 - 2 x.c; keys add at
      // most 2^-18 |v|
      float nx, dd;
      if constexpr (Cfg::XREG) {
        nx = valid ? row_norm2<D>(xr) : 0.0f;
        dd = valid ? row_direct<D>(xr, cs.cm + j1 * CS) : 0.0f;
      } else {
        // rows of 256 / 512 bytes: the warp reads each of its 32 rows with
        // coalesced loads and reduces ||x||^2 and the direct distance to the
        // row's chosen centroid across its lanes
        warp_norm_direct<D>(a.X, tg * TC_M + 32 * q, valid, j1, cs, nx, dd);
      }
      const float rad = sqrtf(nx) * 1.0001f + cs.cmax * 1.0001f;
      float win = 2.0f * 9.765625e-04f * rad * rad;  // 2E, E = 2^-10 (||x|| + max||c||)^2
      if (IB > 0) win += 1.0001f * ldexpf(1.0f, IB - 22) * (fabsf(d1) + fabsf(d2));  // keys
      const bool ok = found && isfinite(nx) && isfinite(win);
      if (valid && !ok) {
        hpc_status_set(a.status, HPC_ERR_NONFINITE);
        valid = false;
      }
      const bool flag = valid && !(d2 - d1 > win);
      bool need64 = false, need_window = false;
      constexpr float rho = (float)(D + 3) * HPC_U32 * 1.001f;  // FP32 direct-form bound
      if (flag) {
        // the two nearest by the tensor-core values, exactly; every other
        // centroid is at least ||x||^2 + d2 - E away
        const float ex2 = row_direct<D>(xr, cs.cm + j2 * CS);
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
        // a third centroid may win: every candidate within the window, exactly
        const float thr = d1 + win;
        float b1 = __int_as_float(0x7f800000), b2 = b1;
        int bj = j1;
#pragma unroll
        for (int c = 0; c < NP / 32; ++c) {
          if (c * 32 >= cs.kp) break;
          float acc[32];
          hpc_tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(sl * NP + c * 32), acc);
#pragma unroll 4
          for (int jj = 0; jj < 32; ++jj) {
            const int j = c * 32 + jj;
            if (need_window && j < cs.kp && cnv[j] + acc[jj] <= thr) {
              const float e = row_dist32<D>(xr, cs.cm + j * CS);
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
        if (need_window) {
          if (b2 - b1 > rho * (b1 + b2)) {
            j1 = bj;
            dd = row_direct<D>(xr, cs.cm + j1 * CS);
          } else {
            need64 = true;
          }
        }
      }
      hpc_tc_fence_before();
      hpc_mbar_arrive(&acce[sl]);
      // unresolved by FP32: the warp rescores in FP64 (ties to the lowest index)
      unsigned m = __ballot_sync(0xffffffffu, need64);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int64_t ri = tg * TC_M + 32 * q + src;
        const int j = hpc_rescore_row<D>(a.X + ri * a.d, a.d, cs);
        if (lane == src && j != j1) {
          j1 = j;
          dd = row_direct<D>(xr, cs.cm + j1 * CS);
        }
      }
      if (valid && !isfinite(dd)) {
        hpc_status_set(a.status, HPC_ERR_NONFINITE);
        valid = false;
      }
      if (valid) {
        fsum += (double)dd;
        if (a.labels) a.labels[row] = j1;
      }
    }
  }

  // ---- objective partial, last block reduces in a fixed order ----
  const double bsum = hpc_block_sum(fsum, s_dsum);
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
    hpc_tmem_dealloc(tmem, TcSlots<NP>::COLS);
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
int tc_launch_t(const hpc_launch &Lc, const ObjArgsHost &h) {
  using Cfg = TcCfg<D>;
  using L = TcSmem<D, NP>;
  auto kern = tc_objective_kernel<D, NP, IB>;
  // as many ring slots as the shared memory allows (2 .. 16, and at least a
  // full tile); at least 120 KB requested so that one block fills an SM
  int nsx = TC_MAX_RING;
  while (nsx > 2 && L::total(nsx, h.k) > (size_t)Lc.smem_optin) --nsx;
  if (L::total(nsx, h.k) > (size_t)Lc.smem_optin || nsx < Cfg::NCH) return HPC_ERR_UNSUPPORTED;
  size_t smem = L::total(nsx, h.k);
  if (smem < 120 * 1024) smem = 120 * 1024;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return HPC_ERR_UNSUPPORTED;
  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)h.d, (cuuint64_t)h.n};
  cuuint64_t gstride[1] = {(cuuint64_t)h.d * 4};
  cuuint32_t box[2] = {(cuuint32_t)Cfg::CK, (cuuint32_t)TC_M};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle swz =
      Cfg::RB == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(h.X), gdim, gstride, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HPC_ERR_CUDA;
  const int64_t ntiles = (h.n + TC_M - 1) / TC_M;
  int64_t G = Lc.num_sms;
  if (G > ntiles) G = ntiles;
  if (G < 1) G = 1;
  if (G > h.max_blocks) G = h.max_blocks;
  TcArgs a;
  a.n = h.n;
  a.d = h.d;
  a.k = h.k;
  a.nsx = nsx;
  a.X = h.X;
  a.C = h.C;
  a.deg = h.deg;
  a.f_out = h.f_out;
  a.labels = h.labels;
  a.status = h.status;
  a.part = h.part;
  a.done_count = h.done_count;
  kern<<<(unsigned)G, TC_THREADS, smem, Lc.stream>>>(map, a);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

// (value, index) keys with 5 index bits for k <= 32, 7 above: the keys'
// error (2^-16 relative at 7 bits) is far inside the TF32 products' window
template <int D>
int tc_dispatch(const hpc_launch &L, const ObjArgsHost &h) {
  if (h.k <= 32) return tc_launch_t<D, 32, 5>(L, h);
  if (h.k <= 64) return tc_launch_t<D, 64, 7>(L, h);
  return tc_launch_t<D, 128, 7>(L, h);
}

}  // namespace

bool hpc_tc_objective_supported(int d, int k, int64_t n) {
  if (k > 128) return hpc_tc_wide_supported(d, k, n);
  return n >= 1 && (d == 16 || d == 32 || d == 64 || d == 128) && k >= 1;
}

int hpc_tc_objective_launch(const hpc_launch &L, const ObjArgsHost &h) {
  if (!hpc_tc_objective_supported(h.d, h.k, h.n)) return HPC_ERR_UNSUPPORTED;
  if (h.k > 128) return hpc_tc_wide_launch(L, h);
  switch (h.d) {
    case 16: return tc_dispatch<16>(L, h);
    case 32: return tc_dispatch<32>(L, h);
    case 64: return tc_dispatch<64>(L, h);
    default: return tc_dispatch<128>(L, h);
  }
}
