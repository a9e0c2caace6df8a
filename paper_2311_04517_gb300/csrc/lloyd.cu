// Lloyd's K-means on one sample (Algorithm 1; stop rule of Section 6.5) as
// one persistent cooperative kernel, and the full-data objective of Eq. 1.
//
// Lloyd: one bounded grid barrier per iteration.  Phase A assigns this
// block's rows (hpc_assign_group), then the warp re-reads its rows with lanes
// mapped to dimensions and adds every coordinate, on an exact 64-bit
// fixed-point grid, into per-block shared-memory sums (lanes of one pass hit
// different dimensions, so they do not collide); the block flushes its sums
// with integer atomics into a global buffer.  Integer sums make the result
// independent of the order of the additions.  After the barrier every block
// reads the same sums and objective partials, takes the same stop decision
// and computes the same new centroids (no second barrier).  The global sum
// buffers rotate over three slots so that zeroing never races a reader.
#include <vector>

#include "assign.cuh"
#include "kernels.h"
#include "round.cuh"

namespace {

struct LloydArgs {
  int W;
  hpc_lloyd_task single;        // W == 1
  const hpc_lloyd_task *tasks;  // W > 1 (device)
  const int *block_task;        // W > 1: task of every block (device)
  int d;
  int max_iter;
  double tol;
  int *status;
  int smem_sums;  // 1: per-block sums in shared memory
  int xstage;     // 1: the block's rows are kept in shared memory for the accumulation
  uint32_t *round_advance;  // nullable: a prepared round's counter (see the kernel's start)
};

// Objective: several rows per thread amortise the centroid reads.
template <int D>
struct Tile {
  static constexpr int R = D <= 4 ? 8 : D <= 16 ? 4 : D <= 64 ? 2 : 1;
  static constexpr int THREADS = 256;
};

// Lloyd: samples are small (10^4 - 10^6 rows): one or two rows per thread
// spread an iteration over every SM (two at d <= 64: every centroid read
// from shared memory serves two rows; at d = 16 a 10^5-row sample then takes
// one row group per block); the accumulation maps lanes to dimensions.
template <int D>
struct LTile {
  static constexpr int R = D <= 64 ? 2 : 1;
  static constexpr int THREADS = 256;
  static constexpr int MINB = D <= 32 ? 2 : 1;
  static constexpr int LPR = D < 32 ? D : 32;          // lanes per row
  static constexpr int RPP = 32 / LPR;                 // rows per pass
  static constexpr int TPL = (D + LPR - 1) / LPR;      // dimensions per lane
  static constexpr int NB = TPL >= 4 ? 4 : 8;          // rows per batch of loads
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared-memory layout of the Lloyd kernel: centroid block, flags, labels,
// optionally the block's k x d sums and counts, optionally the block's rows
// (R x THREADS rows of hpc_cstride(D) floats) for the accumulation.
struct LloydSmem {
  size_t cent, dead, lab, sums, cnt, xs, total;
  __host__ __device__ LloydSmem(int D, int R, int THREADS, int k, int d, bool smem_sums, bool xstage) {
    const int kp = (k + 1) & ~1;
    cent = 0;
    dead = align16(hpc_cent_smem_bytes(D, k));
    lab = dead + align16((size_t)kp);
    sums = lab + align16((size_t)R * THREADS * 4);
    cnt = sums + (smem_sums ? align16((size_t)k * d * 8) : 0);
    xs = cnt + (smem_sums ? align16((size_t)k * 4) : 0);
    total = xs + (xstage ? align16((size_t)R * THREADS * hpc_cstride(D) * 4) : 0);
  }
};

template <int D, int R, int THREADS, int IB>
__global__ void __launch_bounds__(THREADS, LTile<D>::MINB) lloyd_kernel(LloydArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_red[2];
  __shared__ double s_dsum[32];
  __shared__ double s_f;
  __shared__ int s_done;
  __shared__ unsigned s_umax, s_cmax;
  constexpr int LPR = LTile<D>::LPR, RPP = LTile<D>::RPP, TPL = LTile<D>::TPL, NB = LTile<D>::NB;

  // The round's last launch moves a prepared round's counter on: every
  // reader of the round index (sampling, K-means++) ran in earlier launches,
  // and Lloyd itself does not read it.
  if (a.round_advance && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.round_advance, 1u);
  // this block's task (one worker's sample) and its place in the task's group
  const hpc_lloyd_task tk = a.W == 1 ? a.single : a.tasks[a.block_task[blockIdx.x]];
  const int k = tk.k, d = a.d;
  const int64_t s = tk.s;
  const int G = tk.nblocks, lb = (int)blockIdx.x - tk.block0;
  const LloydSmem L(D, R, THREADS, k, d, a.smem_sums != 0, a.xstage != 0);
  hpc_cent_smem cs;
  hpc_cent_bind(cs, smem_raw, D, k);
  uint8_t *dead = smem_raw + L.dead;
  int *wlab = reinterpret_cast<int *>(smem_raw + L.lab);
  unsigned long long *ssum = reinterpret_cast<unsigned long long *>(smem_raw + L.sums);
  unsigned *scnt = reinterpret_cast<unsigned *>(smem_raw + L.cnt);
  float *xs = reinterpret_cast<float *>(smem_raw + L.xs);
  constexpr int XS = hpc_cstride(D);

  const int64_t TR = (int64_t)THREADS * R;
  const int64_t ngroups = (s + TR - 1) / TR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Phase 0: largest |x| of the sample (sets the fixed-point grid and
  // detects non-finite rows: NaN/inf bit patterns compare above finite).
  if (threadIdx.x == 0) s_umax = s_cmax = 0u;
  for (int j = threadIdx.x; j < cs.kp; j += THREADS) dead[j] = (j >= k) || tk.deg[j] != 0;
  // sum slots 0 and 1 start at zero (slot 2 is cleared in iteration 0)
  for (int64_t e = (int64_t)lb * THREADS + threadIdx.x; e < 2ll * k * d; e += (int64_t)G * THREADS)
    tk.gsum[e] = 0ull;
  for (int e = lb * THREADS + threadIdx.x; e < 2 * k; e += G * THREADS) tk.gcount[e] = 0u;
  __syncthreads();
  {
    unsigned m = 0u;
    for (int64_t g = lb; g < ngroups; g += G) {
      const int64_t e1 = min((g + 1) * TR, s) * d;
      for (int64_t e = g * TR * d + threadIdx.x; e < e1; e += THREADS) {
        const unsigned b = __float_as_uint(tk.S[e]) & 0x7fffffffu;
        m = b > m ? b : m;
      }
    }
    atomicMax(&s_umax, m);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(tk.gmaxabs, s_umax);
  }
  constexpr int CS = hpc_cstride(D);
  {
    unsigned m = 0u;  // largest |c| of the live starting centroids
    for (int e = threadIdx.x; e < cs.kp * CS; e += THREADS) {
      const int j = e / CS, t = e - j * CS;
      const float c = (j < k && t < d) ? tk.C[(int64_t)j * d + t] : 0.0f;
      cs.cm[e] = -2.0f * c;
      if (!dead[j]) {
        const unsigned b = __float_as_uint(c) & 0x7fffffffu;
        m = b > m ? b : m;
      }
    }
    atomicMax(&s_cmax, m);
  }
  __syncthreads();
  hpc_cent_finish<D>(cs, k, s_red, [&](int j) { return dead[j] != 0; });
  if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
  const unsigned mabs = __ldcg(tk.gmaxabs);
  if (mabs >= 0x7f800000u) {
    hpc_status_set(a.status, HPC_ERR_NONFINITE);
    return;
  }
  if (cs.live == 0) {
    hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);
    return;
  }
  // grid 2^Fs with |q| < 2^(62 - bitlen(s)) so that any sum of s values fits
  int Fs = 126;
  if (mabs != 0u) Fs = min(126, 62 - hpc_bit_length(s) - hpc_frexp_exp(__uint_as_float(mabs)));
  const float qscale = hpc_pow2f(Fs);
  // the sample objective as an integer sum on the grid 2^-Fo: with M the
  // largest |x| or starting |c| (later centroids are means of rows, so M
  // bounds them too) every distance is at most d (2M)^2, and with a factor
  // 2 of slack the s rows fit 2^62.  Blocks add their rounded partials and
  // every block reads back the one word (the same f everywhere, in any
  // order of arrival).  The sample has no inf/NaN here; the starting
  // centroids are the caller's, and one of them being non-finite is an error.
  const unsigned mc = s_cmax;
  if (mc >= 0x7f800000u) {
    hpc_status_set(a.status, HPC_ERR_NONFINITE);
    return;
  }
  // (in integers: s 8 d M^2 < 2^(bitlen(s) + 3 + bitlen(d) + 2 e(M)))
  int Fo = 126;
  {
    const unsigned mm = max(mabs, mc);
    if (mm != 0u)
      Fo = min(126, 59 - hpc_bit_length(s) - hpc_bit_length(d) - 2 * hpc_frexp_exp(__uint_as_float(mm)));
    Fo = max(Fo, -126);
  }
  const float oscale = hpc_pow2f(Fo);
  const double oinv = hpc_pow2d(-Fo);

  double f_prev = 0.0;
  for (int it = 0;; ++it) {
    const int buf = it % 3;
    unsigned long long *gs = tk.gsum + (size_t)buf * k * d;
    unsigned *gc = tk.gcount + (size_t)buf * k;
    unsigned long long *acc_sum = a.smem_sums ? ssum : gs;
    unsigned *acc_cnt = a.smem_sums ? scnt : gc;
    if (a.smem_sums) {
      for (int e = threadIdx.x; e < k * d; e += THREADS) ssum[e] = 0ull;
      for (int j = threadIdx.x; j < k; j += THREADS) scnt[j] = 0u;
    }
    __syncthreads();
    // Phase A: assignment, then accumulation with lanes over dimensions
    float fp_hi = 0.0f, fp_lo = 0.0f;  // this thread's rows' distances (TwoSum pair)
    for (int64_t g = lb; g < ngroups; g += G) {
      const int64_t base = g * TR;
      int lab[R];
      bool valid[R];
      float x[R][D];
      hpc_sum2_add(fp_hi, fp_lo,
                   hpc_assign_group_x<D, R, THREADS, IB>(tk.S, s, d, base, cs, x, lab, valid,
                                                         a.status));
#pragma unroll
      for (int r = 0; r < R; ++r) {
        wlab[r * THREADS + threadIdx.x] = valid[r] ? lab[r] : -1;
        if (valid[r] && tk.labels) tk.labels[base + (int64_t)r * THREADS + threadIdx.x] = lab[r];
        if (a.xstage) {  // the row, for this warp's accumulation below
          float *xr = xs + (size_t)(r * THREADS + threadIdx.x) * XS;
          if constexpr (D % 4 == 0) {  // XS = D + 4: rows start on 16 bytes
#pragma unroll
            for (int t = 0; t < D; t += 4)
              *reinterpret_cast<float4 *>(xr + t) =
                  make_float4(x[r][t], x[r][t + 1], x[r][t + 2], x[r][t + 3]);
          } else {
#pragma unroll
            for (int t = 0; t < D; ++t) xr[t] = x[r][t];
          }
        }
      }
      __syncwarp();
      // lane (rsub, t0) takes dimensions t0, t0 + LPR, ... of rows
      // rsub, rsub + RPP, ...; NB rows' loads are issued before their atomics
      const int t0 = lane % LPR, rsub = lane / LPR;
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const int64_t row0 = base + (int64_t)r * THREADS + warp * 32;
        const int *wl = wlab + r * THREADS + warp * 32;
#pragma unroll 1
        for (int b0 = 0; b0 < 32 / RPP; b0 += NB) {
          int jj[NB];
          float v[NB][TPL];
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int rr = rsub + RPP * (b0 + i);
            jj[i] = (b0 + i < 32 / RPP) ? wl[rr] : -1;
            const float *xr = a.xstage ? xs + (size_t)(r * THREADS + warp * 32 + rr) * XS
                                       : tk.S + (row0 + rr) * d;
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
              const int t = t0 + u * LPR;
              v[i][u] = (jj[i] >= 0 && jj[i] < k && t < d) ? xr[t] : 0.0f;
            }
          }
#pragma unroll
          for (int i = 0; i < NB; ++i) {
            const int j = jj[i];
            if (j < 0 || j >= k) continue;
#pragma unroll
            for (int u = 0; u < TPL; ++u) {
              const int t = t0 + u * LPR;
              if (t < d)
                atomicAdd(&acc_sum[(size_t)j * d + t],
                          (unsigned long long)__float2ll_rn(v[i][u] * qscale));
            }
            if (t0 == 0) atomicAdd(&acc_cnt[j], 1u);
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (a.smem_sums) {
      for (int e = threadIdx.x; e < k * d; e += THREADS)
        if (ssum[e] != 0ull) atomicAdd(&gs[e], ssum[e]);
      for (int j = threadIdx.x; j < k; j += THREADS)
        if (scnt[j] != 0u) atomicAdd(&gc[j], scnt[j]);
    }
    // the thread's partial on the grid 2^-Fo, summed over the block in
    // integers: no FP64 instruction per thread
    const unsigned long long bq = hpc_block_sum_u64(
        (unsigned long long)(__float2ll_rn(fp_hi * oscale) + __float2ll_rn(fp_lo * oscale)),
        reinterpret_cast<unsigned long long *>(s_dsum));
    if (threadIdx.x == 0 && bq != 0ull) atomicAdd(tk.gobj + buf, bq);
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;

    // Phase B (every block): objective, stop test (thread 0), new centroids
    if (threadIdx.x == 0) {
      const double fo = (double)(long long)__ldcg(tk.gobj + buf) * oinv;
      s_f = fo;
      s_done = (it > 0 && (f_prev == 0.0 || (f_prev - fo) < a.tol * f_prev)) || it == a.max_iter;
    }
    __syncthreads();
    const double f = s_f;
    const bool done = s_done != 0;
    if (done) {
      if (lb == 0) {
        if (threadIdx.x == 0) {
          *tk.f_out = f;
          if (tk.iters_out) *tk.iters_out = it;
        }
        if (tk.fhat) hpc_incumbent_block(tk, d, f, it);  // block-uniform branch
      }
      return;
    }
    for (int e = threadIdx.x; e < k * CS; e += THREADS) {
      const int j = e / CS, t = e - j * CS;
      if (dead[j] || t >= d) continue;
      const unsigned cnt = __ldcg(gc + j);
      if (cnt == 0u) {  // emptied: degenerate for the rest of the run
        // (every thread of centroid j sees cnt == 0 and skips it, so the
        // flag written here changes no other thread's work in this loop)
        if (t == 0) {
          dead[j] = 1;
          if (lb == 0) tk.deg[j] = 1;
        }
        continue;
      }
      const long long q = (long long)__ldcg(gs + (size_t)j * d + t);
      const float v = hpc_mean_f32(q, cnt, Fs);
      cs.cm[e] = -2.0f * v;
      if (lb == 0) tk.C[(int64_t)j * d + t] = v;
    }
    if (lb == 0) {  // recycle the slot read two iterations ago
      const int zb = (it + 2) % 3;
      for (int e = threadIdx.x; e < k * d; e += THREADS) tk.gsum[(size_t)zb * k * d + e] = 0ull;
      for (int j = threadIdx.x; j < k; j += THREADS) tk.gcount[(size_t)zb * k + j] = 0u;
      if (threadIdx.x == 0) tk.gobj[zb] = 0ull;
    }
    __syncthreads();
    hpc_cent_finish<D>(cs, k, s_red, [&](int j) { return dead[j] != 0; });
    f_prev = f;
  }
}

// Full-data objective: grid-stride over row groups, per-thread FP32 TwoSum
// partial, FP64 per-block partial, the last block to finish sums the
// partials in a fixed order.
struct ObjArgs {
  const float *X;
  int64_t n;
  int d, k;
  const float *C;
  const uint8_t *deg;
  double *f_out;
  int32_t *labels;
  int *status;
  double *part;
  unsigned *done_count;
};

template <int D, int R, int THREADS, int IB>
__global__ void __launch_bounds__(THREADS, D <= 16 ? 2 : 1) objective_kernel(ObjArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float s_red[2];
  __shared__ double s_dsum[32];
  __shared__ bool s_last;
  hpc_cent_smem cs;
  hpc_cent_bind(cs, smem_raw, D, a.k);
  hpc_load_centroids<D>(cs, a.C, a.deg, a.k, a.d, s_red);
  const int64_t TR = (int64_t)THREADS * R;
  const int64_t ngroups = (a.n + TR - 1) / TR;
  float fp_hi = 0.0f, fp_lo = 0.0f;  // this thread's rows' distances (TwoSum pair)
  if (cs.live == 0) {
    if (a.n > 0) hpc_status_set(a.status, HPC_ERR_DEGENERATE_ALL);
  } else {
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
      const int64_t base = g * TR;
      int lab[R];
      bool valid[R];
      hpc_sum2_add(fp_hi, fp_lo,
                   hpc_assign_group<D, R, THREADS, IB>(a.X, a.n, a.d, base, cs, lab, valid,
                                                       a.status));
      if (a.labels) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (valid[r]) a.labels[base + (int64_t)r * THREADS + threadIdx.x] = lab[r];
      }
    }
  }
  const double bsum = hpc_block_sum((double)fp_hi + (double)fp_lo, s_dsum);
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
      *a.f_out = (cs.live == 0 && a.n > 0) ? __longlong_as_double(0x7ff8000000000000ll) : f;
      *a.done_count = 0u;
    }
  }
}

template <int D, int IB>
int lloyd_plan_t(const hpc_launch &L, LloydLaunch &h) {
  using T = LTile<D>;
  auto kern = lloyd_kernel<D, T::R, T::THREADS, IB>;
  // per-block sums in shared memory when they fit; then the staged rows,
  // when they fit and cost no resident block
  const size_t cap = (size_t)L.smem_optin;
  const bool smem_sums = LloydSmem(D, T::R, T::THREADS, h.kmax, h.d, true, false).total <= cap;
  const size_t plain = LloydSmem(D, T::R, T::THREADS, h.kmax, h.d, smem_sums, false).total;
  const size_t staged = LloydSmem(D, T::R, T::THREADS, h.kmax, h.d, smem_sums, true).total;
  if (plain > cap) return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(staged <= cap ? staged : plain)) != cudaSuccess)
    return HPC_ERR_CUDA;
  int per_sm = 0, per_sm_staged = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T::THREADS, plain) != cudaSuccess ||
      per_sm < 1)
    return HPC_ERR_UNSUPPORTED;
  if (staged <= cap &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_staged, kern, T::THREADS, staged) !=
          cudaSuccess)
    return HPC_ERR_CUDA;
  const bool xstage = per_sm_staged >= per_sm;
  const size_t smem = xstage ? staged : plain;
  const int64_t per_task = h.task_blocks;
  int64_t total = (int64_t)per_sm * L.num_sms;
  if (total > h.max_blocks) total = h.max_blocks;
  if (total > per_task * h.W) total = per_task * h.W;
  if (h.W > total || h.W > HPC_MAX_TASKS) return HPC_ERR_UNSUPPORTED;
  // blocks in proportion to each task's distance work (rows x clusters)
  std::vector<int64_t> rows(h.W), work(h.W);
  std::vector<int> b0(h.W), nb(h.W);
  for (int w = 0; w < h.W; ++w) {
    rows[w] = h.tasks[w].s;
    work[w] = h.tasks[w].s * (int64_t)h.tasks[w].k;
  }
  hpc_split_blocks(h.W, rows.data(), work.data(), (int64_t)T::THREADS * T::R, total, b0.data(),
                   nb.data());
  int64_t grid = 0;
  for (int w = 0; w < h.W; ++w) {
    if (nb[w] > per_task) nb[w] = (int)per_task;
    h.tasks[w].block0 = (int)grid;
    h.tasks[w].nblocks = nb[w];
    if (h.W > 1)
      for (int b = 0; b < nb[w]; ++b) h.block_task_host[grid + b] = w;
    grid += nb[w];
  }
  h.grid = grid;
  h.smem = smem;
  h.smem_sums = smem_sums ? 1 : 0;
  h.xstage = xstage ? 1 : 0;
  return HPC_OK;
}

template <int D, int IB>
int lloyd_run_t(const hpc_launch &L, const LloydLaunch &h) {
  using T = LTile<D>;
  auto kern = lloyd_kernel<D, T::R, T::THREADS, IB>;
  LloydArgs a;
  a.W = h.W;
  a.single = h.tasks[0];
  a.tasks = h.tasks_dev;
  a.block_task = h.block_task_dev;
  a.d = h.d;
  a.max_iter = h.max_iter;
  a.tol = h.tol;
  a.status = h.status;
  a.smem_sums = h.smem_sums;
  a.xstage = h.xstage;
  a.round_advance = h.round_advance;
  void *args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)h.grid),
                                                    dim3(T::THREADS), args, h.smem, L.stream);
  return e == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

template <int D, int IB>
int objective_launch_t(const hpc_launch &L, const ObjArgsHost &h) {
  using T = Tile<D>;
  auto kern = objective_kernel<D, T::R, T::THREADS, IB>;
  const size_t smem = hpc_cent_smem_bytes(D, h.k);
  if (smem > (size_t)L.smem_optin) return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HPC_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T::THREADS, smem) != cudaSuccess ||
      per_sm < 1)
    return HPC_ERR_UNSUPPORTED;
  const int64_t TR = (int64_t)T::THREADS * T::R;
  const int64_t groups = (h.n + TR - 1) / TR;
  int64_t G = (int64_t)per_sm * L.num_sms;
  if (G > groups) G = groups;
  if (G < 1) G = 1;
  if (G > h.max_blocks) G = h.max_blocks;
  ObjArgs a;
  a.X = h.X;
  a.n = h.n;
  a.d = h.d;
  a.k = h.k;
  a.C = h.C;
  a.deg = h.deg;
  a.f_out = h.f_out;
  a.labels = h.labels;
  a.status = h.status;
  a.part = h.part;
  a.done_count = h.done_count;
  kern<<<(unsigned)G, T::THREADS, smem, L.stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

// index bits of the packed top-2 keys: 5 for k <= 32; larger k keeps values
// and a tracked index (7-bit keys for k <= 128 were measured slower: their
// wider error window sends more rows to the exact stages)
template <int D>
int lloyd_plan_d(const hpc_launch &L, LloydLaunch &h) {
  return h.kmax <= 32 ? lloyd_plan_t<D, 5>(L, h) : lloyd_plan_t<D, 0>(L, h);
}

template <int D>
int lloyd_run_d(const hpc_launch &L, const LloydLaunch &h) {
  return h.kmax <= 32 ? lloyd_run_t<D, 5>(L, h) : lloyd_run_t<D, 0>(L, h);
}

template <int D>
int objective_dispatch(const hpc_launch &L, const ObjArgsHost &h) {
  return h.k <= 32 ? objective_launch_t<D, 5>(L, h) : objective_launch_t<D, 0>(L, h);
}

}  // namespace

void hpc_split_blocks(int W, const int64_t *rows, const int64_t *work, int64_t rows_per_block,
                      int64_t total, int *block0, int *nblocks) {
  // one block each, then the next block always to the task with the most
  // work per block that can still use one (largest first, lowest index on
  // ties); a task uses at most one block per rows_per_block rows
  int64_t left = total - W;
  for (int w = 0; w < W; ++w) nblocks[w] = 1;
  while (left > 0) {
    int best = -1;
    double best_load = 0.0;
    for (int w = 0; w < W; ++w) {
      const int64_t need = (rows[w] + rows_per_block - 1) / rows_per_block;
      if (nblocks[w] >= need) continue;
      const double load = (double)(work ? work[w] : rows[w]) / nblocks[w];
      if (best < 0 || load > best_load) {
        best = w;
        best_load = load;
      }
    }
    if (best < 0) break;
    ++nblocks[best];
    --left;
  }
  int64_t acc = 0;
  for (int w = 0; w < W; ++w) {
    block0[w] = (int)acc;
    acc += nblocks[w];
  }
}

// Where the split-BF16 tensor-core Lloyd runs (mode 2): rows of 64 or 128
// floats with enough centroids that the k columns of a row tile keep the
// tensor cores busy.
static bool tcl_builtin(int d, int kmax) { return hpc_tcl_supported(d, kmax) && kmax >= 48; }

int hpc_lloyd_plan(const hpc_launch &L, LloydLaunch &h) {
  h.form = HPC_SEARCH_SIMT;
  if (h.tc_mode != 0 && hpc_tcl_supported(h.d, h.kmax) &&
      (h.tc_mode == 1 || tcl_builtin(h.d, h.kmax))) {
    const int rc = hpc_tcl_plan(L, h);
    if (rc != HPC_ERR_UNSUPPORTED) return rc;
    h.form = HPC_SEARCH_SIMT;
  }
  switch (hpc_pad_dim(h.d)) {
    case 2: return lloyd_plan_d<2>(L, h);
    case 4: return lloyd_plan_d<4>(L, h);
    case 8: return lloyd_plan_d<8>(L, h);
    case 16: return lloyd_plan_d<16>(L, h);
    case 32: return lloyd_plan_d<32>(L, h);
    case 64: return lloyd_plan_d<64>(L, h);
    default: return lloyd_plan_d<128>(L, h);
  }
}

int hpc_lloyd_run(const hpc_launch &L, const LloydLaunch &h) {
  if (h.form == HPC_SEARCH_SPLIT_BF16) return hpc_tcl_run(L, h);
  switch (hpc_pad_dim(h.d)) {
    case 2: return lloyd_run_d<2>(L, h);
    case 4: return lloyd_run_d<4>(L, h);
    case 8: return lloyd_run_d<8>(L, h);
    case 16: return lloyd_run_d<16>(L, h);
    case 32: return lloyd_run_d<32>(L, h);
    case 64: return lloyd_run_d<64>(L, h);
    default: return lloyd_run_d<128>(L, h);
  }
}

int hpc_objective_launch(const hpc_launch &L, const ObjArgsHost &h) {
  switch (hpc_pad_dim(h.d)) {
    case 2: return objective_dispatch<2>(L, h);
    case 4: return objective_dispatch<4>(L, h);
    case 8: return objective_dispatch<8>(L, h);
    case 16: return objective_dispatch<16>(L, h);
    case 32: return objective_dispatch<32>(L, h);
    case 64: return objective_dispatch<64>(L, h);
    default: return objective_dispatch<128>(L, h);
  }
}
