// Greedy K-means++ seeding of the degenerate centroids (Section 3: empty
// clusters are re-initialised by K-means++ on the sample; Section 6.5: three
// candidates per new centroid) as one persistent cooperative kernel.
//
// Block b owns the contiguous rows [s*b/G, s*(b+1)/G) so that "first row
// whose running weight exceeds the target" can be answered by the block that
// owns the target.  Weights D(x)^2 are float squared distances accumulated in
// dimension order with one fused multiply-add per dimension; the draw and
// the candidate potentials use exact unsigned 64-bit sums on the grid 2^-F,
// F = 62 - bitlen(s) - e (2^(e-1) <= max weight < 2^e), so every block, and
// any reference that follows the same definition, takes the same decisions.
// Four bounded grid barriers per seeded centroid.
#include <vector>

#include "common.cuh"
#include "kernels.h"

#define HPC_MAX_CAND 8

// Threads per block: 512 where the row and the distance chains fit the
// registers that leaves (d = 16 .. 64), 256 otherwise.
template <int D>
constexpr int kpp_threads() { return D >= 16 && D <= 64 ? 512 : 256; }

namespace {

struct KppArgs {
  int W;
  hpc_kpp_task single;        // W == 1
  const hpc_kpp_task *tasks;  // W > 1 (device)
  const int *block_task;      // W > 1 (device)
  int d, L;
  uint64_t seed;
  uint32_t round;
  const uint32_t *round_dev;  // nullable
  int *status;
};

template <int THREADS>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *sh) {
  v = hpc_warp_sum_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  unsigned long long r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < THREADS / 32; ++i) r += sh[i];
  return r;  // valid in thread 0
}

// Inclusive block scan; *total receives the block total (all threads).
template <int THREADS>
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v,
                                                             unsigned long long *sh,
                                                             unsigned long long *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  __syncthreads();
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int i = 0; i < THREADS / 32; ++i) {
      const unsigned long long t = sh[i];
      sh[i] = run;
      run += t;
    }
    sh[THREADS / 32] = run;
  }
  __syncthreads();
  v += sh[wid];
  *total = sh[THREADS / 32];
  return v;
}

template <int D, int THREADS>
__global__ void __launch_bounds__(THREADS) kmeanspp_kernel(KppArgs a) {
  extern __shared__ __align__(16) float smem[];
  __shared__ unsigned long long s_u64[THREADS / 32 + 1];
  __shared__ unsigned s_umax;
  __shared__ int s_owner[HPC_MAX_CAND];
  __shared__ unsigned long long s_tgt[HPC_MAX_CAND];
  __shared__ int s_lstar;

  // this block's task (one worker's sample) and its place in the task's
  // group; blocks the split left without a task have nothing to do
  const int bt = a.W == 1 ? 0 : a.block_task[blockIdx.x];
  if (bt < 0) return;
  const hpc_kpp_task tk = a.W == 1 ? a.single : a.tasks[bt];
  const uint32_t round = a.round_dev ? *a.round_dev : a.round;
  const int k = tk.k, d = a.d, L = a.L;
  const int64_t s = tk.s;
  const int G = tk.nblocks, lb = (int)blockIdx.x - tk.block0;
  const int64_t lo = s * lb / G, hi = s * (lb + 1) / G;
  float *cl = smem;          // k x D live centroids
  float *cr = cl + k * D;    // L x D candidate rows
  uint8_t *flags = reinterpret_cast<uint8_t *>(cr + L * D);  // k: 1 = to be seeded

  for (int j = threadIdx.x; j < k; j += THREADS) flags[j] = tk.deg[j];
  __syncthreads();
  int any_deg = 0, any_live = 0;
  for (int j = threadIdx.x; j < k; j += THREADS) {
    any_deg |= flags[j] != 0;
    any_live |= flags[j] == 0;
  }
  any_deg = __syncthreads_or(any_deg);
  any_live = __syncthreads_or(any_live);
  if (!any_deg) return;  // nothing to seed (same answer in every block)
  for (int e = threadIdx.x; e < k * D; e += THREADS) {
    const int j = e / D, t = e - j * D;
    cl[e] = (t < d && !flags[j]) ? tk.C[(int64_t)j * d + t] : 0.0f;
  }
  __syncthreads();
  if (!any_live) {  // uniform first pick into the lowest slot
    const uint64_t r = hpc_draw(a.seed, tk.worker, round, HPC_TAG_SEED, 0);
    const int64_t i0 = (int64_t)hpc_scale_word(r, (uint64_t)s);
    for (int t = threadIdx.x; t < D; t += THREADS) {
      const float v = t < d ? tk.S[i0 * d + t] : 0.0f;
      cl[t] = v;
      if (lb == 0 && t < d) tk.C[t] = v;
    }
    if (threadIdx.x == 0) {
      flags[0] = 0;
      if (lb == 0) tk.deg[0] = 0;
    }
    __syncthreads();
  }
  // D(x)^2 to the nearest live centroid
  if (threadIdx.x == 0) s_umax = 0u;
  __syncthreads();
  {
    unsigned m = 0u;
    for (int64_t i = lo + threadIdx.x; i < hi; i += THREADS) {
      float x[D];
      hpc_load_row<D>(x, tk.S + i * d, d);
      // four centroids per step as independent chains (each in dimension
      // order, the rounding the decisions are defined in); degenerate and
      // padding slots hold zeros and are skipped by their flag
      float best = __int_as_float(0x7f800000);
      int j = 0;
      for (; j + 4 <= k; j += 4) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
        const float *c0 = cl + j * D;
#pragma unroll
        for (int t = 0; t < D; ++t) {
          const float e0 = __fsub_rn(x[t], c0[t]), e1 = __fsub_rn(x[t], c0[D + t]);
          const float e2 = __fsub_rn(x[t], c0[2 * D + t]), e3 = __fsub_rn(x[t], c0[3 * D + t]);
          a0 = __fmaf_rn(e0, e0, a0);
          a1 = __fmaf_rn(e1, e1, a1);
          a2 = __fmaf_rn(e2, e2, a2);
          a3 = __fmaf_rn(e3, e3, a3);
        }
        if (!flags[j]) best = fminf(best, a0);
        if (!flags[j + 1]) best = fminf(best, a1);
        if (!flags[j + 2]) best = fminf(best, a2);
        if (!flags[j + 3]) best = fminf(best, a3);
      }
      for (; j < k; ++j) {
        if (flags[j]) continue;
        best = fminf(best, hpc_dist32_seq<D>(x, cl + j * D));
      }
      if (!(best <= 3.4028234663852886e38f)) best = __int_as_float(0x7fc00000);  // flag non-finite
      tk.w[i] = best;
      const unsigned b = __float_as_uint(best) & 0x7fffffffu;
      m = b > m ? b : m;
    }
    atomicMax(&s_umax, m);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&tk.mx[0], s_umax);
  }
  if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
  if (__ldcg(&tk.mx[0]) >= 0x7f800000u) {
    hpc_status_set(a.status, HPC_ERR_NONFINITE);
    return;
  }
  const int B = hpc_bit_length(s);
  int t = 0;
  for (int j = 0; j < k; ++j) {
    if (!flags[j]) continue;
    const float M = __uint_as_float(__ldcg(&tk.mx[t & 1]));
    if (!(M > 0.0f)) break;  // every row sits on a live centroid
    const int F = 62 - B - hpc_frexp_exp(M);
    // block sums of the fixed-point weights
    unsigned long long qs = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += THREADS) qs += (unsigned long long)hpc_quant(tk.w[i], F);
    qs = block_sum_u64<THREADS>(qs, s_u64);
    if (threadIdx.x == 0) {
      tk.chunkQ[lb] = qs;
      if (lb == 0) {
        tk.mx[(t + 1) & 1] = 0u;
        for (int l = 0; l < L; ++l) tk.phi[(size_t)((t + 1) & 1) * L + l] = 0ull;
      }
    }
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
    // targets and the block owning each: every block scans the per-block
    // sums in parallel (segments of ceil(G / THREADS) blocks per thread)
    if (threadIdx.x < L) s_owner[threadIdx.x] = -1;
    {
      const int seg = (G + THREADS - 1) / THREADS;
      const int g0 = threadIdx.x * seg, g1 = min(G, g0 + seg);
      unsigned long long loc = 0;
      for (int g = g0; g < g1; ++g) loc += __ldcg(&tk.chunkQ[g]);
      unsigned long long Q;
      const unsigned long long incl = block_scan_u64<THREADS>(loc, s_u64, &Q);
      const unsigned long long excl = incl - loc;
      for (int l = 0; l < L; ++l) {
        const uint64_t r = hpc_draw(a.seed, tk.worker, round, HPC_TAG_SEED,
                                    1ull + (uint64_t)t * (uint64_t)L + (uint64_t)l);
        const unsigned long long target = hpc_scale_word(r, Q);
        if (excl <= target && target < incl) {  // exactly one thread: its segment holds it
          unsigned long long run = excl;
          for (int g = g0; g < g1; ++g) {
            const unsigned long long q = __ldcg(&tk.chunkQ[g]);
            if (run + q > target) {
              s_owner[l] = g;
              s_tgt[l] = target - run;
              break;
            }
            run += q;
          }
        }
      }
    }
    __syncthreads();
    for (int l = 0; l < L; ++l) {
      if (s_owner[l] != lb) continue;
      unsigned long long tgt = s_tgt[l];
      long long found = -1;
      for (int64_t base = lo; base < hi; base += THREADS) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long q = i < hi ? (unsigned long long)hpc_quant(tk.w[i], F) : 0ull;
        unsigned long long tot;
        const unsigned long long incl = block_scan_u64<THREADS>(q, s_u64, &tot);
        const int cnt = __syncthreads_count(i < hi && incl <= tgt);
        const int64_t rows = min((int64_t)THREADS, hi - base);
        if (cnt < rows) {
          found = base + cnt;
          break;
        }
        tgt -= tot;
      }
      if (threadIdx.x == 0) tk.cand[l] = found;
      __syncthreads();
    }
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
    // candidate potentials phi_l = sum_i q(min(w_i, D(x_i, cand_l)^2))
    for (int e = threadIdx.x; e < L * D; e += THREADS) {
      const int l = e / D, tt = e - l * D;
      const long long ci = __ldcg(&tk.cand[l]);
      cr[e] = (tt < d && ci >= 0) ? tk.S[ci * d + tt] : 0.0f;
    }
    __syncthreads();
    unsigned long long ph[HPC_MAX_CAND];
#pragma unroll
    for (int l = 0; l < HPC_MAX_CAND; ++l) ph[l] = 0ull;
    for (int64_t i = lo + threadIdx.x; i < hi; i += THREADS) {
      float x[D];
      hpc_load_row<D>(x, tk.S + i * d, d);
      const float wi = tk.w[i];
#pragma unroll
      for (int l = 0; l < HPC_MAX_CAND; ++l) {
        if (l >= L) break;
        const float v = hpc_dist32_seq<D>(x, cr + l * D);
        tk.dc[(int64_t)l * s + i] = v;
        ph[l] += (unsigned long long)hpc_quant(fminf(wi, v), F);
      }
    }
#pragma unroll
    for (int l = 0; l < HPC_MAX_CAND; ++l) {
      if (l >= L) break;
      const unsigned long long bs = block_sum_u64<THREADS>(ph[l], s_u64);
      if (threadIdx.x == 0 && bs != 0ull) atomicAdd(&tk.phi[(size_t)(t & 1) * L + l], bs);
    }
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
    // keep the candidate with the smallest potential (first drawn on ties)
    if (threadIdx.x == 0) {
      int best = 0;
      unsigned long long bp = __ldcg(&tk.phi[(size_t)(t & 1) * L]);
      for (int l = 1; l < L; ++l) {
        const unsigned long long p = __ldcg(&tk.phi[(size_t)(t & 1) * L + l]);
        if (p < bp) {
          bp = p;
          best = l;
        }
      }
      s_lstar = best;
      s_umax = 0u;
    }
    __syncthreads();
    const int ls = s_lstar;
    if (lb == 0) {
      for (int tt = threadIdx.x; tt < d; tt += THREADS) tk.C[(int64_t)j * d + tt] = cr[ls * D + tt];
      if (threadIdx.x == 0) tk.deg[j] = 0;
    }
    unsigned m = 0u;
    for (int64_t i = lo + threadIdx.x; i < hi; i += THREADS) {
      const float v = fminf(tk.w[i], tk.dc[(int64_t)ls * s + i]);
      tk.w[i] = v;
      const unsigned b = __float_as_uint(v);
      m = b > m ? b : m;
    }
    atomicMax(&s_umax, m);
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&tk.mx[(t + 1) & 1], s_umax);
    if (!hpc_grid_sync(tk.bar, a.status, (unsigned)G)) return;
    ++t;
  }
}

// The blocks of a batched seeding launch, given to the workers that have a
// centroid to seed.  After the first round a round reseeds few centroids in
// few workers (those whose clusters emptied), and each of them first takes
// the D^2 pass over its sample against every live centroid; the host's plan,
// made before the flags are known, spreads the launch over every worker in
// proportion to s k and would leave those workers a few blocks each.  This
// one-block kernel runs before the seeding launch on the same stream (and in
// a recorded round), reads the flags, and splits the launch's G blocks over
// the workers with a degenerate slot in proportion to s (k + (L + 1) n),
// n their degenerate slots: one block each first, at most one block per
// `rows_per_block` rows and `cap` blocks; the other blocks get no task.  The
// seeding decisions do not depend on the split (exact fixed-point sums, one
// global target search).

__global__ void kpp_split_kernel(hpc_kpp_task *tasks, int *block_task, int W, int G,
                                 int rows_per_block, int64_t cap, int L) {
  __shared__ double s_work[HPC_KPP_SPLIT_MAX];
  __shared__ int s_cap[HPC_KPP_SPLIT_MAX], s_nb[HPC_KPP_SPLIT_MAX], s_b0[HPC_KPP_SPLIT_MAX + 1];
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const int k = tasks[w].k;
    const uint8_t *deg = tasks[w].deg;
    const int64_t s = tasks[w].s;
    int nd = 0;
    for (int j = 0; j < k; ++j) nd += deg[j] != 0;
    s_work[w] = nd > 0 && s > 0 ? (double)s * (double)(k + (L + 1) * nd) : 0.0;
    s_cap[w] = (int)min(cap, (s + rows_per_block - 1) / rows_per_block);
    s_nb[w] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int needy = 0;
    double tot = 0.0;
    for (int w = 0; w < W; ++w)
      if (s_work[w] > 0.0) {
        ++needy;
        tot += s_work[w];
      }
    int used = 0;
    if (needy > 0 && needy <= G) {
      const int extra = G - needy;
      for (int w = 0; w < W; ++w) {
        if (s_work[w] <= 0.0) continue;
        const int nb = min(s_cap[w], 1 + (int)floor((double)extra * (s_work[w] / tot)));
        s_nb[w] = max(nb, 1);
        used += s_nb[w];
      }
      // the rest one at a time: to the worker with the most work per block
      // that can still take one
      while (used < G) {
        int best = -1;
        double bl = 0.0;
        for (int w = 0; w < W; ++w) {
          if (s_work[w] <= 0.0 || s_nb[w] >= s_cap[w]) continue;
          const double l = s_work[w] / s_nb[w];
          if (best < 0 || l > bl) {
            best = w;
            bl = l;
          }
        }
        if (best < 0) break;
        ++s_nb[best];
        ++used;
      }
    }
    s_b0[0] = 0;
    for (int w = 0; w < W; ++w) {
      s_b0[w + 1] = s_b0[w] + s_nb[w];
      tasks[w].block0 = s_b0[w];
      tasks[w].nblocks = s_nb[w];
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < G; b += blockDim.x) {
    int owner = -1;
    for (int w = 0; w < W; ++w)
      if (b >= s_b0[w] && b < s_b0[w + 1]) {
        owner = w;
        break;
      }
    block_task[b] = owner;
  }
}

size_t kpp_smem_bytes(int D, int k, int L) {
  return ((size_t)k * D + (size_t)L * D) * 4 + (size_t)k + 16;
}

template <int D>
int kpp_plan_t(const hpc_launch &Lc, KppLaunch &h) {
  auto kern = kmeanspp_kernel<D, kpp_threads<D>()>;
  const size_t smem = kpp_smem_bytes(D, h.kmax, h.L);
  if (smem > (size_t)Lc.smem_optin) return HPC_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HPC_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kpp_threads<D>(), smem) != cudaSuccess ||
      per_sm < 1)
    return HPC_ERR_UNSUPPORTED;
  int64_t total = (int64_t)per_sm * Lc.num_sms;
  if (total > h.max_blocks) total = h.max_blocks;
  if (total > h.chunk_cap * h.W) total = h.chunk_cap * h.W;
  if (h.W > total || h.W > HPC_MAX_TASKS) return HPC_ERR_UNSUPPORTED;
  // blocks in proportion to each task's sample rows times the live
  // centroids its weights start from (at most k)
  std::vector<int64_t> rows(h.W), work(h.W);
  std::vector<int> b0(h.W), nb(h.W);
  for (int w = 0; w < h.W; ++w) {
    rows[w] = h.tasks[w].s;
    work[w] = h.tasks[w].s * (int64_t)h.tasks[w].k;
  }
  hpc_split_blocks(h.W, rows.data(), work.data(), kpp_threads<D>(), total, b0.data(), nb.data());
  int64_t grid = 0;
  for (int w = 0; w < h.W; ++w) {
    if (nb[w] > h.chunk_cap) nb[w] = (int)h.chunk_cap;
    h.tasks[w].block0 = (int)grid;
    h.tasks[w].nblocks = nb[w];
    if (h.W > 1)
      for (int b = 0; b < nb[w]; ++b) h.block_task_host[grid + b] = w;
    grid += nb[w];
  }
  h.grid = grid;
  h.smem = smem;
  return HPC_OK;
}

template <int D>
int kpp_run_t(const hpc_launch &Lc, const KppLaunch &h) {
  auto kern = kmeanspp_kernel<D, kpp_threads<D>()>;
  if (h.W > 1 && h.W <= HPC_KPP_SPLIT_MAX) {
    kpp_split_kernel<<<1, 128, 0, Lc.stream>>>(const_cast<hpc_kpp_task *>(h.tasks_dev),
                                               const_cast<int *>(h.block_task_dev), h.W, (int)h.grid,
                                               kpp_threads<D>(), h.chunk_cap, h.L);
    if (cudaGetLastError() != cudaSuccess) return HPC_ERR_CUDA;
  }
  KppArgs a;
  a.W = h.W;
  a.single = h.tasks[0];
  a.tasks = h.tasks_dev;
  a.block_task = h.block_task_dev;
  a.d = h.d;
  a.L = h.L;
  a.seed = h.seed;
  a.round = h.round;
  a.round_dev = h.round_dev;
  a.status = h.status;
  void *args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)h.grid),
                                                    dim3(kpp_threads<D>()), args, h.smem, Lc.stream);
  return e == cudaSuccess ? HPC_OK : HPC_ERR_CUDA;
}

}  // namespace

int hpc_kmeanspp_plan(const hpc_launch &L, KppLaunch &h) {
  if (h.L < 1 || h.L > HPC_MAX_CAND) return HPC_ERR_ARG;
  switch (hpc_pad_dim(h.d)) {
    case 2: return kpp_plan_t<2>(L, h);
    case 4: return kpp_plan_t<4>(L, h);
    case 8: return kpp_plan_t<8>(L, h);
    case 16: return kpp_plan_t<16>(L, h);
    case 32: return kpp_plan_t<32>(L, h);
    case 64: return kpp_plan_t<64>(L, h);
    default: return kpp_plan_t<128>(L, h);
  }
}

int hpc_kmeanspp_run(const hpc_launch &L, const KppLaunch &h) {
  switch (hpc_pad_dim(h.d)) {
    case 2: return kpp_run_t<2>(L, h);
    case 4: return kpp_run_t<4>(L, h);
    case 8: return kpp_run_t<8>(L, h);
    case 16: return kpp_run_t<16>(L, h);
    case 32: return kpp_run_t<32>(L, h);
    case 64: return kpp_run_t<64>(L, h);
    default: return kpp_run_t<128>(L, h);
  }
}
