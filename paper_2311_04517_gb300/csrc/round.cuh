// Per-worker steps of a batched round (Algorithms 3-5) that run inside other
// kernels: the base selection (in the sampling launch) and the incumbent
// rule (at the end of each worker's Lloyd run).
#pragma once

#include "common.cuh"
#include "kernels.h"

// Base of worker blockIdx.y (Algorithm 3: its own incumbent; Algorithm 4:
// the incumbent with the smallest objective per sample point among the
// workers of its group with its k, lowest index on ties; Algorithm 5: the
// competitive phase for rounds below n_competitive).  All bases are read
// before any incumbent of the round changes (the incumbents change in the
// Lloyd launch), which is the round-start snapshot.  One block of 256
// threads per worker.
__device__ __forceinline__ void hpc_base_select_block(const hpc_base_args &a, int w) {
  __shared__ double s_f[256];
  __shared__ int s_v[256];
  const uint32_t rnd = a.round_dev ? *a.round_dev : a.round;
  const bool cooperative = a.strategy == HPC_COOPERATIVE ||
                           (a.strategy == HPC_HYBRID && (int64_t)rnd >= (int64_t)a.n_competitive);
  const hpc_round_worker me = a.wk[w];
  double bf = a.fhat[w];
  int bv = w;
  if (cooperative) {
    for (int v = threadIdx.x; v < a.W; v += blockDim.x) {
      const hpc_round_worker o = a.wk[v];
      if (o.group != me.group || o.k != me.k) continue;
      const double f = a.fhat[v];
      if (f < bf || (f == bf && v < bv)) {
        bf = f;
        bv = v;
      }
    }
  }
  s_f[threadIdx.x] = bf;
  s_v[threadIdx.x] = bv;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const double f = s_f[threadIdx.x + h];
      const int v = s_v[threadIdx.x + h];
      if (f < s_f[threadIdx.x] || (f == s_f[threadIdx.x] && v < s_v[threadIdx.x])) {
        s_f[threadIdx.x] = f;
        s_v[threadIdx.x] = v;
      }
    }
    __syncthreads();
  }
  const int b = s_v[0];
  const int64_t coff = a.wk[b].C_off, koff = a.wk[b].K_off;
  const int kd = me.k * a.d;
  for (int e = threadIdx.x; e < kd; e += blockDim.x) me.Cn[e] = a.Cpool[coff + e];
  for (int j = threadIdx.x; j < me.k; j += blockDim.x) me.dn[j] = a.Kpool[koff + j];
  if (threadIdx.x == 0) {
    // a run that fails never reaches the incumbent rule: its report says so
    *me.fw = __longlong_as_double(0x7ff8000000000000ll);
    *me.itw = 0;
    if (a.f_new) a.f_new[w] = __longlong_as_double(0x7ff8000000000000ll);
    if (a.iters) a.iters[w] = 0;
    if (a.accepted) a.accepted[w] = 0;
  }
}

// Incumbent rule of Algorithms 3-5 for one Lloyd task, by one whole block:
// replace the worker's incumbent when f / s < fhat (strict), and report f,
// the iteration count and the decision.
__device__ __forceinline__ void hpc_incumbent_block(const hpc_lloyd_task &tk, int d, double f,
                                                    int iters) {
  __shared__ int s_acc;
  if (threadIdx.x == 0) s_acc = (f / (double)tk.s) < *tk.fhat ? 1 : 0;
  __syncthreads();
  const bool acc = s_acc != 0;
  if (acc) {
    const int kd = tk.k * d;
    for (int e = threadIdx.x; e < kd; e += blockDim.x) tk.C_inc[e] = tk.C[e];
    for (int j = threadIdx.x; j < tk.k; j += blockDim.x) tk.deg_inc[j] = tk.deg[j];
  }
  if (threadIdx.x == 0) {
    if (acc) *tk.fhat = f / (double)tk.s;
    if (tk.f_new) *tk.f_new = f;
    if (tk.iters_rep) *tk.iters_rep = iters;
    if (tk.uprev) *tk.uprev = iters;
    if (tk.accepted) *tk.accepted = acc ? 1 : 0;
    // when this worker's run ended (Section 6.4's baseline convergence time
    // is the time until any worker reaches a given sample objective)
    if (tk.t_done) *tk.t_done = hpc_globaltimer();
  }
}
