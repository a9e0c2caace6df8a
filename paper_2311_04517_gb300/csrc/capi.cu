// C ABI of the HPClust hot path: context, scratch memory, argument checks and
// the round orchestration (Algorithms 3 and 4).  Every numerical step runs in
// the kernels of sample.cu, kmeanspp.cu and lloyd.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

struct hpc_ctx {
  int device;
  cudaStream_t stream;
  hpc_launch L;
  int64_t grid_bound;
  // long-lived device words: [0] status, [1] objective done-counter
  int *dwords;
  void *ws;
  size_t ws_bytes;
  int64_t launches;
  int use_tc;  // 0 never, 1 wherever built, 2 (default) for d >= 64
  char err[256];
};

namespace {

struct Carver {
  char *base;
  size_t off;
  size_t cap;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

int fail(hpc_ctx *c, int code, const char *msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return code;
}

int cuda_fail(hpc_ctx *c, cudaError_t e, const char *where) {
  if (c) snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
  return HPC_ERR_CUDA;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Grows the scratch buffer to at least `bytes` (synchronises the stream
// before freeing the old buffer).
int ensure_ws(hpc_ctx *c, size_t bytes) {
  if (bytes <= c->ws_bytes) return HPC_OK;
  cudaError_t e;
  if (c->ws) {
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  size_t want = std::max(bytes, (size_t)1 << 20);
  if ((e = cudaMalloc(&c->ws, want)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HPC_ERR_NOMEM, "scratch allocation failed");
  }
  c->ws_bytes = want;
  return HPC_OK;
}

int check_dims(hpc_ctx *c, int32_t d) {
  if (d < 1 || d > HPC_MAX_D) return fail(c, HPC_ERR_ARG, "d must be in [1, 128]");
  return HPC_OK;
}

// ---- scratch layouts (one per operation) ----
size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t lloyd_ws(const hpc_ctx *c, int64_t s, int d, int k) {
  (void)s;
  return pad256(64) + pad256((size_t)3 * k * d * 8) + pad256((size_t)3 * k * 4) +
         pad256((size_t)2 * c->grid_bound * 8) + pad256((size_t)k) + 256;
}

size_t kpp_ws(const hpc_ctx *c, int64_t s, int L) {
  return pad256(64) + pad256((size_t)s * 4) + pad256((size_t)L * s * 4) +
         pad256((size_t)c->grid_bound * 8) + pad256((size_t)L * 8) + pad256((size_t)2 * L * 8) +
         256;
}

size_t obj_ws(const hpc_ctx *c) { return pad256((size_t)c->grid_bound * 8) + 256; }

// Launches Lloyd with scratch carved from `cv` (layout of lloyd_ws).
int run_lloyd(hpc_ctx *c, Carver &cv, const float *S, int64_t s, int d, int k, float *C,
              uint8_t *deg, int max_iter, double tol, int32_t *labels, double *f_out,
              int32_t *iters_out) {
  char *zero_begin = cv.base + ((cv.off + 255) & ~(size_t)255);
  hpc_gridbar *bar = cv.take<hpc_gridbar>(1);
  unsigned *gmax = reinterpret_cast<unsigned *>(bar + 1);
  unsigned long long *gsum = cv.take<unsigned long long>((size_t)3 * k * d);
  unsigned *gcount = cv.take<unsigned>((size_t)3 * k);
  char *zero_end = cv.base + cv.off;
  double *gpart = cv.take<double>((size_t)2 * c->grid_bound);
  uint8_t *degbuf = deg;
  if (!degbuf) degbuf = cv.take<uint8_t>((size_t)k);
  cudaError_t e = cudaMemsetAsync(zero_begin, 0, (size_t)(zero_end - zero_begin), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  if (!deg && (e = cudaMemsetAsync(degbuf, 0, (size_t)k, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  LloydArgsHost h{};
  h.S = S;
  h.s = s;
  h.d = d;
  h.k = k;
  h.C = C;
  h.deg = degbuf;
  h.max_iter = max_iter;
  h.tol = tol;
  h.labels = labels;
  h.f_out = f_out;
  h.iters_out = iters_out;
  h.bar = bar;
  h.status = c->dwords;
  h.gmaxabs = gmax;
  h.gsum = gsum;
  h.gcount = gcount;
  h.gpart = gpart;
  h.grid_cap = c->grid_bound;
  int rc = hpc_lloyd_launch(c->L, h);
  if (rc == HPC_ERR_CUDA) return cuda_fail(c, cudaGetLastError(), "lloyd launch");
  if (rc) return fail(c, rc, "lloyd: unsupported shape");
  c->launches += 1;
  return HPC_OK;
}

int run_kmeanspp(hpc_ctx *c, Carver &cv, const float *S, int64_t s, int d, int k, float *C,
                 uint8_t *deg, int L, uint64_t seed, uint32_t worker, uint32_t round) {
  char *zero_begin = cv.base + ((cv.off + 255) & ~(size_t)255);
  hpc_gridbar *bar = cv.take<hpc_gridbar>(1);
  unsigned *mx = reinterpret_cast<unsigned *>(bar + 1);  // 2 words
  unsigned long long *phi = cv.take<unsigned long long>((size_t)2 * L);
  char *zero_end = cv.base + cv.off;
  float *w = cv.take<float>((size_t)s);
  float *dc = cv.take<float>((size_t)L * s);
  unsigned long long *chunkQ = cv.take<unsigned long long>((size_t)c->grid_bound);
  long long *cand = cv.take<long long>((size_t)L);
  cudaError_t e = cudaMemsetAsync(zero_begin, 0, (size_t)(zero_end - zero_begin), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  KppArgsHost h{};
  h.S = S;
  h.s = s;
  h.d = d;
  h.k = k;
  h.C = C;
  h.deg = deg;
  h.L = L;
  h.seed = seed;
  h.worker = worker;
  h.round = round;
  h.bar = bar;
  h.status = c->dwords;
  h.w = w;
  h.dc = dc;
  h.chunkQ = chunkQ;
  h.cand = cand;
  h.phi = phi;
  h.mx = mx;
  h.grid_cap = c->grid_bound;
  int rc = hpc_kmeanspp_launch(c->L, h);
  if (rc == HPC_ERR_CUDA) return cuda_fail(c, cudaGetLastError(), "kmeanspp launch");
  if (rc) return fail(c, rc, "kmeanspp: unsupported shape");
  c->launches += 1;
  return HPC_OK;
}

int run_objective(hpc_ctx *c, Carver &cv, const float *X, int64_t n, int d, const float *C, int k,
                  const uint8_t *deg, double *f_out, int32_t *labels) {
  double *part = cv.take<double>((size_t)c->grid_bound);
  ObjArgsHost h{};
  h.X = X;
  h.n = n;
  h.d = d;
  h.k = k;
  h.C = C;
  h.deg = deg;
  h.f_out = f_out;
  h.labels = labels;
  h.status = c->dwords;
  h.part = part;
  h.done_count = reinterpret_cast<unsigned *>(c->dwords + 1);
  h.max_blocks = c->grid_bound;
  const bool want_tc = c->use_tc == 1 || (c->use_tc == 2 && d >= 64);
  int rc = (want_tc && X && aligned16(X) && hpc_tc_objective_supported(d, k, n))
               ? hpc_tc_objective_launch(c->L, h)
               : HPC_ERR_UNSUPPORTED;
  if (rc == HPC_ERR_UNSUPPORTED) rc = hpc_objective_launch(c->L, h);
  if (rc == HPC_ERR_CUDA) return cuda_fail(c, cudaGetLastError(), "objective launch");
  if (rc) return fail(c, rc, "objective: unsupported shape");
  c->launches += 1;
  return HPC_OK;
}

// Cooperative base selection and incumbent rule (Algorithms 3 and 4).
__global__ void base_select_kernel(const double *__restrict__ fhat_snap, const int32_t *__restrict__ peers,
                                   int npeers, int self, const float *__restrict__ C_snap,
                                   const uint8_t *__restrict__ deg_snap, const int64_t *__restrict__ coff,
                                   const int64_t *__restrict__ koff, int kd, int k, float *__restrict__ C_base,
                                   uint8_t *__restrict__ deg_base) {
  __shared__ int s_b;
  if (threadIdx.x == 0) {
    int b = self;
    for (int p = 0; p < npeers; ++p) {
      const int v = peers[p];
      if (fhat_snap[v] < fhat_snap[b] || (fhat_snap[v] == fhat_snap[b] && v < b)) b = v;
    }
    s_b = b;
  }
  __syncthreads();
  const int b = s_b;
  for (int e = threadIdx.x; e < kd; e += blockDim.x) C_base[e] = C_snap[coff[b] + e];
  for (int j = threadIdx.x; j < k; j += blockDim.x) deg_base[j] = deg_snap[koff[b] + j];
}

__global__ void incumbent_kernel(const double *__restrict__ f, int64_t s, double *__restrict__ fhat,
                                 const float *__restrict__ C_new, const uint8_t *__restrict__ deg_new,
                                 float *__restrict__ C_w, uint8_t *__restrict__ deg_w, int kd, int k,
                                 double *f_new_out, int32_t *iters_out, const int32_t *iters,
                                 uint8_t *acc_out) {
  const double per = *f / (double)s;
  const bool acc = per < *fhat;
  for (int e = threadIdx.x; e < kd; e += blockDim.x)
    if (acc) C_w[e] = C_new[e];
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    if (acc) deg_w[j] = deg_new[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc) *fhat = per;
    if (f_new_out) *f_new_out = *f;
    if (iters_out) *iters_out = *iters;
    if (acc_out) *acc_out = acc ? 1 : 0;
  }
}

// Block 0 waits at a grid barrier that block 1 never reaches; the bounded
// wait gives up after limit_ns and records HPC_ERR_TIMEOUT.
__global__ void selftest_timeout_kernel(hpc_gridbar *bar, int *status, uint64_t limit_ns) {
  if (blockIdx.x == 1) return;
  hpc_grid_sync(bar, status, limit_ns);
}

}  // namespace

int64_t hpc_grid_bound(const hpc_launch &L) { return (int64_t)L.num_sms * 8; }

extern "C" {

int hpc_create(hpc_ctx **ctx, int device, void *stream) {
  if (!ctx) return HPC_ERR_ARG;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HPC_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) return HPC_ERR_CUDA;
  hpc_ctx *c = new hpc_ctx();
  memset(c->err, 0, sizeof(c->err));
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->L.stream = c->stream;
  cudaDeviceGetAttribute(&c->L.num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&c->L.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->L.smem_optin -= 2048;  // keep room for the kernels' static shared memory
  c->grid_bound = hpc_grid_bound(c->L);
  c->use_tc = 2;
  if (cudaMalloc(&c->dwords, 256) != cudaSuccess) {
    delete c;
    return HPC_ERR_NOMEM;
  }
  cudaMemset(c->dwords, 0, 256);
  cudaDeviceSynchronize();
  *ctx = c;
  return HPC_OK;
}

int hpc_destroy(hpc_ctx *c) {
  if (!c) return HPC_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->ws) cudaFree(c->ws);
  if (c->dwords) cudaFree(c->dwords);
  delete c;
  return HPC_OK;
}

int hpc_set_stream(hpc_ctx *c, void *stream) {
  if (!c) return HPC_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  c->L.stream = c->stream;
  return HPC_OK;
}

int hpc_sync_status(hpc_ctx *c) {
  if (!c) return HPC_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  int st = 0;
  if ((e = cudaMemcpy(&st, c->dwords, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(c, e, "status read");
  if (st != 0) {
    cudaMemset(c->dwords, 0, sizeof(int));
    const char *m = st == HPC_ERR_TIMEOUT     ? "device wait timed out"
                    : st == HPC_ERR_NONFINITE ? "non-finite input rows"
                    : st == HPC_ERR_DEGENERATE_ALL ? "no live centroid"
                                                   : "device error";
    snprintf(c->err, sizeof(c->err), "%s", m);
  }
  return st;
}

const char *hpc_last_error(hpc_ctx *c) { return c ? c->err : "null context"; }

int hpc_set_tensor_cores(hpc_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 2) return HPC_ERR_ARG;
  c->use_tc = mode;
  return HPC_OK;
}

int64_t hpc_launch_count(hpc_ctx *c) { return c ? c->launches : 0; }

int hpc_reserve(hpc_ctx *c, int64_t bytes) {
  if (!c || bytes < 0) return HPC_ERR_ARG;
  return ensure_ws(c, (size_t)bytes);
}

int hpc_draw_sample(hpc_ctx *c, const float *X, int64_t n, int32_t d, uint64_t seed,
                    uint32_t worker, uint32_t round, int64_t s, float *S_out, int64_t *idx_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (s < 0 || (s > 0 && (n < 1 || !X || !S_out))) return fail(c, HPC_ERR_ARG, "bad sample size");
  if (s > 0 && (!aligned16(X) || !aligned16(S_out))) return fail(c, HPC_ERR_ARG, "unaligned");
  if (s == 0) return HPC_OK;
  cudaSetDevice(c->device);
  int64_t *idx = idx_out;
  if (!idx) {
    if (int rc = ensure_ws(c, pad256((size_t)s * 8) + 256)) return rc;
    idx = reinterpret_cast<int64_t *>(c->ws);
  }
  int rc = hpc_sample_launch(c->L, X, n, d, seed, worker, round, s, S_out, idx);
  if (rc) return cuda_fail(c, cudaGetLastError(), "sample launch");
  c->launches += 2;
  return HPC_OK;
}

int hpc_kmeanspp(hpc_ctx *c, const float *S, int64_t s, int32_t d, int32_t k, float *C_inout,
                 uint8_t *degenerate_inout, int32_t n_candidates, uint64_t seed, uint32_t worker,
                 uint32_t round) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (s < 1 || k < 1 || !S || !C_inout) return fail(c, HPC_ERR_ARG, "bad sizes");
  if (n_candidates < 1 || n_candidates > 8) return fail(c, HPC_ERR_ARG, "n_candidates in [1, 8]");
  if (!aligned16(S) || !aligned16(C_inout)) return fail(c, HPC_ERR_ARG, "unaligned");
  cudaSetDevice(c->device);
  size_t need = kpp_ws(c, s, n_candidates) + (degenerate_inout ? 0 : pad256((size_t)k));
  if (int rc = ensure_ws(c, need)) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  uint8_t *deg = degenerate_inout;
  if (!deg) {
    deg = cv.take<uint8_t>((size_t)k);
    cudaMemsetAsync(deg, 1, (size_t)k, c->stream);
  }
  return run_kmeanspp(c, cv, S, s, d, k, C_inout, deg, n_candidates, seed, worker, round);
}

int hpc_lloyd(hpc_ctx *c, const float *S, int64_t s, int32_t d, int32_t k, float *C_inout,
              uint8_t *degenerate_inout, int32_t max_iter, double rel_tol, int32_t prec,
              int32_t *labels_out, double *f_out, int32_t *iters_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (s < 1 || k < 1 || max_iter < 0 || !S || !C_inout || !f_out)
    return fail(c, HPC_ERR_ARG, "bad sizes");
  if (max_iter > HPC_MAX_ITER) return fail(c, HPC_ERR_ARG, "max_iter above 100000");
  if (prec != HPC_FP32) return fail(c, HPC_ERR_UNSUPPORTED, "only HPC_FP32 is built");
  if (!aligned16(S) || !aligned16(C_inout)) return fail(c, HPC_ERR_ARG, "unaligned");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, lloyd_ws(c, s, d, k))) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  return run_lloyd(c, cv, S, s, d, k, C_inout, degenerate_inout, max_iter, rel_tol, labels_out,
                   f_out, iters_out);
}

int hpc_objective(hpc_ctx *c, const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                  const uint8_t *degenerate, int32_t prec, double *f_out, int32_t *labels_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (n < 0 || k < 1 || !C || !f_out || (n > 0 && !X)) return fail(c, HPC_ERR_ARG, "bad sizes");
  if (prec != HPC_FP32) return fail(c, HPC_ERR_UNSUPPORTED, "only HPC_FP32 is built");
  if ((X && !aligned16(X)) || !aligned16(C)) return fail(c, HPC_ERR_ARG, "unaligned");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, obj_ws(c))) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  return run_objective(c, cv, X, n, d, C, k, degenerate, f_out, labels_out);
}

int hpc_selftest_wait_timeout(hpc_ctx *c, int64_t limit_ns) {
  if (!c || limit_ns < 1000 || limit_ns > 1000000000ll)
    return fail(c, HPC_ERR_ARG, "limit_ns in [1 us, 1 s]");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, 512)) return rc;
  hpc_gridbar *bar = reinterpret_cast<hpc_gridbar *>(c->ws);
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(hpc_gridbar), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  int *st = c->dwords;
  uint64_t lim = (uint64_t)limit_ns;
  void *args[] = {&bar, &st, &lim};
  e = cudaLaunchCooperativeKernel((const void *)selftest_timeout_kernel, dim3(2), dim3(32), args, 0,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "selftest launch");
  c->launches += 1;
  return HPC_OK;
}

int hpc_round(hpc_ctx *c, const float *X, int64_t n, int32_t d, const hpc_batch *b,
              int32_t strategy, uint64_t seed, uint32_t round, int32_t max_iter, double rel_tol,
              int32_t n_candidates, int32_t prec) {
  if (!c || !b) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (n < 1 || !X || b->W < 1 || !b->s || !b->k || !b->C_off || !b->K_off || !b->C ||
      !b->degenerate || !b->fhat)
    return fail(c, HPC_ERR_ARG, "malformed batch");
  if (strategy != HPC_COMPETITIVE && strategy != HPC_COOPERATIVE)
    return fail(c, HPC_ERR_ARG, "unknown strategy");
  if (prec != HPC_FP32) return fail(c, HPC_ERR_UNSUPPORTED, "only HPC_FP32 is built");
  if (n_candidates < 1 || n_candidates > 8) return fail(c, HPC_ERR_ARG, "n_candidates in [1, 8]");
  if (max_iter < 0 || max_iter > HPC_MAX_ITER) return fail(c, HPC_ERR_ARG, "max_iter out of range");
  if (!aligned16(X) || !aligned16(b->C)) return fail(c, HPC_ERR_ARG, "unaligned");
  const int W = b->W;
  int64_t smax = 0, kmax = 0, poolf = 0, poolk = 0;
  for (int w = 0; w < W; ++w) {
    if (b->s[w] < 1 || b->k[w] < 1 || b->C_off[w] < 0 || b->K_off[w] < 0 || (b->C_off[w] & 3))
      return fail(c, HPC_ERR_ARG, "malformed batch entry");
    smax = std::max<int64_t>(smax, b->s[w]);
    kmax = std::max<int64_t>(kmax, b->k[w]);
    poolf = std::max<int64_t>(poolf, b->C_off[w] + (int64_t)b->k[w] * d);
    poolk = std::max<int64_t>(poolk, b->K_off[w] + b->k[w]);
  }
  cudaSetDevice(c->device);
  // persistent part of the round's scratch, then room for the inner calls
  const size_t fixed = pad256((size_t)smax * d * 4) + pad256((size_t)smax * 8) +
                       pad256((size_t)kmax * d * 4) + pad256((size_t)kmax) + pad256(8) +
                       pad256(4) + pad256((size_t)poolf * 4) + pad256((size_t)poolk) +
                       pad256((size_t)W * 8) + pad256(((size_t)W * W + W) * 4) +
                       pad256((size_t)W * 2 * 8) + 4096;
  const size_t inner =
      std::max(lloyd_ws(c, smax, d, (int)kmax), kpp_ws(c, smax, n_candidates));
  if (int rc = ensure_ws(c, fixed + inner)) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  float *Sw = cv.take<float>((size_t)smax * d);
  int64_t *idx = cv.take<int64_t>((size_t)smax);
  float *Cn = cv.take<float>((size_t)kmax * d);
  uint8_t *dn = cv.take<uint8_t>((size_t)kmax);
  double *fw = cv.take<double>(1);
  int32_t *itw = cv.take<int32_t>(1);
  float *C_snap = cv.take<float>((size_t)poolf);
  uint8_t *deg_snap = cv.take<uint8_t>((size_t)poolk);
  double *fhat_snap = cv.take<double>((size_t)W);
  int32_t *peers_dev = cv.take<int32_t>((size_t)W * W + W);
  int64_t *offs_dev = cv.take<int64_t>((size_t)W * 2);
  const size_t inner_off = cv.off;
  cudaError_t e;
  std::vector<int32_t> npeers(W, 0);
  if (strategy == HPC_COOPERATIVE) {
    if ((e = cudaMemcpyAsync(C_snap, b->C, (size_t)poolf * 4, cudaMemcpyDeviceToDevice, c->stream)) ||
        (e = cudaMemcpyAsync(deg_snap, b->degenerate, (size_t)poolk, cudaMemcpyDeviceToDevice,
                             c->stream)) ||
        (e = cudaMemcpyAsync(fhat_snap, b->fhat, (size_t)W * 8, cudaMemcpyDeviceToDevice, c->stream)))
      return cuda_fail(c, e, "snapshot");
    // peers of worker w: the workers of its group with its k (flat W x W)
    std::vector<int64_t> offs(2 * W);
    std::vector<int32_t> peers((size_t)W * W, 0);
    for (int w = 0; w < W; ++w) {
      offs[w] = b->C_off[w];
      offs[W + w] = b->K_off[w];
      const int gw = b->group ? b->group[w] : 0;
      for (int v = 0; v < W; ++v)
        if ((b->group ? b->group[v] : 0) == gw && b->k[v] == b->k[w])
          peers[(size_t)w * W + npeers[w]++] = v;
    }
    if ((e = cudaMemcpyAsync(offs_dev, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice,
                             c->stream)) ||
        (e = cudaMemcpyAsync(peers_dev, peers.data(), peers.size() * 4, cudaMemcpyHostToDevice,
                             c->stream)) ||
        (e = cudaStreamSynchronize(c->stream)))  // host vectors must outlive the copies
      return cuda_fail(c, e, "peer tables");
  }
  for (int w = 0; w < W; ++w) {
    const int64_t s = b->s[w];
    const int k = b->k[w];
    const int kd = k * d;
    float *Cw = b->C + b->C_off[w];
    uint8_t *dw = b->degenerate + b->K_off[w];
    if (int rc = hpc_draw_sample(c, X, n, d, seed, (uint32_t)w, round, s, Sw, idx)) return rc;
    if (strategy == HPC_COOPERATIVE) {
      base_select_kernel<<<1, 256, 0, c->stream>>>(fhat_snap, peers_dev + (size_t)w * W, npeers[w], w,
                                                   C_snap, deg_snap, offs_dev, offs_dev + W, kd, k, Cn,
                                                   dn);
    } else {
      if ((e = cudaMemcpyAsync(Cn, Cw, (size_t)kd * 4, cudaMemcpyDeviceToDevice, c->stream)) ||
          (e = cudaMemcpyAsync(dn, dw, (size_t)k, cudaMemcpyDeviceToDevice, c->stream)))
        return cuda_fail(c, e, "base copy");
    }
    // NaN until Lloyd writes it: a failed run is never accepted
    if ((e = cudaMemsetAsync(fw, 0xff, 8, c->stream))) return cuda_fail(c, e, "memset");
    if (strategy == HPC_COOPERATIVE) c->launches += 1;
    cv.off = inner_off;
    if (int rc = run_kmeanspp(c, cv, Sw, s, d, k, Cn, dn, n_candidates, seed, (uint32_t)w, round))
      return rc;
    cv.off = inner_off;
    if (int rc = run_lloyd(c, cv, Sw, s, d, k, Cn, dn, max_iter, rel_tol, nullptr, fw, itw))
      return rc;
    incumbent_kernel<<<1, 256, 0, c->stream>>>(fw, s, b->fhat + w, Cn, dn, Cw, dw, kd, k,
                                               b->f_new ? b->f_new + w : nullptr,
                                               b->iters ? b->iters + w : nullptr, itw,
                                               b->accepted ? b->accepted + w : nullptr);
    if ((e = cudaGetLastError())) return cuda_fail(c, e, "incumbent launch");
    c->launches += 1;
  }
  return HPC_OK;
}

}  // extern "C"
