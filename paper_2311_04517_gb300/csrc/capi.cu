// C ABI of the HPClust hot path: context, scratch memory, argument checks and
// the round orchestration (Algorithms 3 and 4).  Every numerical step runs in
// the kernels of sample.cu, kmeanspp.cu and lloyd.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "costmodel.h"
#include "kernels.h"

// Workers of one round launch per persistent kernel (every launch has at
// least one block per SM, so at least this many tasks fit).
#define HPC_ROUND_CHUNK 128
#define HPC_MAX_WORKERS 65535
// events of one timed round: rounds of up to 31 launch chunks are timed
#define HPC_TIMING_EVENTS 64
// search forms of the objective (hpc_search)
#define HPC_NFORMS 4
// rows per CTA the tensor-core Lloyd settles against every centroid after
// each pass (beyond it, where they arise)
#define HPC_LLOYD_QUEUE_CAP 16384

struct hpc_round_plan;

struct hpc_ctx {
  int device;
  cudaStream_t stream;
  hpc_launch L;
  int64_t grid_bound;
  // long-lived device words: [0] status, [1] objective done-counter
  int *dwords;
  void *ws;
  size_t ws_bytes;
  // each worker's updates in its latest run, read by the next round's Lloyd
  // CTA plan (hpc_round; a prepared round keeps its own): zero when allocated
  int32_t *upd;
  int64_t upd_cap;
  int64_t launches;
  int use_tc;  // 0 never, 1 wherever built, 2 (default): where measured faster
  // objective search forms chosen by hpc_autotune_objective / set by the
  // caller, per (d, k); consulted in mode 2 before the built-in choice
  std::vector<std::pair<int64_t, int>> forms;
  int force_form;  // >= 0 while hpc_autotune_objective times one form
  // pinned staging ring for the per-round descriptor tables: slot i is
  // rewritten only after the launch that read it last time has run
  void *stage_host[4];
  void *stage_dev[4];  // the same pinned slot, mapped into the device's address space
  size_t stage_bytes[4];
  cudaEvent_t stage_ev[4];
  bool stage_used[4];
  int stage_next;
  // a prepared round (hpc_round_prepare): its own device memory, so other
  // calls on the context never overwrite it
  hpc_round_plan *plan;
  void *plan_mem;
  size_t plan_bytes;
  uint32_t *plan_round;  // device round counter, advanced by every enqueued round
  // phase timing of rounds (hpc_set_phase_timing): an event before the
  // round's first launch and one after each launch; tev_kind[i] is the
  // phase (0 sampling, 1 K-means++, 2 Lloyd) of the launch that ends at
  // event i (i >= 1)
  int timing;
  int stats_on;  // hpc_set_search_stats: the tensor-core searches count their stages
  cudaEvent_t tev[HPC_TIMING_EVENTS];
  int tev_kind[HPC_TIMING_EVENTS];
  int tev_n;
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

// The context's per-worker update counts, at least W of them; new ones are
// zero (no run yet).
int ensure_upd(hpc_ctx *c, int64_t W) {
  if (W <= c->upd_cap) return HPC_OK;
  cudaError_t e;
  if (c->upd) {
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
    cudaFree(c->upd);
    c->upd = nullptr;
    c->upd_cap = 0;
  }
  const int64_t want = std::max<int64_t>(W, 128);
  if ((e = cudaMalloc(&c->upd, (size_t)want * sizeof(int32_t))) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HPC_ERR_NOMEM, "update-count allocation failed");
  }
  if ((e = cudaMemsetAsync(c->upd, 0, (size_t)want * sizeof(int32_t), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  c->upd_cap = want;
  return HPC_OK;
}

int check_dims(hpc_ctx *c, int32_t d) {
  if (d < 1 || d > HPC_MAX_D) return fail(c, HPC_ERR_ARG, "d must be in [1, 128]");
  return HPC_OK;
}

// ---- scratch layouts (one per operation) ----
size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

// Per-task words that must be zero when the persistent kernels start: the
// Lloyd barrier and max |x| word, the K-means++ barrier, max-weight words
// and candidate potentials.  One 256-byte header per task.
struct TaskHeader {
  hpc_gridbar lbar;
  unsigned gmaxabs;
  unsigned pad0;
  hpc_gridbar kbar;
  unsigned mx[2];
  unsigned long long phi[2 * 8];
  unsigned long long gobj[3];  // Lloyd's fixed-point sample objectives
  unsigned lpop;               // a batched tensor-core Lloyd launch's next follow-up (first worker of the chunk)
  unsigned pad2;
  unsigned char pad1[256 - 32 - 128 - 24 - 8];
};
static_assert(sizeof(TaskHeader) == 256, "task header is one 256-byte line");

// what the split-BF16 tensor-core Lloyd adds per task: the rows' previous
// labels and the exact centroid block
size_t tcl_ws(int d, int k, int64_t s) {
  return hpc_tcl_supported(d, k) ? pad256((size_t)s * 4) + pad256(hpc_tcl_gcent_bytes(d, k)) : 0;
}

// the tensor-core Lloyd's per-CTA queues (one launch at a time uses them)
size_t tcl_queue_ws(const hpc_ctx *c, int d, int kmax) {
  return hpc_tcl_supported(d, kmax) ? pad256((size_t)c->L.num_sms * HPC_LLOYD_QUEUE_CAP * 8) : 0;
}

size_t lloyd_ws(const hpc_ctx *c, int d, int k, int64_t s) {
  return sizeof(TaskHeader) + pad256((size_t)3 * k * d * 8) + pad256((size_t)3 * k * 4) +
         pad256((size_t)k) + tcl_ws(d, k, s) + tcl_queue_ws(c, d, k) + 512;
}

size_t kpp_ws(const hpc_ctx *c, int64_t s, int L) {
  return sizeof(TaskHeader) + pad256((size_t)s * 4) + pad256((size_t)L * s * 4) +
         pad256((size_t)c->grid_bound * 8) + pad256((size_t)L * 8) + 256;
}

// near-tie rows the tensor-core search settles after its main loop, per block
#define HPC_OBJ_QUEUE_CAP 32768


// the wide tensor-core search's exact centroid block, at its largest shape
#define HPC_OBJ_CENT_BYTES ((size_t)320 * 1024)

size_t obj_ws(const hpc_ctx *c) {
  return pad256((size_t)c->grid_bound * 8) + pad256((size_t)c->L.num_sms * HPC_OBJ_QUEUE_CAP * 8) +
         HPC_OBJ_CENT_BYTES + 768;
}

// Lloyd scratch of one task (header zeroed by the caller).
void lloyd_task_scratch(const hpc_ctx *c, Carver &cv, TaskHeader *hd, int d, int k,
                        hpc_lloyd_task &t) {
  t.bar = &hd->lbar;
  t.gmaxabs = &hd->gmaxabs;
  t.gsum = cv.take<unsigned long long>((size_t)3 * k * d);
  t.gcount = cv.take<unsigned>((size_t)3 * k);
  t.gobj = hd->gobj;
  t.plab = nullptr;
  t.gcent = nullptr;
  if (hpc_tcl_supported(d, k)) {
    t.plab = t.labels ? t.labels : cv.take<int32_t>((size_t)t.s);
    t.gcent = cv.take<float>(hpc_tcl_gcent_bytes(d, k) / 4);
  }
}

void kpp_task_scratch(const hpc_ctx *c, Carver &cv, TaskHeader *hd, int64_t s, int L,
                      hpc_kpp_task &t) {
  t.bar = &hd->kbar;
  t.mx = hd->mx;
  t.phi = hd->phi;
  t.w = cv.take<float>((size_t)s);
  t.dc = cv.take<float>((size_t)L * s);
  t.chunkQ = cv.take<unsigned long long>((size_t)c->grid_bound);
  t.cand = cv.take<long long>((size_t)L);
}

// The search-stage counters (four words in the context's device words,
// after the status and the objective's done-counter), or null when off.
unsigned long long *stats_ptr(const hpc_ctx *c) {
  return c->stats_on ? reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(c->dwords) + 64)
                     : nullptr;
}

int plan_fail(hpc_ctx *c, int rc, const char *what) {
  if (rc == HPC_ERR_CUDA) return cuda_fail(c, cudaGetLastError(), what);
  return fail(c, rc, what);
}

// The Lloyd search mode a precision asks for: HPC_FP32 leaves the choice to
// the context (hpc_set_tensor_cores); HPC_BF16 asks for the split-BF16
// tensor-core search, built for d = 64 (k <= 512) and d = 128 (k <= 256).
int prec_lloyd_mode(hpc_ctx *c, int prec, int d, int kmax, int *mode) {
  if (prec == HPC_FP32) {
    *mode = c->use_tc;
    return HPC_OK;
  }
  if (prec == HPC_BF16) {
    if (!hpc_tcl_supported(d, kmax))
      return fail(c, HPC_ERR_UNSUPPORTED, "HPC_BF16: split-BF16 search not built for this shape");
    *mode = 1;
    return HPC_OK;
  }
  if (prec == HPC_FP8) return fail(c, HPC_ERR_UNSUPPORTED, "HPC_FP8 is not built");
  return fail(c, HPC_ERR_ARG, "unknown precision");
}

// Launches Lloyd on one sample with scratch carved from `cv`.
int run_lloyd(hpc_ctx *c, Carver &cv, const float *S, int64_t s, int d, int k, float *C,
              uint8_t *deg, int max_iter, double tol, int32_t *labels, double *f_out,
              int32_t *iters_out, int tc_mode) {
  TaskHeader *hd = cv.take<TaskHeader>(1);
  hpc_lloyd_task t{};
  t.S = S;
  t.s = s;
  t.k = k;
  t.C = C;
  t.labels = labels;
  t.f_out = f_out;
  t.iters_out = iters_out;
  lloyd_task_scratch(c, cv, hd, d, k, t);
  t.deg = deg ? deg : cv.take<uint8_t>((size_t)k);
  cudaError_t e = cudaMemsetAsync(hd, 0, sizeof(TaskHeader), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  if (!deg && (e = cudaMemsetAsync(t.deg, 0, (size_t)k, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "memset");
  LloydLaunch h{};
  h.W = 1;
  h.tasks = &t;
  h.d = d;
  h.kmax = k;
  h.max_iter = max_iter;
  h.tol = tol;
  h.status = c->dwords;
  h.max_blocks = c->grid_bound;
  h.task_blocks = c->grid_bound;
  h.tc_mode = tc_mode;
  h.stats = stats_ptr(c);
  if (hpc_tcl_supported(d, k)) {
    h.queue = cv.take<int64_t>((size_t)c->L.num_sms * HPC_LLOYD_QUEUE_CAP);
    h.queue_cap = HPC_LLOYD_QUEUE_CAP;
    h.queue_ctas = c->L.num_sms;
  }
  int rc = hpc_lloyd_plan(c->L, h);
  if (rc) return plan_fail(c, rc, "lloyd: unsupported shape");
  if ((rc = hpc_lloyd_run(c->L, h))) return plan_fail(c, rc, "lloyd launch");
  c->launches += 1;
  return HPC_OK;
}

int run_kmeanspp(hpc_ctx *c, Carver &cv, const float *S, int64_t s, int d, int k, float *C,
                 uint8_t *deg, int L, uint64_t seed, uint32_t worker, uint32_t round) {
  TaskHeader *hd = cv.take<TaskHeader>(1);
  hpc_kpp_task t{};
  t.S = S;
  t.s = s;
  t.k = k;
  t.worker = worker;
  t.C = C;
  t.deg = deg;
  kpp_task_scratch(c, cv, hd, s, L, t);
  cudaError_t e = cudaMemsetAsync(hd, 0, sizeof(TaskHeader), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "memset");
  KppLaunch h{};
  h.W = 1;
  h.tasks = &t;
  h.d = d;
  h.kmax = k;
  h.L = L;
  h.seed = seed;
  h.round = round;
  h.status = c->dwords;
  h.max_blocks = c->grid_bound;
  h.chunk_cap = c->grid_bound;
  int rc = hpc_kmeanspp_plan(c->L, h);
  if (rc) return plan_fail(c, rc, "kmeanspp: unsupported shape");
  if ((rc = hpc_kmeanspp_run(c->L, h))) return plan_fail(c, rc, "kmeanspp launch");
  c->launches += 1;
  return HPC_OK;
}

bool form_supported(int form, int d, int k, int64_t n) {
  switch (form) {
    case HPC_SEARCH_SIMT: return true;
    case HPC_SEARCH_SPLIT_TF32: return hpc_tcs_objective_supported(d, k, n);
    case HPC_SEARCH_TF32: return hpc_tc_objective_supported(d, k, n);
    case HPC_SEARCH_SPLIT_BF16: return n >= 1 && hpc_tcl_supported(d, k);
    default: return false;
  }
}

int64_t form_key(int d, int k) { return (int64_t)d << 32 | (uint32_t)k; }

int builtin_form(int d, int k, int64_t n);

// The search form hpc_objective runs for (d, k, n) in the context's mode.
int objective_form(const hpc_ctx *c, int d, int k, int64_t n) {
  if (c->force_form >= 0) return c->force_form;
  if (c->use_tc == 0) return HPC_SEARCH_SIMT;
  if (c->use_tc == 1) {
    if (hpc_tcs_objective_supported(d, k, n)) return HPC_SEARCH_SPLIT_TF32;
    if (hpc_tc_objective_supported(d, k, n) && d >= 64 && k <= 128) return HPC_SEARCH_TF32;
    if (form_supported(HPC_SEARCH_SPLIT_BF16, d, k, n)) return HPC_SEARCH_SPLIT_BF16;
    return HPC_SEARCH_SIMT;
  }
  for (const auto &f : c->forms)
    if (f.first == form_key(d, k) && form_supported(f.second, d, k, n)) return f.second;
  return builtin_form(d, k, n);
}

int builtin_form(int d, int k, int64_t n) {
  // built-in choice, from measurements on GB300 with the incumbents the
  // method produces: split TF32 for d = 32 (1.5x the CUDA-core search at
  // k = 25, 1.45x at k = 100); TF32 for d = 64 / 128 with k <= 128; at d = 16
  // the two are within a few percent and the CUDA cores are kept.  For k > 128 the TF32 search wins only where few rows
  // sit near a tie (5x at k = 500 with one centroid per mixture component,
  // 2x slower with several per component, as K-means leaves them on skewed
  // mixtures): the CUDA cores unless a measurement says otherwise
  if (d == 32 && hpc_tcs_objective_supported(d, k, n)) return HPC_SEARCH_SPLIT_TF32;
  if (d >= 64 && k <= 128 && hpc_tc_objective_supported(d, k, n)) return HPC_SEARCH_TF32;
  // above 128 centroids at d = 64 / 128 the split-BF16 products keep the
  // error window as narrow as split TF32, so that rows near a tie stay rare
  // with the method's own incumbents
  if (d >= 64 && form_supported(HPC_SEARCH_SPLIT_BF16, d, k, n)) return HPC_SEARCH_SPLIT_BF16;
  return HPC_SEARCH_SIMT;
}

int run_objective(hpc_ctx *c, Carver &cv, const float *X, int64_t n, int d, const float *C, int k,
                  const uint8_t *deg, double *f_out, int32_t *labels, int form_req = -1) {
  double *part = cv.take<double>((size_t)c->grid_bound);
  int64_t *queue = cv.take<int64_t>((size_t)c->L.num_sms * HPC_OBJ_QUEUE_CAP);
  unsigned char *cent = cv.take<unsigned char>(HPC_OBJ_CENT_BYTES);
  ObjArgsHost h{};
  h.cent_scratch = cent;
  h.cent_scratch_bytes = (int64_t)HPC_OBJ_CENT_BYTES;
  h.queue = queue;
  h.queue_cap = HPC_OBJ_QUEUE_CAP;
  h.queue_ctas = c->L.num_sms;
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
  h.stats = stats_ptr(c);
  int form = form_req >= 0 ? form_req : objective_form(c, d, k, n);
  if (!X || !aligned16(X)) form = HPC_SEARCH_SIMT;
  int rc = HPC_ERR_UNSUPPORTED;
  if (form == HPC_SEARCH_SPLIT_TF32)
    rc = hpc_tcs_objective_launch(c->L, h);
  else if (form == HPC_SEARCH_TF32)
    rc = hpc_tc_objective_launch(c->L, h);
  else if (form == HPC_SEARCH_SPLIT_BF16)
    rc = hpc_tcb_objective_launch(c->L, h);
  if (rc == HPC_ERR_UNSUPPORTED) rc = hpc_objective_launch(c->L, h);
  if (rc == HPC_ERR_CUDA) return cuda_fail(c, cudaGetLastError(), "objective launch");
  if (rc) return fail(c, rc, "objective: unsupported shape");
  c->launches += 1;
  return HPC_OK;
}

__global__ void timestamp_kernel(unsigned long long *out) { *out = hpc_globaltimer(); }

// Block 0 waits at a grid barrier that block 1 never reaches; the bounded
// wait gives up after limit_ns and records HPC_ERR_TIMEOUT.
__global__ void selftest_timeout_kernel(hpc_gridbar *bar, int *status, uint64_t limit_ns) {
  if (blockIdx.x == 1) return;
  hpc_grid_sync(bar, status, 2u, limit_ns);
}

// Round set-up on the device: the round's tables are read from the pinned
// staging slot (mapped into the device's address space, loads that bypass
// the caches) and the task headers are cleared.  One kernel instead of a
// host-to-device copy and a memset keeps the round's stream off the copy
// engines, where a large copy issued on another stream (the next batch of
// data) would hold the round back until it has finished.
__global__ void round_setup_kernel(uint4 *tab, const uint4 *src, size_t n16, uint4 *hdr,
                                   size_t hdr16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
    tab[i] = __ldcv(src + i);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < hdr16; i += stride)
    hdr[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Pinned host slot `slot` of the staging ring, at least `bytes` long; waits
// for the launch that read it last time.
int stage_acquire(hpc_ctx *c, int slot, size_t bytes, char **out) {
  cudaError_t e;
  if (c->stage_used[slot]) {
    if ((e = cudaEventSynchronize(c->stage_ev[slot])) != cudaSuccess)
      return cuda_fail(c, e, "staging wait");
    c->stage_used[slot] = false;
  }
  if (c->stage_bytes[slot] < bytes) {
    if (c->stage_host[slot]) cudaFreeHost(c->stage_host[slot]);
    c->stage_host[slot] = nullptr;
    c->stage_dev[slot] = nullptr;
    c->stage_bytes[slot] = 0;
    const size_t want = std::max(bytes, (size_t)1 << 16);
    if ((e = cudaHostAlloc(&c->stage_host[slot], want, cudaHostAllocMapped)) != cudaSuccess) {
      cudaGetLastError();
      c->stage_host[slot] = nullptr;
      return fail(c, HPC_ERR_NOMEM, "pinned staging allocation failed");
    }
    if ((e = cudaHostGetDevicePointer(&c->stage_dev[slot], c->stage_host[slot], 0)) !=
        cudaSuccess) {
      cudaFreeHost(c->stage_host[slot]);
      c->stage_host[slot] = nullptr;
      c->stage_dev[slot] = nullptr;
      return cuda_fail(c, e, "staging device pointer");
    }
    c->stage_bytes[slot] = want;
  }
  if (!c->stage_ev[slot] &&
      (e = cudaEventCreateWithFlags(&c->stage_ev[slot], cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(c, e, "event");
  *out = static_cast<char *>(c->stage_host[slot]);
  return HPC_OK;
}

// Marks the copies just issued from `slot`; the next call uses the next slot.
int stage_release(hpc_ctx *c, int slot) {
  const cudaError_t e = cudaEventRecord(c->stage_ev[slot], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "event record");
  c->stage_used[slot] = true;
  c->stage_next = (slot + 1) % 4;
  return HPC_OK;
}

}  // namespace

int64_t hpc_grid_bound(const hpc_launch &L) { return (int64_t)L.num_sms * 8; }

// ---------------------------------------------------------------------------
// Batched round (Algorithms 3-5): set-up shared by hpc_round and
// hpc_round_prepare, and the launches of one round.

// Everything one round needs once its descriptor tables are on the device.
struct hpc_round_plan {
  int W = 0, d = 0;
  int64_t n = 0, smax = 0;
  uint64_t seed = 0;
  int strategy = 0;  // HPC_HYBRID is resolved on the device from the round
  int32_t n_competitive = 0;
  const float *X = nullptr;
  float *C = nullptr;
  uint8_t *deg = nullptr;
  double *fhat = nullptr, *f_new = nullptr;
  int32_t *iters = nullptr;
  uint8_t *accepted = nullptr;
  TaskHeader *hdr = nullptr;
  const hpc_round_worker *rw_d = nullptr;
  const hpc_sample_task *st_d = nullptr;
  std::vector<char> host;  // host image of the tables of a prepared round
  std::vector<KppLaunch> kl;
  std::vector<LloydLaunch> ll;
};

static int round_check(hpc_ctx *c, const float *X, int64_t n, int32_t d, const hpc_batch *b,
                       int32_t strategy, int32_t max_iter, int32_t n_candidates, int32_t prec) {
  if (int rc = check_dims(c, d)) return rc;
  if (n < 1 || !X || b->W < 1 || b->W > HPC_MAX_WORKERS || !b->s || !b->k || !b->C_off ||
      !b->K_off || !b->C || !b->degenerate || !b->fhat || b->worker0 < 0)
    return fail(c, HPC_ERR_ARG, "malformed batch");
  if (strategy != HPC_COMPETITIVE && strategy != HPC_COOPERATIVE && strategy != HPC_HYBRID)
    return fail(c, HPC_ERR_ARG, "unknown strategy");
  if (n_candidates < 1 || n_candidates > 8) return fail(c, HPC_ERR_ARG, "n_candidates in [1, 8]");
  if (max_iter < 0 || max_iter > HPC_MAX_ITER) return fail(c, HPC_ERR_ARG, "max_iter out of range");
  if (!aligned16(X) || !aligned16(b->C)) return fail(c, HPC_ERR_ARG, "unaligned");
  int kmax = 0;
  for (int w = 0; w < b->W; ++w) {
    if (b->s[w] < 1 || b->k[w] < 1 || b->C_off[w] < 0 || b->K_off[w] < 0 || (b->C_off[w] & 3))
      return fail(c, HPC_ERR_ARG, "malformed batch entry");
    kmax = std::max(kmax, (int)b->k[w]);
  }
  int mode = 0;
  return prec_lloyd_mode(c, prec, d, kmax, &mode);
}

// Device bytes of one round's scratch and tables (tables: *tab_bytes).
static size_t round_scratch_bytes(const hpc_ctx *c, const hpc_batch *b, int d, int L,
                                  size_t *tab_bytes) {
  const int W = b->W;
  const int nchunks = (W + HPC_ROUND_CHUNK - 1) / HPC_ROUND_CHUNK;
  size_t need = pad256((size_t)W * sizeof(TaskHeader)) + 4096;
  for (int w = 0; w < W; ++w) {
    const int64_t s = b->s[w];
    const int k = b->k[w];
    need += pad256((size_t)s * d * 4) + pad256((size_t)k * d * 4) + pad256((size_t)k) +
            pad256((size_t)3 * k * d * 8) + pad256((size_t)3 * k * 4) + pad256((size_t)s * 4) +
            pad256((size_t)L * s * 4) + pad256((size_t)c->grid_bound * 8) + pad256((size_t)L * 8) +
            tcl_ws(d, k, s);
  }
  int kmax = 0;
  for (int w = 0; w < W; ++w) kmax = std::max(kmax, (int)b->k[w]);
  need += tcl_queue_ws(c, d, kmax);
  *tab_bytes = pad256((size_t)W * sizeof(hpc_sample_task)) + pad256((size_t)W * sizeof(hpc_round_worker)) +
               pad256((size_t)W * sizeof(hpc_kpp_task)) + pad256((size_t)W * sizeof(hpc_lloyd_task)) +
               3 * (size_t)nchunks * pad256((size_t)c->grid_bound * 4);
  return need + pad256((size_t)W * 8) + 2 * pad256((size_t)W * 4) + *tab_bytes + 1024;
}

// Carves the round's scratch from cv, writes the descriptor tables into
// tab_host (their device home is tab_dev, same layout) and plans the
// persistent launches.
static int round_build(hpc_ctx *c, const float *X, int64_t n, int d, const hpc_batch *b,
                       int strategy, uint64_t seed, uint32_t round, int max_iter, double rel_tol,
                       int L, Carver &cv, char *tab_host, char *tab_dev, size_t tab_bytes,
                       int32_t *uprev, hpc_round_plan &p, int tc_mode) {
  const int W = b->W;
  const int nchunks = (W + HPC_ROUND_CHUNK - 1) / HPC_ROUND_CHUNK;
  int64_t smax = 0;
  for (int w = 0; w < W; ++w) smax = std::max<int64_t>(smax, b->s[w]);
  TaskHeader *hdr = cv.take<TaskHeader>((size_t)W);
  double *fw = cv.take<double>((size_t)W);
  int32_t *itw = cv.take<int32_t>((size_t)W);
  // uprev: each worker's updates in its latest run (W of them, kept between
  // rounds by the caller), read by this round's Lloyd plan and rewritten by it
  Carver th{tab_host, 0, tab_bytes}, td{tab_dev, 0, tab_bytes};
  hpc_sample_task *st_h = th.take<hpc_sample_task>((size_t)W);
  hpc_sample_task *st_d = td.take<hpc_sample_task>((size_t)W);
  hpc_round_worker *rw_h = th.take<hpc_round_worker>((size_t)W);
  hpc_round_worker *rw_d = td.take<hpc_round_worker>((size_t)W);
  hpc_kpp_task *kt_h = th.take<hpc_kpp_task>((size_t)W);
  hpc_kpp_task *kt_d = td.take<hpc_kpp_task>((size_t)W);
  hpc_lloyd_task *lt_h = th.take<hpc_lloyd_task>((size_t)W);
  hpc_lloyd_task *lt_d = td.take<hpc_lloyd_task>((size_t)W);
  for (int w = 0; w < W; ++w) {
    const int64_t s = b->s[w];
    const int k = b->k[w];
    float *S = cv.take<float>((size_t)s * d);
    float *Cn = cv.take<float>((size_t)k * d);
    uint8_t *dn = cv.take<uint8_t>((size_t)k);
    st_h[w] = hpc_sample_task{S, nullptr, s, (uint32_t)(b->worker0 + w)};
    rw_h[w] = hpc_round_worker{s, b->C_off[w], b->K_off[w], k, b->group ? b->group[w] : 0, Cn, dn,
                          fw + w, itw + w};
    hpc_kpp_task &kt = kt_h[w];
    kt = hpc_kpp_task{};
    kt.S = S;
    kt.s = s;
    kt.k = k;
    kt.worker = (uint32_t)(b->worker0 + w);
    kt.C = Cn;
    kt.deg = dn;
    kpp_task_scratch(c, cv, hdr + w, s, L, kt);
    hpc_lloyd_task &lt = lt_h[w];
    lt = hpc_lloyd_task{};
    lt.S = S;
    lt.s = s;
    lt.k = k;
    lt.C = Cn;
    lt.deg = dn;
    lt.f_out = fw + w;
    lt.iters_out = itw + w;
    lloyd_task_scratch(c, cv, hdr + w, d, k, lt);
    // the incumbent rule runs at the end of the worker's Lloyd run
    lt.fhat = b->fhat + w;
    lt.C_inc = b->C + b->C_off[w];
    lt.deg_inc = b->degenerate + b->K_off[w];
    lt.f_new = b->f_new ? b->f_new + w : nullptr;
    lt.iters_rep = b->iters ? b->iters + w : nullptr;
    lt.uprev = uprev + w;
    lt.accepted = b->accepted ? b->accepted + w : nullptr;
    lt.t_done = b->t_done ? reinterpret_cast<unsigned long long *>(b->t_done) + w : nullptr;
  }
  // the tensor-core Lloyd's queues, shared by the chunks' launches (which
  // run one after another)
  int kall = 0;
  for (int w = 0; w < W; ++w) kall = std::max(kall, (int)b->k[w]);
  int64_t *lqueue = hpc_tcl_supported(d, kall)
                        ? cv.take<int64_t>((size_t)c->L.num_sms * HPC_LLOYD_QUEUE_CAP) : nullptr;
  // plans of the persistent launches, HPC_ROUND_CHUNK workers each
  p.kl.assign(nchunks, KppLaunch{});
  p.ll.assign(nchunks, LloydLaunch{});
  for (int ch = 0; ch < nchunks; ++ch) {
    const int w0 = ch * HPC_ROUND_CHUNK, cw = std::min(W - w0, HPC_ROUND_CHUNK);
    int kk = 0;
    for (int w = w0; w < w0 + cw; ++w) kk = std::max(kk, b->k[w]);
    KppLaunch &kh = p.kl[ch];
    kh.W = cw;
    kh.tasks = kt_h + w0;
    kh.block_task_host = th.take<int>((size_t)c->grid_bound);
    kh.tasks_dev = kt_d + w0;
    kh.block_task_dev = td.take<int>((size_t)c->grid_bound);
    kh.d = d;
    kh.kmax = kk;
    kh.L = L;
    kh.seed = seed;
    kh.round = round;
    kh.status = c->dwords;
    kh.max_blocks = c->grid_bound;
    kh.chunk_cap = c->grid_bound;
    if (int rc = hpc_kmeanspp_plan(c->L, kh)) return plan_fail(c, rc, "kmeanspp: unsupported shape");
    LloydLaunch &lh = p.ll[ch];
    lh.W = cw;
    lh.tasks = lt_h + w0;
    lh.block_task_host = th.take<int>(2 * (size_t)c->grid_bound);  // first tasks, then follow-ups
    lh.tasks_dev = lt_d + w0;
    lh.block_task_dev = td.take<int>(2 * (size_t)c->grid_bound);
    lh.d = d;
    lh.kmax = kk;
    lh.max_iter = max_iter;
    lh.tol = rel_tol;
    lh.status = c->dwords;
    lh.max_blocks = c->grid_bound;
    lh.task_blocks = c->grid_bound;
    lh.tc_mode = tc_mode;
    lh.stats = stats_ptr(c);
    lh.queue = lqueue;
    lh.queue_cap = lqueue ? HPC_LLOYD_QUEUE_CAP : 0;
    lh.queue_ctas = c->L.num_sms;
    lh.pop = &hdr[w0].lpop;
    if (int rc = hpc_lloyd_plan(c->L, lh)) return plan_fail(c, rc, "lloyd: unsupported shape");
  }
  if (cv.off > cv.cap || th.off > th.cap) return fail(c, HPC_ERR_NOMEM, "round scratch layout overflow");
  p.W = W;
  p.d = d;
  p.n = n;
  p.smax = smax;
  p.seed = seed;
  p.strategy = strategy;
  p.n_competitive = b->n_competitive;
  p.X = X;
  p.C = b->C;
  p.deg = b->degenerate;
  p.fhat = b->fhat;
  p.f_new = b->f_new;
  p.iters = b->iters;
  p.accepted = b->accepted;
  p.hdr = hdr;
  p.rw_d = rw_d;
  p.st_d = st_d;
  return HPC_OK;
}

// One round: the set-up launch (tables, task headers), the sampling launch
// (which also selects every worker's base) and per chunk of workers the
// K-means++ and Lloyd launches, each with its planning launch when batched
// (each Lloyd task applies the incumbent rule when its run is done); no host
// synchronisation, no allocation (a stream capture can record it).  The round index is `round`,
// or *round_dev when that is given (a prepared round, whose last Lloyd
// launch then advances it).
// Records timing event i of a round on the context's stream; inside a
// stream capture the record becomes a node of the graph, so that every
// replay takes the time again.
static int timing_mark(hpc_ctx *c, int i, int kind) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
  if (e == cudaSuccess)
    e = cs == cudaStreamCaptureStatusNone
            ? cudaEventRecord(c->tev[i], c->stream)
            : cudaEventRecordWithFlags(c->tev[i], c->stream, cudaEventRecordExternal);
  if (e != cudaSuccess) return cuda_fail(c, e, "timing event");
  c->tev_kind[i] = kind;
  c->tev_n = i + 1;
  return HPC_OK;
}

// Enqueues a built round.  `tab_src` (device-visible pinned memory,
// `tab_bytes` long, a multiple of 16) holds the tables that the set-up
// kernel copies to `tab_dev`; null when they are already there.
static int round_enqueue(hpc_ctx *c, const hpc_round_plan &p, uint32_t *round_dev, uint32_t round,
                         char *tab_dev, const char *tab_src, size_t tab_bytes) {
  const bool timed = c->timing && 2 + 2 * (int)p.kl.size() <= HPC_TIMING_EVENTS;
  int ev = 0;
  c->tev_n = 0;
  if (timed)
    if (int rc = timing_mark(c, ev++, -1)) return rc;
  {
    const size_t n16 = tab_src ? tab_bytes / 16 : 0;
    const size_t hdr16 = (size_t)p.W * sizeof(TaskHeader) / 16;
    const size_t units = std::max(n16, hdr16);
    const int blocks = (int)std::min<size_t>((size_t)c->L.num_sms, (units + 1023) / 1024 + 1);
    round_setup_kernel<<<blocks, 256, 0, c->stream>>>(
        reinterpret_cast<uint4 *>(tab_dev), reinterpret_cast<const uint4 *>(tab_src), n16,
        reinterpret_cast<uint4 *>(p.hdr), hdr16);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "round set-up");
    c->launches += 1;
  }
  hpc_base_args base{};
  base.wk = p.rw_d;
  base.W = p.W;
  base.strategy = p.strategy;
  base.n_competitive = p.n_competitive;
  base.round_dev = round_dev;
  base.round = round;
  base.fhat = p.fhat;
  base.Cpool = p.C;
  base.Kpool = p.deg;
  base.d = p.d;
  base.f_new = p.f_new;
  base.iters = p.iters;
  base.accepted = p.accepted;
  if (int rc = hpc_sample_batch_launch(c->L, p.X, p.n, p.d, p.seed, round, round_dev, p.W, p.st_d,
                                       p.smax, base))
    return plan_fail(c, rc, "sample launch");
  c->launches += 1;
  if (timed)
    if (int rc = timing_mark(c, ev++, 0)) return rc;
  for (size_t ch = 0; ch < p.kl.size(); ++ch) {
    KppLaunch kh = p.kl[ch];
    kh.round = round;
    kh.round_dev = round_dev;
    if (int rc = hpc_kmeanspp_run(c->L, kh)) return plan_fail(c, rc, "kmeanspp launch");
    if (timed)
      if (int rc = timing_mark(c, ev++, 1)) return rc;
    LloydLaunch lh = p.ll[ch];
    lh.round_advance = ch + 1 == p.kl.size() ? round_dev : nullptr;
    if (int rc = hpc_lloyd_run(c->L, lh)) return plan_fail(c, rc, "lloyd launch");
    if (timed)
      if (int rc = timing_mark(c, ev++, 2)) return rc;
    c->launches += 2 + (kh.W > 1 && kh.W <= HPC_KPP_SPLIT_MAX ? 1 : 0) +
                   (lh.W > 1 && lh.form == HPC_SEARCH_SPLIT_BF16 ? 1 : 0);
  }
  return HPC_OK;
}

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
  c->force_form = -1;
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
  if (c->upd) cudaFree(c->upd);
  for (int i = 0; i < 4; ++i) {
    if (c->stage_host[i]) cudaFreeHost(c->stage_host[i]);
    if (c->stage_ev[i]) cudaEventDestroy(c->stage_ev[i]);
  }
  if (c->plan_mem) cudaFree(c->plan_mem);
  for (int i = 0; i < HPC_TIMING_EVENTS; ++i)
    if (c->tev[i]) cudaEventDestroy(c->tev[i]);
  delete c->plan;
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
  int mode = 0;
  if (int rc = prec_lloyd_mode(c, prec, d, k, &mode)) return rc;
  if (!aligned16(S) || !aligned16(C_inout)) return fail(c, HPC_ERR_ARG, "unaligned");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, lloyd_ws(c, d, k, s))) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  return run_lloyd(c, cv, S, s, d, k, C_inout, degenerate_inout, max_iter, rel_tol, labels_out,
                   f_out, iters_out, mode);
}

int hpc_objective(hpc_ctx *c, const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                  const uint8_t *degenerate, int32_t prec, double *f_out, int32_t *labels_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (n < 0 || k < 1 || !C || !f_out || (n > 0 && !X)) return fail(c, HPC_ERR_ARG, "bad sizes");
  int form = -1;
  if (prec == HPC_BF16) {
    if (!hpc_tcl_supported(d, k))
      return fail(c, HPC_ERR_UNSUPPORTED, "HPC_BF16: split-BF16 search not built for this shape");
    if (n > 0) form = HPC_SEARCH_SPLIT_BF16;
  } else if (prec == HPC_FP8) {
    return fail(c, HPC_ERR_UNSUPPORTED, "HPC_FP8 is not built");
  } else if (prec != HPC_FP32) {
    return fail(c, HPC_ERR_ARG, "unknown precision");
  }
  if ((X && !aligned16(X)) || !aligned16(C)) return fail(c, HPC_ERR_ARG, "unaligned");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, obj_ws(c))) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  return run_objective(c, cv, X, n, d, C, k, degenerate, f_out, labels_out, form);
}

int hpc_set_objective_form(hpc_ctx *c, int32_t d, int32_t k, int32_t form) {
  if (!c || d < 1 || d > 128 || k < 1 || form < -1 || form > HPC_SEARCH_SPLIT_BF16)
    return fail(c, HPC_ERR_ARG, "bad objective form");
  if (form >= 0 && !form_supported(form, d, k, 1))
    return fail(c, HPC_ERR_UNSUPPORTED, "objective form not built for this shape");
  auto &v = c->forms;
  v.erase(std::remove_if(v.begin(), v.end(),
                         [&](const std::pair<int64_t, int> &f) { return f.first == form_key(d, k); }),
          v.end());
  if (form >= 0) v.emplace_back(form_key(d, k), form);
  return HPC_OK;
}

int hpc_objective_form(hpc_ctx *c, int64_t n, int32_t d, int32_t k) {
  if (!c || d < 1 || d > 128 || k < 1 || n < 0) return HPC_ERR_ARG;
  return objective_form(c, d, k, n);
}

int hpc_lloyd_cta_plan(int32_t W, const int64_t *s, const int32_t *k, const int32_t *u,
                       int32_t ctas, int32_t *cta_task, int32_t *list, int32_t *nlist,
                       int32_t *next, int32_t *nblocks) {
  if (!s || !k || !u || !cta_task || !list || !nlist || !next || !nblocks) return HPC_ERR_ARG;
  return hpc_tcl_cta_plan(W, s, k, u, ctas, cta_task, list, nlist, next, nblocks);
}

int hpc_lloyd_schedule(hpc_ctx *c, int64_t s, int32_t d, int32_t k, int32_t *out, int32_t nout) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (s < 1 || k < 1 || !out || nout < 1) return fail(c, HPC_ERR_ARG, "bad sizes");
  cudaSetDevice(c->device);
  hpc_lloyd_task t{};
  t.s = s;
  t.k = k;
  LloydLaunch h{};
  h.W = 1;
  h.tasks = &t;
  h.d = d;
  h.kmax = k;
  h.max_blocks = c->grid_bound;
  h.task_blocks = c->grid_bound;
  h.tc_mode = c->use_tc;
  if (int rc = hpc_lloyd_plan(c->L, h)) return plan_fail(c, rc, "lloyd: unsupported shape");
  const int32_t v[5] = {(int32_t)h.grid, h.smem_sums, h.xstage, (int32_t)h.smem, h.form};
  for (int i = 0; i < nout && i < 5; ++i) out[i] = v[i];
  return HPC_OK;
}

int hpc_set_search_stats(hpc_ctx *c, int32_t on) {
  if (!c || on < 0 || on > 1) return HPC_ERR_ARG;
  c->stats_on = on;
  return HPC_OK;
}

int hpc_search_stats(hpc_ctx *c, int64_t *out, int32_t reset) {
  if (!c || !out) return HPC_ERR_ARG;
  cudaSetDevice(c->device);
  unsigned long long *p =
      reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(c->dwords) + 64);
  unsigned long long v[4];
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(v, p, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(p, 0, sizeof(v));
  if (e != cudaSuccess) return cuda_fail(c, e, "search counters");
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)v[i];
  return HPC_OK;
}

int hpc_set_phase_timing(hpc_ctx *c, int32_t on) {
  if (!c || on < 0 || on > 1) return HPC_ERR_ARG;
  cudaSetDevice(c->device);
  if (on && !c->tev[0]) {
    for (int i = 0; i < HPC_TIMING_EVENTS; ++i) {
      cudaError_t e = cudaEventCreate(&c->tev[i]);
      if (e != cudaSuccess) return cuda_fail(c, e, "timing events");
    }
  }
  c->timing = on;
  c->tev_n = 0;
  return HPC_OK;
}

int hpc_phase_times(hpc_ctx *c, float *ms_out) {
  if (!c || !ms_out) return HPC_ERR_ARG;
  if (c->tev_n < 2) return fail(c, HPC_ERR_ARG, "no timed round");
  cudaSetDevice(c->device);
  cudaError_t e = cudaEventSynchronize(c->tev[c->tev_n - 1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "timing wait");
  float acc[3] = {0.0f, 0.0f, 0.0f};
  for (int i = 1; i < c->tev_n; ++i) {
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, c->tev[i - 1], c->tev[i])) != cudaSuccess)
      return cuda_fail(c, e, "timing read");
    const int kind = c->tev_kind[i];
    if (kind >= 0 && kind < 3) acc[kind] += ms;
  }
  for (int i = 0; i < 3; ++i) ms_out[i] = acc[i];
  return HPC_OK;
}

namespace {

// Times `reps` calls of the objective in search form `form` (after one
// warm-up call) with CUDA events on the context's stream: *ms per call.
int time_form(hpc_ctx *c, const Carver &cv, double *f, const float *X, int64_t n, int32_t d,
              const float *C, int32_t k, const uint8_t *degenerate, int32_t reps, int form,
              cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  c->force_form = form;
  Carver cw = cv;
  int rc = run_objective(c, cw, X, n, d, C, k, degenerate, f, nullptr);  // warm-up
  cudaEventRecord(e0, c->stream);
  for (int r = 0; r < reps && rc == HPC_OK; ++r) {
    cw = cv;
    rc = run_objective(c, cw, X, n, d, C, k, degenerate, f, nullptr);
  }
  cudaEventRecord(e1, c->stream);
  c->force_form = -1;
  if (rc != HPC_OK) return rc;
  float t = 0.0f;
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune timing");
  if ((rc = hpc_sync_status(c)) != HPC_OK) return rc;  // a device error ends the sweep
  *ms = t / (float)reps;
  return HPC_OK;
}

int check_autotune_args(hpc_ctx *c, const float *X, int64_t n, int32_t d, const float *C,
                        int32_t k, int32_t reps) {
  if (int rc = check_dims(c, d)) return rc;
  if (n < 1 || k < 1 || !X || !C || reps < 1 || reps > 1000)
    return fail(c, HPC_ERR_ARG, "bad sizes");
  if (!aligned16(X) || !aligned16(C)) return fail(c, HPC_ERR_ARG, "unaligned");
  return HPC_OK;
}

// Times the forms in `order` (count entries; those with timed_mask[i] == 0
// are skipped when the mask is given) and
// keeps the fastest; within 1% of it the built-in form stays, so that timing
// noise does not move the choice from run to run.
int autotune_forms(hpc_ctx *c, const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                   const uint8_t *degenerate, int32_t reps, const int *order, int count,
                   const int32_t *timed_mask, int32_t *form_out, float *ms_out,
                   int32_t *timed_out) {
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, obj_ws(c) + 512)) return rc;
  if (int st = hpc_sync_status(c)) return st;  // start from a clean status
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  double *f = cv.take<double>(1);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(c, cudaGetLastError(), "event create");
  int best = -1, timed = 0;
  float best_ms = 0.0f, tms[HPC_NFORMS] = {-1.0f, -1.0f, -1.0f, -1.0f};
  int rc = HPC_OK;
  for (int i = 0; i < count && rc == HPC_OK; ++i) {
    const int form = order[i];
    if (timed_mask && !timed_mask[i]) continue;  // guided: predicted too slow
    float ms = 0.0f;
    rc = time_form(c, cv, f, X, n, d, C, k, degenerate, reps, form, e0, e1, &ms);
    if (rc != HPC_OK) break;
    ++timed;
    tms[form] = ms;
    if (best < 0 || ms < best_ms) {
      best = form;
      best_ms = ms;
    }
  }
  c->force_form = -1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != HPC_OK) return rc;
  const int bi = builtin_form(d, k, n);
  if (bi != best && tms[bi] > 0.0f && tms[bi] <= 1.01f * best_ms) best = bi;
  if (ms_out)
    for (int q = 0; q < HPC_NFORMS; ++q) ms_out[q] = tms[q];
  if (form_out) *form_out = best;
  if (timed_out) *timed_out = timed;
  return hpc_set_objective_form(c, d, k, best);
}

// ---- cost-model inputs (host) ----

// log2(max ||c||^2 / min ||c_i - c_j||^2) over live centroids, clamped to
// [0, 40] and divided by 40; 1 when two live centroids coincide, 0 with
// fewer than two live.
float cm_separation(const float *Ch, const uint8_t *degh, int d, int k) {
  double cmax2 = 0.0, minsep = -1.0;
  int live = 0;
  for (int i = 0; i < k; ++i) {
    if (degh && degh[i]) continue;
    ++live;
    double s = 0.0;
    for (int t = 0; t < d; ++t) s += (double)Ch[(size_t)i * d + t] * Ch[(size_t)i * d + t];
    cmax2 = std::max(cmax2, s);
    for (int j = 0; j < i; ++j) {
      if (degh && degh[j]) continue;
      double q = 0.0;
      for (int t = 0; t < d; ++t) {
        const double u = (double)Ch[(size_t)i * d + t] - Ch[(size_t)j * d + t];
        q += u * u;
      }
      if (minsep < 0.0 || q < minsep) minsep = q;
    }
  }
  if (live < 2) return 0.0f;
  if (minsep <= 0.0) return 1.0f;
  if (cmax2 <= 0.0) return 0.0f;
  const double r = std::log2(cmax2 / minsep);
  return (float)(std::min(std::max(r, 0.0), 40.0) / 40.0);
}

void cm_features(int d, int k, float sep, float *out) {
  const int cols = k <= 32 ? 32 : k <= 64 ? 64 : k <= 128 ? 128 : k <= 256 ? 256 : 512;
  for (int form = 0; form < 3; ++form) {
    float *r = out + form * HPC_CM_NFEAT;
    r[0] = (float)(std::log2((double)d) / 7.0);
    r[1] = (float)(std::log2((double)k) / 9.0);
    r[2] = (float)((double)cols / k - 1.0);
    r[3] = sep;
    r[4] = form == HPC_SEARCH_SIMT ? 1.0f : 0.0f;
    r[5] = form == HPC_SEARCH_SPLIT_TF32 ? 1.0f : 0.0f;
    r[6] = form == HPC_SEARCH_TF32 ? 1.0f : 0.0f;
    r[7] = k > 128 ? 1.0f : 0.0f;
  }
}

}  // namespace

int hpc_autotune_objective(hpc_ctx *c, const float *X, int64_t n, int32_t d, const float *C,
                           int32_t k, const uint8_t *degenerate, int32_t reps, int32_t *form_out,
                           float *ms_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_autotune_args(c, X, n, d, C, k, reps)) return rc;
  int order[HPC_NFORMS], count = 0;
  for (int form = HPC_SEARCH_SIMT; form <= HPC_SEARCH_SPLIT_BF16; ++form)
    if (form_supported(form, d, k, n)) order[count++] = form;
  return autotune_forms(c, X, n, d, C, k, degenerate, reps, order, count, nullptr, form_out,
                        ms_out, nullptr);
}

int hpc_costmodel_plan(const float *pred, const int32_t *supported, float margin,
                       int32_t *order_out, int32_t *timed_out) {
  if (!pred || !supported || !order_out || !timed_out || !(margin >= 0.0f)) return HPC_ERR_ARG;
  int order[3], count = 0;
  for (int f = 0; f < 3; ++f) {
    order_out[f] = -1;
    timed_out[f] = 0;
    if (!supported[f]) continue;
    if (!std::isfinite(pred[f])) return HPC_ERR_ARG;
    order[count++] = f;
  }
  // rank by predicted time, ties to the lower form index
  std::stable_sort(order, order + count, [&](int a, int b) { return pred[a] < pred[b]; });
  for (int i = 0; i < count; ++i) {
    order_out[i] = order[i];
    timed_out[i] =
        i == 0 || std::exp((double)pred[order[i]] - (double)pred[order[0]]) <= 1.0 + (double)margin
            ? 1
            : 0;
  }
  return count;
}

int hpc_costmodel_features(hpc_ctx *c, const float *C, const uint8_t *degenerate, int32_t d,
                           int32_t k, float *feats_out, int32_t *supported_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_dims(c, d)) return rc;
  if (k < 1 || k > 1 << 16 || !C || !feats_out) return fail(c, HPC_ERR_ARG, "bad sizes");
  cudaSetDevice(c->device);
  std::vector<float> Ch((size_t)k * d);
  std::vector<uint8_t> dh(degenerate ? (size_t)k : 0);
  cudaError_t e = cudaMemcpyAsync(Ch.data(), C, Ch.size() * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && degenerate)
    e = cudaMemcpyAsync(dh.data(), degenerate, dh.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cost-model inputs");
  cm_features(d, k, cm_separation(Ch.data(), degenerate ? dh.data() : nullptr, d, k), feats_out);
  if (supported_out)
    for (int form = 0; form < 3; ++form) supported_out[form] = form_supported(form, d, k, 1) ? 1 : 0;
  return HPC_OK;
}

namespace {
int check_cm_args(hpc_ctx *c, const void *params, const void *feats, int32_t N) {
  if (!params || !feats) return fail(c, HPC_ERR_ARG, "NULL cost-model array");
  if (N < 1 || N > (1 << 20)) return fail(c, HPC_ERR_ARG, "cost-model samples in [1, 2^20]");
  return HPC_OK;
}
}  // namespace

int hpc_costmodel_loss_grad(hpc_ctx *c, const float *params, const float *feats,
                            const float *targets, int32_t N, float *loss_out, float *grad_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_cm_args(c, params, feats, N)) return rc;
  if (!targets || !loss_out || !grad_out) return fail(c, HPC_ERR_ARG, "NULL cost-model array");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, hpc_cm_part_floats(N) * 4 + 256)) return rc;
  if (hpc_cm_grad_launch(c->L, params, feats, targets, N, reinterpret_cast<float *>(c->ws),
                         nullptr, nullptr, 0.0f, 1.0f, 1.0f, grad_out, loss_out))
    return cuda_fail(c, cudaGetLastError(), "cost-model gradient launch");
  c->launches += 2;
  return HPC_OK;
}

int hpc_costmodel_train(hpc_ctx *c, float *params, float *m, float *v, const float *feats,
                        const float *targets, int32_t N, int32_t steps, int32_t step0, float lr,
                        float *loss_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_cm_args(c, params, feats, N)) return rc;
  if (!targets || !m || !v) return fail(c, HPC_ERR_ARG, "NULL cost-model array");
  if (steps < 0 || step0 < 0 || !(lr > 0.0f) || !std::isfinite(lr))
    return fail(c, HPC_ERR_ARG, "bad training schedule");
  cudaSetDevice(c->device);
  if (int rc = ensure_ws(c, hpc_cm_part_floats(N) * 4 + 256)) return rc;
  for (int s = 0; s < steps; ++s) {
    const double t = (double)step0 + s + 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, t)), bc2 = (float)(1.0 - std::pow(0.999, t));
    if (hpc_cm_grad_launch(c->L, params, feats, targets, N, reinterpret_cast<float *>(c->ws), m,
                           v, lr, bc1, bc2, nullptr, loss_out ? loss_out + s : nullptr))
      return cuda_fail(c, cudaGetLastError(), "cost-model training launch");
    c->launches += 2;
  }
  return HPC_OK;
}

int hpc_costmodel_predict(hpc_ctx *c, const float *params, const float *feats, int32_t N,
                          float *out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_cm_args(c, params, feats, N)) return rc;
  if (!out) return fail(c, HPC_ERR_ARG, "NULL cost-model array");
  cudaSetDevice(c->device);
  if (hpc_cm_predict_launch(c->L, params, feats, N, out))
    return cuda_fail(c, cudaGetLastError(), "cost-model prediction launch");
  c->launches += 1;
  return HPC_OK;
}

int hpc_autotune_objective_guided(hpc_ctx *c, const float *X, int64_t n, int32_t d,
                                  const float *C, int32_t k, const uint8_t *degenerate,
                                  int32_t reps, const float *params, float margin,
                                  int32_t *form_out, float *ms_out, int32_t *timed_out) {
  if (!c) return HPC_ERR_ARG;
  if (int rc = check_autotune_args(c, X, n, d, C, k, reps)) return rc;
  if (!params || !(margin >= 0.0f)) return fail(c, HPC_ERR_ARG, "bad cost model or margin");
  float feats[3 * HPC_CM_NFEAT];
  int32_t sup[3];
  if (int rc = hpc_costmodel_features(c, C, degenerate, d, k, feats, sup)) return rc;
  for (int form = HPC_SEARCH_SIMT; form <= HPC_SEARCH_TF32; ++form)
    sup[form] = sup[form] && form_supported(form, d, k, n) ? 1 : 0;
  // predictions for the three forms, by the network on the device
  if (int rc = ensure_ws(c, 512 + obj_ws(c))) return rc;
  float *dfeat = reinterpret_cast<float *>(c->ws);
  float *dpred = dfeat + 3 * HPC_CM_NFEAT;
  float pred[3];
  cudaError_t e = cudaMemcpyAsync(dfeat, feats, sizeof(feats), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cost-model inputs");
  if (hpc_cm_predict_launch(c->L, params, dfeat, 3, dpred))
    return cuda_fail(c, cudaGetLastError(), "cost-model prediction launch");
  c->launches += 1;
  e = cudaMemcpyAsync(pred, dpred, sizeof(pred), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cost-model prediction");
  int32_t order[3], timed[3];
  const int count = hpc_costmodel_plan(pred, sup, margin, order, timed);
  if (count < 0) return fail(c, HPC_ERR_ARG, "cost model predicts a non-finite time");
  // the split-BF16 form is newer than the network's inputs: timed whenever
  // it is built
  int ord[HPC_NFORMS] = {order[0], order[1], order[2], HPC_SEARCH_SPLIT_BF16};
  int32_t tm[HPC_NFORMS] = {timed[0], timed[1], timed[2], 1};
  const int cnt = count + (form_supported(HPC_SEARCH_SPLIT_BF16, d, k, n) ? 1 : 0);
  if (cnt > count) {
    ord[count] = HPC_SEARCH_SPLIT_BF16;
    tm[count] = 1;
  }
  return autotune_forms(c, X, n, d, C, k, degenerate, reps, ord, cnt, tm, form_out, ms_out,
                        timed_out);
}

// ---- checkpoint of a worker batch ----------------------------------------

namespace {

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t W, d, strategy;
  uint32_t next_round;
  int32_t n_competitive;
  uint64_t seed;
  int64_t floats, flags;
  uint64_t checksum;  // FNV-1a (64-bit) of every byte after the header
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header layout");

const char kCkptMagic[8] = {'H', 'P', 'C', 'B', 'A', 'T', 'C', 'H'};

uint64_t fnv1a(const unsigned char *p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

// Per-worker descriptor as stored: s, k, group.
struct CkptWorker {
  int64_t s;
  int32_t k, group;
};

int ckpt_sizes(const hpc_batch *b, int d, int64_t *floats, int64_t *flags) {
  *floats = *flags = 0;
  for (int w = 0; w < b->W; ++w) {
    if (b->k[w] < 1 || b->s[w] < 1 || b->C_off[w] < 0 || b->K_off[w] < 0) return HPC_ERR_ARG;
    *floats += (int64_t)b->k[w] * d;
    *flags += b->k[w];
  }
  return HPC_OK;
}

size_t ckpt_bytes(int W, int64_t floats, int64_t flags) {
  return sizeof(CkptHeader) + (size_t)W * sizeof(CkptWorker) + (size_t)floats * 4 +
         (size_t)flags + (size_t)W * 8;
}

}  // namespace

int hpc_batch_save(hpc_ctx *c, const hpc_batch *b, int32_t d, uint32_t next_round, uint64_t seed,
                   int32_t strategy, void *host_buf, int64_t cap, int64_t *bytes_out) {
  if (!c || !b || !bytes_out || b->W < 1 || b->W > HPC_MAX_WORKERS || !b->s || !b->k ||
      !b->C_off || !b->K_off || !b->C || !b->degenerate || !b->fhat || d < 1 || d > 128)
    return fail(c, HPC_ERR_ARG, "malformed batch");
  int64_t floats = 0, flags = 0;
  if (ckpt_sizes(b, d, &floats, &flags)) return fail(c, HPC_ERR_ARG, "malformed batch entry");
  const size_t need = ckpt_bytes(b->W, floats, flags);
  *bytes_out = (int64_t)need;
  if (!host_buf) return HPC_OK;  // size query
  if (cap < (int64_t)need) return fail(c, HPC_ERR_ARG, "checkpoint buffer too small");
  cudaSetDevice(c->device);
  unsigned char *out = static_cast<unsigned char *>(host_buf);
  CkptHeader h{};
  memcpy(h.magic, kCkptMagic, 8);
  h.version = 1;
  h.W = b->W;
  h.d = d;
  h.strategy = strategy;
  h.next_round = next_round;
  h.n_competitive = b->n_competitive;
  h.seed = seed;
  h.floats = floats;
  h.flags = flags;
  CkptWorker *wk = reinterpret_cast<CkptWorker *>(out + sizeof(CkptHeader));
  float *cf = reinterpret_cast<float *>(wk + b->W);
  unsigned char *fl = reinterpret_cast<unsigned char *>(cf + floats);
  unsigned char *fh = fl + flags;
  cudaError_t e = cudaSuccess;
  int64_t of = 0, og = 0;
  for (int w = 0; w < b->W && e == cudaSuccess; ++w) {
    const int k = b->k[w];
    CkptWorker x{b->s[w], k, b->group ? b->group[w] : 0};
    memcpy(&wk[w], &x, sizeof(x));
    e = cudaMemcpyAsync(cf + of, b->C + b->C_off[w], (size_t)k * d * 4, cudaMemcpyDeviceToHost,
                        c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(fl + og, b->degenerate + b->K_off[w], (size_t)k, cudaMemcpyDeviceToHost,
                          c->stream);
    of += (int64_t)k * d;
    og += k;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(fh, b->fhat, (size_t)b->W * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint read");
  h.checksum = fnv1a(out + sizeof(CkptHeader), need - sizeof(CkptHeader));
  memcpy(out, &h, sizeof(h));
  return HPC_OK;
}

int hpc_batch_load(hpc_ctx *c, const hpc_batch *b, int32_t d, const void *host_buf, int64_t bytes,
                   uint32_t *next_round, uint64_t *seed, int32_t *strategy) {
  if (!c || !b || !host_buf || b->W < 1 || b->W > HPC_MAX_WORKERS || !b->s || !b->k ||
      !b->C_off || !b->K_off || !b->C || !b->degenerate || !b->fhat || d < 1 || d > 128)
    return fail(c, HPC_ERR_ARG, "malformed batch");
  const unsigned char *in = static_cast<const unsigned char *>(host_buf);
  if (bytes < (int64_t)sizeof(CkptHeader)) return fail(c, HPC_ERR_ARG, "checkpoint truncated");
  CkptHeader h;
  memcpy(&h, in, sizeof(h));
  if (memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
    return fail(c, HPC_ERR_ARG, "not a batch checkpoint");
  int64_t floats = 0, flags = 0;
  if (ckpt_sizes(b, d, &floats, &flags)) return fail(c, HPC_ERR_ARG, "malformed batch entry");
  if (h.W != b->W || h.d != d || h.floats != floats || h.flags != flags ||
      (h.strategy == HPC_HYBRID && h.n_competitive != b->n_competitive))
    return fail(c, HPC_ERR_ARG, "checkpoint does not match the batch");
  const size_t need = ckpt_bytes(b->W, floats, flags);
  if (bytes != (int64_t)need) return fail(c, HPC_ERR_ARG, "checkpoint size mismatch");
  if (fnv1a(in + sizeof(CkptHeader), need - sizeof(CkptHeader)) != h.checksum)
    return fail(c, HPC_ERR_ARG, "checkpoint checksum mismatch");
  const CkptWorker *wk = reinterpret_cast<const CkptWorker *>(in + sizeof(CkptHeader));
  for (int w = 0; w < b->W; ++w) {
    CkptWorker x;
    memcpy(&x, &wk[w], sizeof(x));
    if (x.s != b->s[w] || x.k != b->k[w] || x.group != (b->group ? b->group[w] : 0))
      return fail(c, HPC_ERR_ARG, "checkpoint workers differ from the batch");
  }
  cudaSetDevice(c->device);
  const float *cf = reinterpret_cast<const float *>(wk + b->W);
  const unsigned char *fl = reinterpret_cast<const unsigned char *>(cf + floats);
  const unsigned char *fh = fl + flags;
  cudaError_t e = cudaSuccess;
  int64_t of = 0, og = 0;
  for (int w = 0; w < b->W && e == cudaSuccess; ++w) {
    const int k = b->k[w];
    e = cudaMemcpyAsync(b->C + b->C_off[w], cf + of, (size_t)k * d * 4, cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->degenerate + b->K_off[w], fl + og, (size_t)k, cudaMemcpyHostToDevice,
                          c->stream);
    of += (int64_t)k * d;
    og += k;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->fhat, fh, (size_t)b->W * 8, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint write");
  if (next_round) *next_round = h.next_round;
  if (seed) *seed = h.seed;
  if (strategy) *strategy = h.strategy;
  return HPC_OK;
}

int hpc_timestamp(hpc_ctx *c, uint64_t *dev_out) {
  if (!c || !dev_out) return HPC_ERR_ARG;
  cudaSetDevice(c->device);
  timestamp_kernel<<<1, 1, 0, c->stream>>>(reinterpret_cast<unsigned long long *>(dev_out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "timestamp launch");
  c->launches += 1;
  return HPC_OK;
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
  if (int rc = round_check(c, X, n, d, b, strategy, max_iter, n_candidates, prec)) return rc;
  cudaSetDevice(c->device);
  size_t tab_bytes = 0;
  const size_t need = round_scratch_bytes(c, b, d, n_candidates, &tab_bytes);
  if (int rc = ensure_ws(c, need)) return rc;
  if (int rc = ensure_upd(c, b->W)) return rc;
  Carver cv{reinterpret_cast<char *>(c->ws), 0, c->ws_bytes};
  char *tab_dev = cv.take<char>(tab_bytes);
  char *tab_host = nullptr;
  const int slot = c->stage_next;
  if (int rc = stage_acquire(c, slot, tab_bytes, &tab_host)) return rc;
  int kmax = 0, mode = 0;
  for (int w = 0; w < b->W; ++w) kmax = std::max(kmax, (int)b->k[w]);
  if (int rc = prec_lloyd_mode(c, prec, d, kmax, &mode)) return rc;
  hpc_round_plan p;
  if (int rc = round_build(c, X, n, d, b, strategy, seed, round, max_iter, rel_tol, n_candidates,
                           cv, tab_host, tab_dev, tab_bytes, c->upd, p, mode))
    return rc;
  // the set-up launch reads the tables from the pinned staging slot
  const int rc = round_enqueue(c, p, nullptr, round, tab_dev, (const char *)c->stage_dev[slot],
                               tab_bytes);
  if (int rr = stage_release(c, slot)) return rc ? rc : rr;
  return rc;
}

int hpc_round_prepare(hpc_ctx *c, const float *X, int64_t n, int32_t d, const hpc_batch *b,
                      int32_t strategy, uint64_t seed, uint32_t round0, int32_t max_iter,
                      double rel_tol, int32_t n_candidates, int32_t prec) {
  if (!c || !b) return HPC_ERR_ARG;
  if (int rc = round_check(c, X, n, d, b, strategy, max_iter, n_candidates, prec)) return rc;
  cudaSetDevice(c->device);
  cudaError_t e;
  size_t tab_bytes = 0;
  const size_t need = round_scratch_bytes(c, b, d, n_candidates, &tab_bytes) + 256;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "sync");
  if (need > c->plan_bytes) {
    if (c->plan_mem) cudaFree(c->plan_mem);
    c->plan_mem = nullptr;
    c->plan_bytes = 0;
    if ((e = cudaMalloc(&c->plan_mem, need)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HPC_ERR_NOMEM, "prepared-round allocation failed");
    }
    c->plan_bytes = need;
  }
  if (!c->plan) c->plan = new hpc_round_plan();
  hpc_round_plan &p = *c->plan;
  p = hpc_round_plan();
  Carver cv{reinterpret_cast<char *>(c->plan_mem), 0, c->plan_bytes};
  c->plan_round = cv.take<uint32_t>(1);
  char *tab_dev = cv.take<char>(tab_bytes);
  int32_t *uprev = cv.take<int32_t>((size_t)b->W);  // no run yet: zero below
  p.host.assign(tab_bytes, 0);
  int kmax = 0, mode = 0;
  for (int w = 0; w < b->W; ++w) kmax = std::max(kmax, (int)b->k[w]);
  if (int rc = prec_lloyd_mode(c, prec, d, kmax, &mode)) {
    p.W = 0;
    return rc;
  }
  if (int rc = round_build(c, X, n, d, b, strategy, seed, round0, max_iter, rel_tol, n_candidates,
                           cv, p.host.data(), tab_dev, tab_bytes, uprev, p, mode)) {
    p.W = 0;
    return rc;
  }
  if ((e = cudaMemsetAsync(uprev, 0, (size_t)b->W * sizeof(int32_t), c->stream)) ||
      (e = cudaMemcpyAsync(tab_dev, p.host.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->plan_round, &round0, sizeof(uint32_t), cudaMemcpyHostToDevice,
                           c->stream)) ||
      (e = cudaStreamSynchronize(c->stream))) {
    p.W = 0;
    return cuda_fail(c, e, "prepared-round tables");
  }
  return HPC_OK;
}

int hpc_round_enqueue(hpc_ctx *c) {
  if (!c) return HPC_ERR_ARG;
  if (!c->plan || c->plan->W < 1) return fail(c, HPC_ERR_ARG, "no prepared round");
  cudaSetDevice(c->device);
  return round_enqueue(c, *c->plan, c->plan_round, 0, nullptr, nullptr, 0);
}

}  // extern "C"
