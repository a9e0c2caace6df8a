/*
 * hpclust.h — C ABI of the GB300 (sm_103a) HPClust hot path.
 *
 * HPClust (arXiv 2311.04517) clusters very tall data by letting each worker
 * repeatedly draw a random sample S of size s from the data X, re-seed its
 * degenerate centroids with K-means++ on S, run K-means (Lloyd) on S from its
 * incumbent centroids, and keep the result if the sample objective improved
 * (Section 3; Algorithms 3-5).  This library runs those steps, and the
 * full-data objective of Eq. 1, as CUDA kernels on one GPU.
 *
 * Conventions shared by every call below
 *  - Arrays are row-major.  X is n x d float, S is s x d float, C is k x d
 *    float.  Unless a parameter says "host", every pointer is a DEVICE
 *    pointer owned by the caller; the library never frees or retains it.
 *    Float arrays must be 16-byte aligned; sizes are int64 (rows) and int32
 *    (dimensions, clusters).  Supported dimensions: 1 <= d <= 128.
 *  - Every call is asynchronous on the stream given to hpc_create /
 *    hpc_set_stream; outputs are valid once that stream has synchronised.
 *    Calls on one context must not run concurrently from several host
 *    threads (the context's scratch memory is shared).
 *  - Return value: HPC_OK (0) or a negative hpc_status for errors found on
 *    the host (bad arguments, allocation or launch failure).  Errors found
 *    on the device (non-finite input, a bounded wait that ran out) are
 *    recorded in the context's device status word and returned by
 *    hpc_sync_status().  hpc_last_error() describes the latest error.
 *  - Degenerate flags are one byte per centroid, 1 = degenerate (an empty
 *    cluster, Section 3).  Degenerate centroids take no part in any
 *    assignment; a NULL flag array means "all live" where it is an input.
 *  - Random draws come from Philox4x64-10 (Salmon et al., SC'11): draw j of
 *    stream (seed, worker, round, tag) is word j mod 4 of the block at
 *    counter (j div 4, round, tag, 0) under key (seed, worker).  Tag 0 gives
 *    the sample rows, tag 1 the K-means++ draws.  The same arguments give the
 *    same sample and the same seeding on every run.
 */
#ifndef HPCLUST_H
#define HPCLUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpc_ctx hpc_ctx;

typedef enum hpc_status {
  HPC_OK = 0,
  HPC_ERR_ARG = -1,            /* invalid argument (size, alignment, NULL) */
  HPC_ERR_NOMEM = -2,          /* device scratch allocation failed */
  HPC_ERR_CUDA = -3,           /* a CUDA runtime call or launch failed */
  HPC_ERR_TIMEOUT = -4,        /* a bounded device-side wait gave up */
  HPC_ERR_NONFINITE = -5,      /* NaN or infinity in the input rows */
  HPC_ERR_DEGENERATE_ALL = -6, /* no live centroid to assign to */
  HPC_ERR_UNSUPPORTED = -7     /* a valid request the library does not implement */
} hpc_status;

/* Precision of the nearest-centroid search.  Whatever the precision, every
 * search proves its winner against the error bound of its products or
 * settles the row exactly (FP32 direct form, then FP64 in the oracle's
 * operation order), so all return the labels of the double-precision
 * assignment and objectives equal within rounding: the precision changes
 * the speed, not the result. */
typedef enum hpc_precision {
  HPC_FP32 = 0, /* the context's choice (hpc_set_tensor_cores, hpc_set_objective_form):
                   FP32 CUDA-core, split-TF32, TF32 or split-BF16 products */
  HPC_BF16 = 1, /* split-BF16 tensor-core products (three BF16 MMAs per K step, FP32
                   accumulation) with rescoring of near ties; built for d = 64
                   (k <= 512) and d = 128 (k <= 256), HPC_ERR_UNSUPPORTED elsewhere */
  HPC_FP8 = 2   /* not built (HPC_ERR_UNSUPPORTED): FP8 e4m3 products leave an error
                   window that holds most rows of the method's own incumbents */
} hpc_precision;

typedef enum hpc_search {
  HPC_SEARCH_SIMT = 0,       /* FP32 expanded form on the CUDA cores */
  HPC_SEARCH_SPLIT_TF32 = 1, /* tensor cores, three TF32 products per K step (d in {16, 32}) */
  HPC_SEARCH_TF32 = 2,       /* tensor cores, one TF32 product (d in {16, 32, 64}: k <= 512;
                                d = 128: k <= 256) */
  HPC_SEARCH_SPLIT_BF16 = 3  /* tensor cores, three BF16 products per K step (d = 64: k <= 512;
                                d = 128: k <= 256); also the Lloyd iterations' search */
} hpc_search;

typedef enum hpc_strategy {
  HPC_COMPETITIVE = 0, /* Algorithm 3: each worker starts from its own incumbent */
  HPC_COOPERATIVE = 1, /* Algorithm 4: from the best incumbent of its group */
  HPC_HYBRID = 2       /* Algorithm 5: competitive while round < batch->n_competitive,
                          cooperative afterwards */
} hpc_strategy;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device` that launches on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle.  Returns HPC_ERR_ARG for a NULL ctx or a bad device. */
int hpc_create(hpc_ctx **ctx, int device, void *stream);

/* Frees the context and its scratch memory (synchronises its stream first).
 * NULL is accepted and ignored. */
int hpc_destroy(hpc_ctx *ctx);

/* Makes later calls on `ctx` launch on `stream` (a cudaStream_t). */
int hpc_set_stream(hpc_ctx *ctx, void *stream);

/* Synchronises the context's stream, then returns and clears the device
 * status word: HPC_OK, or the first device-side error since the last call
 * (HPC_ERR_TIMEOUT, HPC_ERR_NONFINITE, HPC_ERR_DEGENERATE_ALL). */
int hpc_sync_status(hpc_ctx *ctx);

/* Static description of the latest error on this context ("" if none). */
const char *hpc_last_error(hpc_ctx *ctx);

/* Number of kernels this context has launched so far. */
int64_t hpc_launch_count(hpc_ctx *ctx);

/* Pre-allocates at least `bytes` of device scratch so that later calls do
 * not allocate (useful before timing or stream capture). */
int hpc_reserve(hpc_ctx *ctx, int64_t bytes);

/* Chooses where hpc_objective runs its nearest-centroid search on the
 * tensor cores instead of the FP32 CUDA-core form: mode 0 never; 1 wherever
 * built (d in {16, 32}: split-TF32 products, three MMAs per K step, row
 * operand written to tensor memory; d in {64, 128}: TF32 products; k <= 128
 * for both); 2 (default) the form set for (d, k) by hpc_set_objective_form
 * or hpc_autotune_objective, else where it was measured faster on GB300:
 * d = 32 with k <= 128 (split TF32) and d in {64, 128} with k <= 128 (TF32).
 * For 128 < k <= 512 the TF32 form splits each row tile's 256 or 512
 * accumulator columns over four warpgroups; it is chosen only when set or
 * measured faster (it wins where few rows lie near a tie).  Every form
 * proves its winner against its products' error bound or settles the row
 * exactly, so all return the same labels and objectives within rounding;
 * they differ in speed only, and the speed depends on the data (rows near
 * a tie between two centroids take the exact path). */
int hpc_set_tensor_cores(hpc_ctx *ctx, int mode);

/* Sets the search form (hpc_search) hpc_objective uses for shape (d, k) in
 * mode 2; form -1 removes the setting.  Errors: HPC_ERR_ARG for a bad shape
 * or form, HPC_ERR_UNSUPPORTED if the form is not built for the shape. */
int hpc_set_objective_form(hpc_ctx *ctx, int32_t d, int32_t k, int32_t form);

/* The search form hpc_objective would run for (n, d, k) now, or
 * HPC_ERR_ARG for a bad shape. */
int hpc_objective_form(hpc_ctx *ctx, int64_t n, int32_t d, int32_t k);

/* Tile-schedule choice by measurement (the search form is the one choice
 * that changes the objective's speed several-fold): times every form built
 * for (d, k) on the caller's rows X (n x d; a prefix larger than L2, 129 MB,
 * gives representative times) and centroids C (k x d, flags as in
 * hpc_objective), reps timed calls each after one warm-up, with CUDA events
 * on the context's stream; keeps the fastest for (d, k) as
 * hpc_set_objective_form would (the built-in form when it is within 1% of
 * the fastest, so that timing noise does not move the choice).  *form_out
 * (nullable) receives it, ms_out (host float[4], nullable) the average
 * milliseconds per call of each form (indexed by hpc_search), -1 where not
 * built.  Synchronises the stream.  Errors: as
 * hpc_objective; a device error recorded during the sweep ends it and is
 * returned. */
int hpc_autotune_objective(hpc_ctx *ctx, const float *X, int64_t n, int32_t d, const float *C,
                           int32_t k, const uint8_t *degenerate, int32_t reps,
                           int32_t *form_out, float *ms_out);

/* The schedule hpc_lloyd would launch for one sample of s rows (s x d, k
 * centroids), for reporting and tests (the paper has no counterpart: this
 * is a launch configuration, not a step of the method).  out (host,
 * nout int32 entries, up to 5 written):
 *   [0] blocks of the persistent launch
 *   [1] 1 if each block sums its rows into k x d fixed-point sums in shared
 *       memory, 0 if it adds them straight into the global sums (k x d x 8
 *       bytes above what a block can hold)
 *   [2] 1 if each block keeps its rows in shared memory between the
 *       assignment and the accumulation
 *   [3] dynamic shared memory per block (bytes)
 *   [4] search form of the assignment (hpc_search)
 * Errors: HPC_ERR_ARG (sizes, NULL out), HPC_ERR_UNSUPPORTED (no kernel for
 * the shape). */
int hpc_lloyd_schedule(hpc_ctx *ctx, int64_t s, int32_t d, int32_t k, int32_t *out,
                       int32_t nout);

/* The CTA plan of a batched split-BF16 Lloyd launch (the paper has no
 * counterpart: the spread of Algorithm 3-5's workers over the GPU).  Host
 * only (no context, no device): what the launch's one-thread planner
 * computes before every launch of a round, from each worker's sample size
 * s[w], centroid count k[w] and updates in its previous run u[w] (host
 * arrays of W <= 128; negative u counts as 0, u above 1000 as 1000).  The
 * work of worker w is s k (u + 1).  Workers with fewer than 16 128-row
 * tiles go to the list, largest first, which keeps L = round(ctas x its
 * share of the work) CTAs (at least 1, at most its length, at most
 * ctas - 1 while other workers remain, all of them when none do).  The
 * other workers are dealt into max(1, min(their number, (ctas - L) / 16))
 * sets, largest first each to the set with the least work so far (lowest
 * index on ties); every set gets one CTA, then the remaining ctas - L go
 * one at a time to the set with the most work per CTA among those with
 * fewer CTAs than the tiles of their smallest sample; the sets take
 * contiguous CTA ranges from CTA 0 in set order.  A set runs its workers
 * one after another, each on all of its CTAs.
 * Output (host): cta_task[ctas] the first worker of each CTA's set (-2: no
 * set; such a CTA takes workers from the list), list[W] the workers CTAs
 * take one at a time as they become free, sets done or without one (its
 * length returned through *nlist), next[W] the worker a set runs after
 * worker w (-1 after its last, and for listed workers), nblocks[W] each
 * worker's CTAs (its set's; 1 for listed workers).
 * Errors: HPC_ERR_ARG (W outside 1..128, ctas < 1, a NULL array, s < 1 or
 * k < 1). */
int hpc_lloyd_cta_plan(int32_t W, const int64_t *s, const int32_t *k, const int32_t *u,
                       int32_t ctas, int32_t *cta_task, int32_t *list, int32_t *nlist,
                       int32_t *next, int32_t *nblocks);

/* Per-phase timing of rounds (the paper has no counterpart: measurement
 * only).  With timing on, every round enqueued on the context (hpc_round,
 * hpc_round_enqueue) records CUDA events on the context's stream around
 * each of its launches; a round enqueued while a stream is captured records
 * them as nodes of the graph, so each replay of that graph times itself
 * again.  hpc_phase_times waits for the latest timed round (the last one
 * enqueued, or the last replay of a graph recorded with timing on) and
 * writes the milliseconds it spent in each phase to ms_out (host, 3 floats:
 * sampling with base selection, K-means++, Lloyd with the incumbent rule).
 * Rounds of more than 31 launch chunks (3968 workers) are not timed.
 * Errors: HPC_ERR_ARG (bad flag, NULL ms_out, no timed round yet),
 * HPC_ERR_CUDA. */
int hpc_set_phase_timing(hpc_ctx *ctx, int32_t on);
int hpc_phase_times(hpc_ctx *ctx, float *ms_out);

/* Stage counters of the split-BF16 tensor-core search (the paper has no
 * counterpart: measurement only).  With counting on, every objective and
 * Lloyd assignment that runs that search adds to four device counters:
 * [0] rows assigned, [1] rows whose tensor-core top-2 margin fell inside
 * the error window (their two candidates were computed exactly), [2] rows
 * settled against every centroid (a third candidate could not be ruled
 * out), [3] rows settled in FP64.  hpc_search_stats synchronises the stream
 * and copies them to out (host, 4 int64); reset != 0 zeroes them.  A
 * prepared round keeps the setting it was prepared with.  Errors:
 * HPC_ERR_ARG, HPC_ERR_CUDA. */
int hpc_set_search_stats(hpc_ctx *ctx, int32_t on);
int hpc_search_stats(hpc_ctx *ctx, int64_t *out, int32_t reset);

/* ---- the hot path ------------------------------------------------------ */

/* Random sample of size s from X (Section 3: a worker starts every round by
 * drawing a random subset of s rows of the data; Algorithms 3-5, first step
 * of the worker loop).  Reading: with replacement; sample row i is X[floor(r_i * n / 2^64)]
 * where r_i is draw i of stream (seed, worker, round, tag 0).
 *   X        device, n x d float (input)
 *   S_out    device, s x d float (output)
 *   idx_out  device, s int64 (output, nullable): the drawn row indices
 * Errors: HPC_ERR_ARG if s < 0, d out of range, or s > 0 with n < 1. */
int hpc_draw_sample(hpc_ctx *ctx, const float *X, int64_t n, int32_t d,
                    uint64_t seed, uint32_t worker, uint32_t round, int64_t s,
                    float *S_out, int64_t *idx_out);

/* Greedy K-means++ seeding of the degenerate centroids (Section 3: empty
 * clusters are re-initialised with K-means++ on the current sample; Section
 * 6.5: each new centroid is the best of three candidates drawn by the D^2
 * rule).  Live centroids are left untouched; degenerate slots are filled in
 * index order.  If no centroid is live, the lowest slot first takes sample
 * row floor(r_0 * s / 2^64) (draw 0 of tag 1).  Each further slot draws
 * n_candidates rows with probability proportional to D(x)^2 (draws
 * 1 + t*n_candidates + l, t = slots seeded so far) and keeps the one with the
 * smallest potential sum_i min(D(x_i)^2, ||x_i - cand||^2).  D^2 is the
 * float squared distance accumulated in dimension order with one fused
 * multiply-add per dimension; the draw and the potentials use exact 64-bit
 * fixed-point sums of those values (grid 2^-F, F = 62 - bitlen(s) - e with
 * 2^(e-1) <= max D^2 < 2^e).  If every row already sits on a live centroid
 * the remaining slots stay degenerate.
 *   S                  device, s x d float (input)
 *   C_inout            device, k x d float (in/out)
 *   degenerate_inout   device, k bytes (in/out); NULL = all degenerate
 * Errors: HPC_ERR_ARG for s < 1, k < 1 or n_candidates < 1;
 * HPC_ERR_NONFINITE (device status) for non-finite rows. */
int hpc_kmeanspp(hpc_ctx *ctx, const float *S, int64_t s, int32_t d, int32_t k,
                 float *C_inout, uint8_t *degenerate_inout, int32_t n_candidates,
                 uint64_t seed, uint32_t worker, uint32_t round);

/* Lloyd's K-means on one sample (Algorithm 1, iterative part) with the stop
 * rule of Section 6.5: at most max_iter centroid updates, and stop at the
 * first assignment whose objective improved on the previous one by less
 * than rel_tol of it (or when the objective is zero).  Each assignment takes
 * every row to its nearest live centroid (Eq. 1; ties to the lowest index);
 * each update sets a centroid to the mean of its members, and a centroid
 * left without members becomes degenerate (keeps its value, excluded from
 * later assignments of this run).  The returned centroids are the ones last
 * assigned, so *f_out = f(C_out, S).
 *   S                 device, s x d float (input)
 *   C_inout           device, k x d float (in/out)
 *   degenerate_inout  device, k bytes (in/out, NULL = all live)
 *   labels_out        device, s int32 (output, nullable)
 *   f_out             device, 1 double (output): the sample objective
 *   iters_out         device, 1 int32 (output, nullable): updates performed
 * The assignment runs on the CUDA cores, or for d = 64 (k <= 512) and
 * d = 128 (k <= 256) on the tensor cores in split BF16 (HPC_BF16, or
 * hpc_set_tensor_cores mode 1, or mode 2 with k >= 48), where the centroid
 * sums are kept incrementally: each assignment after the first adds and
 * removes only the rows whose label changed, on the same exact fixed-point
 * grid.  Errors: HPC_ERR_ARG for s < 1, k < 1, max_iter outside
 * [0, 100000]; HPC_ERR_UNSUPPORTED for HPC_FP8, or HPC_BF16 on a shape it is
 * not built for; device status HPC_ERR_DEGENERATE_ALL if no centroid is
 * live, HPC_ERR_NONFINITE for non-finite rows. */
int hpc_lloyd(hpc_ctx *ctx, const float *S, int64_t s, int32_t d, int32_t k,
              float *C_inout, uint8_t *degenerate_inout, int32_t max_iter,
              double rel_tol, int32_t prec, int32_t *labels_out, double *f_out,
              int32_t *iters_out);

/* Full-data objective f(C, X) = sum_i min_j ||x_i - c_j||^2 (Eq. 1) over the
 * live centroids, accumulated in double precision, with the optional final
 * assignment Y (Section 3, last step; Algorithms 3-5, last line).  n = 0
 * gives 0.
 *   X           device, n x d float (input)
 *   C           device, k x d float (input)
 *   degenerate  device, k bytes (input, nullable = all live)
 *   f_out       device, 1 double (output)
 *   labels_out  device, n int32 (output, nullable)
 * prec HPC_BF16 runs the split-BF16 search (HPC_SEARCH_SPLIT_BF16) whatever
 * the context's choice.  Errors: HPC_ERR_ARG, HPC_ERR_UNSUPPORTED (prec);
 * device status HPC_ERR_DEGENERATE_ALL (n > 0 and no live centroid). */
int hpc_objective(hpc_ctx *ctx, const float *X, int64_t n, int32_t d,
                  const float *C, int32_t k, const uint8_t *degenerate,
                  int32_t prec, double *f_out, int32_t *labels_out);

/* Worker set of one HPClust run.  Host arrays describe the workers; device
 * arrays hold their state between rounds. */
typedef struct hpc_batch {
  int32_t W;            /* number of workers */
  const int64_t *s;     /* host [W]: sample size of each worker (>= 1) */
  const int32_t *k;     /* host [W]: clusters of each worker (>= 1) */
  const int32_t *group; /* host [W]: cooperative sharing group (nullable = one group) */
  const int64_t *C_off; /* host [W]: float offset of worker w's centroids in C */
  const int64_t *K_off; /* host [W]: byte offset of worker w's flags in degenerate */
  float *C;             /* device: centroid pool (incumbents C_w) */
  uint8_t *degenerate;  /* device: flag pool; all 1 before the first round */
  double *fhat;         /* device [W]: incumbent sample objective per point; +inf at start */
  double *f_new;        /* device [W] (nullable): this round's Lloyd objective */
  int32_t *iters;       /* device [W] (nullable): this round's Lloyd updates */
  uint8_t *accepted;    /* device [W] (nullable): 1 if the incumbent was replaced */
  int32_t n_competitive; /* HPC_HYBRID: rounds 0 .. n_competitive - 1 form the
                            competitive phase (Algorithm 5's N1); ignored otherwise */
  int32_t worker0;       /* global index of worker 0: worker w draws its sample and its
                            K-means++ candidates from stream (seed, worker0 + w), so a run
                            split over several batches (processes, GPUs) draws what one
                            batch of all workers would; 0 for a batch of all workers */
  uint64_t *t_done;      /* device [W] (nullable): per round, the device time (globaltimer
                            ns, as hpc_timestamp) at which worker w's run ended, after its
                            incumbent test: with f_new it gives Section 6.4's baseline
                            convergence time, the time until any worker first reaches a
                            given sample objective */
} hpc_batch;

/* One HPClust round for every worker of `batch` (one pass of the loop body
 * of Algorithm 3 or 4).  Worker w draws S_w (hpc_draw_sample with worker w),
 * takes as base its own incumbent (HPC_COMPETITIVE) or that of the worker
 * with the smallest fhat in its group and with its k (HPC_COOPERATIVE;
 * snapshot at the start of the round, lowest index on ties), re-seeds the
 * base's degenerate centroids (hpc_kmeanspp), runs hpc_lloyd, and replaces
 * its incumbent when f / s_w < fhat[w] (Algorithm 3's strict test, per
 * sample point because sample sizes may differ between workers).
 * Errors: as the calls it makes; HPC_ERR_ARG for a malformed batch. */
int hpc_round(hpc_ctx *ctx, const float *X, int64_t n, int32_t d,
              const hpc_batch *batch, int32_t strategy, uint64_t seed,
              uint32_t round, int32_t max_iter, double rel_tol,
              int32_t n_candidates, int32_t prec);

/* A round whose set-up is done once: hpc_round_prepare checks the batch,
 * reserves the round's scratch in memory of its own (later calls on the
 * context never overwrite it), writes the descriptor tables to the device and
 * sets a device round counter to round0 (it synchronises the stream).
 * hpc_round_enqueue then enqueues one round exactly as hpc_round would for
 * the counter's current value, and the round's last kernel advances the
 * counter: no host synchronisation, no allocation and no host-to-device copy,
 * so a stream capture can record it once and a CUDA graph can replay it
 * round after round (Algorithms 3-5 run the same round body every time).
 * HPC_HYBRID is resolved on the device from the counter.  The prepared round
 * reads X, the batch's device arrays and its host descriptors' sizes as they
 * were at preparation: prepare again after changing any of them.  One
 * prepared round per context; preparing again replaces it.
 * Errors: as hpc_round; hpc_round_enqueue returns HPC_ERR_ARG when nothing is
 * prepared. */
int hpc_round_prepare(hpc_ctx *ctx, const float *X, int64_t n, int32_t d,
                      const hpc_batch *batch, int32_t strategy, uint64_t seed,
                      uint32_t round0, int32_t max_iter, double rel_tol,
                      int32_t n_candidates, int32_t prec);
int hpc_round_enqueue(hpc_ctx *ctx);

/* Writes the device's time (the globaltimer register, nanoseconds) into
 * *dev_out (device, one uint64) once the work queued before it on the
 * context's stream has run: the origin against which hpc_batch.t_done is
 * read.  Errors: HPC_ERR_ARG, HPC_ERR_CUDA. */
int hpc_timestamp(hpc_ctx *ctx, uint64_t *dev_out);

/* ---- checkpoint ----------------------------------------------------------- */

/* The state an HPClust run resumes from is its workers' incumbents (C_w,
 * their degenerate flags, fhat_w) plus the next round index and the seed:
 * every random draw of round r is a function of (seed, worker, r), so a run
 * resumed from a checkpoint continues exactly as the uninterrupted run
 * would (Algorithms 3-5 keep no other state between rounds).
 *
 * hpc_batch_save writes that state into the HOST buffer host_buf (cap
 * bytes): a 64-byte header (magic "HPCBATCH", version 1, W, d, strategy,
 * next_round, n_competitive, seed, counts, FNV-1a checksum of the rest),
 * then per worker (s_w int64, k_w int32, group_w int32), the centroids of
 * every worker in worker order (k_w x d float each), their flags (k_w bytes
 * each) and fhat (W doubles); little-endian, no padding.  *bytes_out
 * receives the size; host_buf NULL only queries it.  It reads the device
 * arrays on the context's stream after the work queued before it, and
 * synchronises the stream.
 * hpc_batch_load checks a buffer written by hpc_batch_save against `batch`
 * (same W, d, s_w, k_w, group_w, and n_competitive for HPC_HYBRID) and its
 * checksum, writes C, degenerate and fhat of `batch`, and returns the
 * recorded next round, seed and strategy (each out-pointer nullable); it
 * synchronises the stream.  A prepared round reads the device round counter
 * it was prepared with: prepare again from the loaded round.
 * Errors: HPC_ERR_ARG for a malformed batch, a short buffer, a foreign or
 * corrupted checkpoint or one of another batch; HPC_ERR_CUDA on a copy
 * failure. */
int hpc_batch_save(hpc_ctx *ctx, const hpc_batch *batch, int32_t d, uint32_t next_round,
                   uint64_t seed, int32_t strategy, void *host_buf, int64_t cap,
                   int64_t *bytes_out);
int hpc_batch_load(hpc_ctx *ctx, const hpc_batch *batch, int32_t d, const void *host_buf,
                   int64_t bytes, uint32_t *next_round, uint64_t *seed, int32_t *strategy);

/* ---- allocation-free variant ------------------------------------------- */

/* The full-data objective of hpc_objective (CUDA-core search; same labels,
 * same objective) for callers that cannot allocate device memory when they
 * need it: code running while a stream is captured into a CUDA graph, loops
 * with a fixed memory budget, hosts that hand out device memory only through
 * their own pool.  The paper has no counterpart: this is a calling
 * convention, not a step of the method.  No context and no allocation: the
 * kernel's per-block partial sums live in a fixed array inside the library
 * (about 16 KB per device, kept until the process exits); the caller passes
 * inputs and outputs as for hpc_objective, plus status_out, a device int
 * that receives HPC_OK or the device-side error (HPC_ERR_NONFINITE,
 * HPC_ERR_DEGENERATE_ALL) once `stream` (a cudaStream_t) has run the call.
 * Every call on a device shares that array, so calls that may overlap on
 * the GPU race: serialise them.  A call made while `stream` is not being
 * captured looks the array's address up with the current device; a call
 * made during a stream capture reuses the address the latest uncaptured call
 * on that device found (HPC_ERR_ARG if there was none), so make one
 * uncaptured call first, with the same padded dimension (the next of 2, 4,
 * 8, 16, 32, 64, 128) and the same k class (k <= 32 or k > 32) as the
 * captured call: it also loads the kernel and sets its shared-memory limit.
 * Errors: HPC_ERR_ARG for bad sizes or unaligned pointers,
 * HPC_ERR_UNSUPPORTED if the centroid block does not fit in shared memory,
 * HPC_ERR_CUDA if a launch fails. */
int hpc_objective_noalloc(const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                          const uint8_t *degenerate, double *f_out, int32_t *labels_out,
                          int32_t *status_out, void *stream);

/* ---- learned cost model of the objective's search forms ------------------ */

/* The paper has no learned component (Sections 3-4).  This network serves
 * only the schedule choice of hpc_autotune_objective (which search form the
 * full-data objective of Eq. 1 runs); it never touches an assignment or an
 * objective value.  It is a perceptron with two hidden layers of
 * HPC_CM_HIDDEN ReLU units that maps HPC_CM_NFEAT inputs to a predicted
 * ln(nanoseconds per row) of one form:
 *   y(x) = b3 + w3 . relu(b2 + W2 relu(b1 + W1 x)),
 * trained on measured times with the mean squared error
 *   L = (1/N) sum_i (y(x_i) - t_i)^2
 * and full-batch Adam (Kingma and Ba 2015; beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-8).  Parameters are one float array of HPC_CM_NPARAM values:
 * W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3 (row-major, F = HPC_CM_NFEAT,
 * H = HPC_CM_HIDDEN).  Inputs per form (hpc_costmodel_features):
 *   [0] log2(d) / 7            [1] log2(k) / 9
 *   [2] padded columns / k - 1 (columns: the next of 32, 64, ..., 512)
 *   [3] centroid separation: log2(max ||c||^2 / min ||c_i - c_j||^2) over
 *       live centroids, clamped to [0, 40], / 40 (1 if two coincide, 0 with
 *       fewer than two live)
 *   [4..6] one-hot form (HPC_SEARCH_SIMT, _SPLIT_TF32, _TF32)
 *   [7] 1 if k > 128 (the wide tensor-core kernel), else 0. */
#define HPC_CM_NFEAT 8
#define HPC_CM_HIDDEN 32
#define HPC_CM_NPARAM 1377

/* Mean squared error of the network `params` on N samples (feats N x
 * HPC_CM_NFEAT, targets N) and its gradient: *loss_out (device float) and
 * grad_out (device, HPC_CM_NPARAM floats).  FP32; the per-sample gradients
 * are summed in a fixed order, so repeated calls give identical results.
 * Errors: HPC_ERR_ARG (N < 1 or N > 2^20, NULL pointer), HPC_ERR_NOMEM,
 * HPC_ERR_CUDA. */
int hpc_costmodel_loss_grad(hpc_ctx *ctx, const float *params, const float *feats,
                            const float *targets, int32_t N, float *loss_out, float *grad_out);

/* `steps` full-batch Adam steps on params, with the first and second
 * moments m and v (device, HPC_CM_NPARAM floats each, zero for a fresh
 * start) carried by the caller; step s uses the bias corrections of step
 * number step0 + s + 1, so training resumes exactly where an earlier call
 * stopped.  loss_out (device, `steps` floats, nullable) receives the loss at
 * the parameters each step started from.  Two launches per step.  Errors as
 * hpc_costmodel_loss_grad, and HPC_ERR_ARG for steps < 0, step0 < 0 or a
 * learning rate that is not positive and finite. */
int hpc_costmodel_train(hpc_ctx *ctx, float *params, float *m, float *v, const float *feats,
                        const float *targets, int32_t N, int32_t steps, int32_t step0, float lr,
                        float *loss_out);

/* Predictions y for N input rows (device feats N x HPC_CM_NFEAT, out N). */
int hpc_costmodel_predict(hpc_ctx *ctx, const float *params, const float *feats, int32_t N,
                          float *out);

/* The network inputs of each of the three search forms for centroids C
 * (device, k x d; degenerate nullable = all live): feats_out (HOST,
 * 3 x HPC_CM_NFEAT floats, row f = form f) and supported_out (HOST, 3 ints,
 * nullable: 1 where the form is built for (d, k)).  Copies C and the flags
 * to the host and synchronises the stream.  Errors: HPC_ERR_ARG, HPC_ERR_CUDA. */
int hpc_costmodel_features(hpc_ctx *ctx, const float *C, const uint8_t *degenerate, int32_t d,
                           int32_t k, float *feats_out, int32_t *supported_out);

/* The guided search's plan, on the host (no GPU needed): the built forms
 * (supported[f] != 0) ranked by predicted ln time pred[f] (host float[3];
 * ties to the lower form index) into order_out (host int[3]), and timed_out
 * (host int[3]) = 1 for the ranked forms that are timed: the best-ranked one
 * and each other one whose predicted time is within a factor (1 + margin) of
 * the best-ranked one's.  Returns the number of built forms (entries of
 * order_out past it are -1), or HPC_ERR_ARG for NULL arrays, a negative or
 * NaN margin, or a non-finite prediction of a built form. */
int hpc_costmodel_plan(const float *pred, const int32_t *supported, float margin,
                       int32_t *order_out, int32_t *timed_out);

/* hpc_autotune_objective guided by the network `params` (device): the forms
 * built for (d, k) are ranked by predicted time; the best-ranked one is
 * timed, and each other one only if its predicted time is within a factor
 * (1 + margin) of the best-ranked one's; HPC_SEARCH_SPLIT_BF16, which the
 * network's inputs do not describe, is timed whenever it is built.  The
 * fastest timed form is kept as hpc_autotune_objective would keep it.
 * ms_out (host float[4], nullable) gets the time per call of each timed
 * form, -1 for the others;
 * timed_out (host, nullable) the number of forms timed.  margin >= 0; a
 * very large margin times every form (the unguided search). */
int hpc_autotune_objective_guided(hpc_ctx *ctx, const float *X, int64_t n, int32_t d,
                                  const float *C, int32_t k, const uint8_t *degenerate,
                                  int32_t reps, const float *params, float margin,
                                  int32_t *form_out, float *ms_out, int32_t *timed_out);

/* ---- diagnostics -------------------------------------------------------- */

/* Throughput probes (the paper has no counterpart): the rates against which
 * the CUDA-core kernels' rooflines are stated.  Kinds: FP32 FMA (fma.rn.f32,
 * FMA/s), packed FP32 FMA (fma.rn.f32x2, FMA/s counting both lanes), FP64
 * FMA (FMA/s), FP32 min (ops/s; the top-2 search's compare pipe), L2 read
 * (bytes/s, a 64 MiB buffer read 40 times) and HBM read (bytes/s, a 4 GiB
 * buffer read once).  Runs on `device` and `stream` (a cudaStream_t; NULL =
 * the legacy default stream): one warm-up launch, then three launches timed
 * with CUDA events; *rate_out receives the rate, *ms_out (nullable) the time
 * of one launch.  Allocates and frees its buffers; synchronises the stream.
 * Errors: HPC_ERR_ARG (kind, device), HPC_ERR_NOMEM, HPC_ERR_CUDA. */
typedef enum hpc_probe {
  HPC_PROBE_FFMA = 0,
  HPC_PROBE_FFMA2 = 1,
  HPC_PROBE_DFMA = 2,
  HPC_PROBE_FMIN = 3,
  HPC_PROBE_L2_READ = 4,
  HPC_PROBE_HBM_READ = 5
} hpc_probe;
int hpc_peak_probe(int32_t kind, int32_t device, void *stream, double *rate_out, double *ms_out);

/* Failure-detection self-test (the paper has no counterpart).  Launches a
 * two-block cooperative kernel in which one block never reaches the grid
 * barrier; the other block's bounded wait gives up after limit_ns
 * nanoseconds (1e3 .. 1e9) and records HPC_ERR_TIMEOUT in the device status
 * word, which the next hpc_sync_status() returns.  No fault, no hang: this
 * is how every device-side wait in the library ends when a peer block never
 * arrives (the library's own waits give up after 4 s). */
int hpc_selftest_wait_timeout(hpc_ctx *ctx, int64_t limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* HPCLUST_H */
