// Host-side launch descriptors of the HPClust kernels (internal).
//
// The persistent kernels (Lloyd, K-means++) take a batch of independent
// problems ("tasks", one per worker): every task gets its own contiguous
// group of blocks and its own bounded group barrier, so workers with
// different sample sizes and cluster counts iterate independently inside
// one cooperative launch.  A batch of one task is passed by value; larger
// batches live in device memory together with a block -> task map.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct hpc_gridbar;

// Largest batch of independent problems one launch takes.
#define HPC_MAX_TASKS 4096
// batched seeding launches of up to this many workers are re-split on the
// device over the workers with a centroid to seed (one more launch)
#define HPC_KPP_SPLIT_MAX 128

struct hpc_launch {
  cudaStream_t stream;
  int num_sms;
  int smem_optin;  // max dynamic shared memory per block
};

// ---- Lloyd (one task = one sample) ----
struct hpc_lloyd_task {
  const float *S;
  int64_t s;
  int k;
  int block0, nblocks;  // filled by the launcher
  float *C;
  uint8_t *deg;         // never null
  int32_t *labels;      // nullable
  double *f_out;
  int32_t *iters_out;   // nullable
  hpc_gridbar *bar;     // zero at launch
  unsigned *gmaxabs;    // zero at launch
  unsigned long long *gsum;  // 3 * k * d
  unsigned *gcount;          // 3 * k
  unsigned long long *gobj;  // 3 rotating fixed-point sample objectives, zero at launch
  // tensor-core Lloyd only: each row's label of the previous assignment (s;
  // the caller's labels array when it gives one) and the exact centroid
  // block read by its exact stages (hpc_tcl_gcent_bytes(d, k) bytes)
  int32_t *plab;
  float *gcent;
  // incumbent rule at the end of the run (rounds only; fhat null otherwise)
  double *fhat;              // this worker's incumbent objective per point
  float *C_inc;              // its incumbent centroids (k x d) in the pool
  uint8_t *deg_inc;          // and their flags
  double *f_new;             // nullable reports
  int32_t *iters_rep;
  uint8_t *accepted;
  unsigned long long *t_done;  // nullable: the time (globaltimer ns) the run ended
  // nullable: the worker's updates in its latest run (a buffer of the
  // caller's that keeps its value from round to round), written at the end
  // of a run and read by the split-BF16 Lloyd's plan of the next round
  int32_t *uprev;
};
// Lloyd zeroes gsum / gcount itself; bar and gmaxabs must be zero at launch.

struct LloydLaunch {
  int W;
  hpc_lloyd_task *tasks;       // host array [W]; block0 / nblocks written by the plan
  int *block_task_host;        // host [grid] (W > 1), written by the plan; the
                               // tensor-core plan also uses [max_blocks, 2 max_blocks)
  const hpc_lloyd_task *tasks_dev;  // device copy of tasks (W > 1), uploaded by the caller
  const int *block_task_dev;        // device copy of block_task_host (W > 1)
  int d, kmax;
  int max_iter;
  double tol;
  int *status;
  int64_t max_blocks;          // blocks the caller's scratch allows in total
  int64_t task_blocks;         // most blocks one task may use
  // written by the plan
  int64_t grid;
  size_t smem;
  int smem_sums;
  int xstage;
  // nullable: a prepared round's counter, advanced once the run is done
  uint32_t *round_advance;
  // search: 0 CUDA cores only, 1 tensor cores wherever built, 2 where
  // measured faster (the plan writes the one chosen into `form`)
  int tc_mode;
  int form;  // written by the plan: hpc_search (0 CUDA cores, 3 split BF16)
  // nullable: counters of the tensor-core search (rows, rows near a tie,
  // rows settled against every centroid, rows settled in FP64)
  unsigned long long *stats;
  // nullable: rows the tensor-core Lloyd settles after each pass (queue_cap
  // per CTA, queue_ctas CTAs at most)
  int64_t *queue;
  int64_t queue_cap;
  int64_t queue_ctas;
  // nullable, zero at launch: the counter from which the tensor-core Lloyd's
  // CTAs take the tasks left to them (W > 1); nfollow written by the plan
  unsigned *pop;
  int nfollow;
};

// ---- K-means++ (one task = one sample) ----
struct hpc_kpp_task {
  const float *S;
  int64_t s;
  int k;
  int block0, nblocks;
  uint32_t worker;
  float *C;
  uint8_t *deg;  // never null
  hpc_gridbar *bar;           // zero at launch
  unsigned *mx;               // 2 words, zero at launch
  unsigned long long *phi;    // 2 * L, zero at launch
  float *w;                   // s
  float *dc;                  // L * s
  unsigned long long *chunkQ; // blocks of the task
  long long *cand;            // L
};

struct KppLaunch {
  int W;
  hpc_kpp_task *tasks;         // host [W]; block0 / nblocks written by the plan
  int *block_task_host;        // host [grid] (W > 1)
  const hpc_kpp_task *tasks_dev;
  const int *block_task_dev;
  int d, kmax, L;
  uint64_t seed;
  uint32_t round;
  const uint32_t *round_dev;  // nullable: read the round from the device instead
  int *status;
  int64_t max_blocks;
  int64_t chunk_cap;  // chunkQ entries reserved per task (1 per block)
  // written by the plan
  int64_t grid;
  size_t smem;
};

struct ObjArgsHost {
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
  int64_t max_blocks;
  // optional: near-tie rows deferred by the split-TF32 search (queue_cap
  // rows for each of queue_ctas blocks)
  int64_t *queue;
  int64_t queue_cap;
  int64_t queue_ctas;
  // optional: global scratch for the exact centroid block of the wide
  // (k > 128) tensor-core search, hpc_tc_wide_scratch_bytes(d, k) bytes
  unsigned char *cent_scratch;
  int64_t cent_scratch_bytes;
  // nullable: counters of the split-BF16 search (as LloydLaunch::stats)
  unsigned long long *stats;
};

// ---- sampling (one task = one worker's sample) ----
struct hpc_sample_task {
  float *S;
  int64_t *idx;
  int64_t s;
  uint32_t worker;
};

// ---- round bookkeeping (Algorithms 3-5) ----
struct hpc_round_worker {
  int64_t s;
  int64_t C_off, K_off;
  int k, group;
  float *Cn;    // base, then Lloyd's result
  uint8_t *dn;
  double *fw;   // Lloyd objective (NaN until written)
  int32_t *itw;
};

// Base selection, run by extra blocks of the batched sampling launch.
struct hpc_base_args {
  const hpc_round_worker *wk;  // device [W]; null: no base selection
  int W;
  int strategy;
  int32_t n_competitive;
  const uint32_t *round_dev;   // nullable
  uint32_t round;
  const double *fhat;
  const float *Cpool;
  const uint8_t *Kpool;
  int d;
  double *f_new;               // nullable reports, reset for the round
  int32_t *iters;
  uint8_t *accepted;
};

// Plan: chooses the kernel variant and the grid, splits the blocks over the
// tasks (tasks[w].block0 / nblocks, block_task_host).  Run: one cooperative
// launch; for W > 1 the caller has copied tasks and block_task_host to
// tasks_dev / block_task_dev on the same stream before it.
int hpc_lloyd_plan(const hpc_launch &L, LloydLaunch &h);
int hpc_lloyd_run(const hpc_launch &L, const LloydLaunch &h);
int hpc_kmeanspp_plan(const hpc_launch &L, KppLaunch &h);
int hpc_kmeanspp_run(const hpc_launch &L, const KppLaunch &h);
int hpc_objective_launch(const hpc_launch &L, const ObjArgsHost &h);
// TF32 tensor-core search for 128 < k <= 512 (d in {16, 32, 64}) and
// 128 < k <= 256 (d = 128); hpc_tc_objective_launch dispatches to it.
bool hpc_tc_wide_supported(int d, int k, int64_t n);
int hpc_tc_wide_launch(const hpc_launch &L, const ObjArgsHost &h);
size_t hpc_tc_wide_scratch_bytes(int d, int k);
bool hpc_tc_objective_supported(int d, int k, int64_t n);
int hpc_tc_objective_launch(const hpc_launch &L, const ObjArgsHost &h);
// split-TF32 tensor-core search for rows of 16 or 32 floats
bool hpc_tcs_objective_supported(int d, int k, int64_t n);
int hpc_tcs_objective_launch(const hpc_launch &L, const ObjArgsHost &h);
int hpc_sample_launch(const hpc_launch &L, const float *X, int64_t n, int d, uint64_t seed,
                      uint32_t worker, uint32_t round, int64_t s, float *S, int64_t *idx);
// W samples at once; tasks_dev is a device array [W], smax the largest s;
// the round is *round_dev when that is not null.
int hpc_sample_batch_launch(const hpc_launch &L, const float *X, int64_t n, int d, uint64_t seed,
                            uint32_t round, const uint32_t *round_dev, int W,
                            const hpc_sample_task *tasks_dev, int64_t smax,
                            const hpc_base_args &base);

// Split-BF16 tensor-core Lloyd (d = 64: k <= 512; d = 128: k <= 256).
bool hpc_tcl_supported(int d, int kmax);
size_t hpc_tcl_gcent_bytes(int d, int k);
int hpc_tcl_plan(const hpc_launch &L, LloydLaunch &h);
int hpc_tcl_cta_plan(int W, const int64_t *s, const int32_t *k, const int32_t *u, int64_t ctas,
                     int32_t *cta_task, int32_t *list, int32_t *nlist, int32_t *next,
                     int32_t *nblocks);
int hpc_tcl_run(const hpc_launch &L, const LloydLaunch &h);
// Split-BF16 tensor-core full-data objective (same shapes); needs
// h.cent_scratch of hpc_tcl_gcent_bytes(d, k) + 256 bytes.
int hpc_tcb_objective_launch(const hpc_launch &L, const ObjArgsHost &h);

// Blocks the cooperative kernels may use at most (upper bound for scratch
// sizing): resident blocks per SM times SMs.
int64_t hpc_grid_bound(const hpc_launch &L);

// Splits `total` co-resident blocks over W tasks in proportion to their work
// (rows when work is null): each task gets at least one block and at most
// one per rows_per_block of its rows.
void hpc_split_blocks(int W, const int64_t *rows, const int64_t *work, int64_t rows_per_block,
                      int64_t total, int *block0, int *nblocks);
