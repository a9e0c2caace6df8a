// Host-side launch descriptors of the HPClust kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct hpc_gridbar;

struct hpc_launch {
  cudaStream_t stream;
  int num_sms;
  int smem_optin;  // max dynamic shared memory per block
};

struct LloydArgsHost {
  const float *S;
  int64_t s;
  int d, k;
  float *C;
  uint8_t *deg;
  int max_iter;
  double tol;
  int32_t *labels;
  double *f_out;
  int32_t *iters_out;
  hpc_gridbar *bar;
  int *status;
  unsigned *gmaxabs;
  unsigned long long *gsum;
  unsigned *gcount;
  double *gpart;
  int64_t grid_cap;  // upper bound on blocks (size of gpart / 2)
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
};

struct KppArgsHost {
  const float *S;
  int64_t s;
  int d, k;
  float *C;
  uint8_t *deg;
  int L;
  uint64_t seed;
  uint32_t worker, round;
  hpc_gridbar *bar;
  int *status;
  float *w;
  float *dc;
  unsigned long long *chunkQ;
  long long *cand;
  unsigned long long *phi;
  unsigned *mx;
  int64_t grid_cap;
};

int hpc_lloyd_launch(const hpc_launch &L, const LloydArgsHost &h);
int hpc_objective_launch(const hpc_launch &L, const ObjArgsHost &h);
bool hpc_tc_objective_supported(int d, int k, int64_t n);
int hpc_tc_objective_launch(const hpc_launch &L, const ObjArgsHost &h);
int hpc_kmeanspp_launch(const hpc_launch &L, const KppArgsHost &h);
int hpc_sample_launch(const hpc_launch &L, const float *X, int64_t n, int d, uint64_t seed,
                      uint32_t worker, uint32_t round, int64_t s, float *S, int64_t *idx);

// Blocks the cooperative kernels may use at most (upper bound for scratch
// sizing): resident blocks per SM times SMs.
int64_t hpc_grid_bound(const hpc_launch &L);
