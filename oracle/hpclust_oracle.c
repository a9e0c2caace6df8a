/*
 * HPClust CPU oracle — plain, slow, obviously-correct reference.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file; the GPU library never links, includes
 * or calls it, and it shares no code, header, table or constant generator with
 * the CUDA path.  It is written from the paper "HPClust: hybrid parallel
 * approaches for minimum sum-of-squares clustering of infinitely tall data"
 * (arXiv 2311.04517) and from the published Philox definition.
 *
 * Precision: every distance, objective and centroid mean is computed in
 * double precision from the float inputs, except the two places where a
 * floating-point value decides an integer that the GPU must reproduce
 * exactly (the K-means++ D^2 draw and the greedy-candidate choice).  Those
 * take the decision in the kernel's precision: float squared distances
 * accumulated in dimension order with one fused multiply-add per dimension,
 * and 64-bit fixed-point sums of those weights (see orc_quant below).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC.  Contraction is
 * off so that x86 and Arm hosts round identically.
 *
 * OpenMP is used over rows only, for the per-row distance loops.  Every sum
 * that ends in a reported value is taken sequentially in row order.
 *
 * Parity pins (tests/test_oracle_pins.py): Philox against numpy's Philox,
 * brute-force optimal partitions for n<=12, k<=3, the k=1 closed form,
 * monotone objective, centroid = mean of members, the 1-D dynamic-programming
 * optimum, chi-square frequencies of the D^2 draw, the greedy candidate rule,
 * the sum-of-squares decomposition identity and composed round traces.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes (same numeric meaning as the GPU library, defined here
 * independently). */
#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOMEM (-2)
#define ORC_ERR_DEGENERATE_ALL (-6)

/* Philox stream tags: which draw family a counter belongs to. */
#define ORC_TAG_SAMPLE 0u  /* sample row indices (§3: random sample of size s) */
#define ORC_TAG_SEED 1u    /* K-means++ draws (§3, §6.5) */

#define ORC_STRAT_COMPETITIVE 0 /* Algorithm 3 */
#define ORC_STRAT_COOPERATIVE 1 /* Algorithm 4 */
#define ORC_STRAT_HYBRID 2      /* Algorithm 5: competitive phase, then cooperative */

typedef unsigned __int128 orc_u128;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  The paper asks for parallel, independent random
 * streams per worker (§5.3, parallel random number generation); a
 * counter-based generator gives every (seed, worker, round, draw) its own
 * number without shared state.
 *
 * One round maps (x0,x1,x2,x3) with key (k0,k1) to
 *   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
 * and the key is bumped by the Weyl constants between rounds. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    orc_u128 p0 = (orc_u128)M0 * x0;
    orc_u128 p1 = (orc_u128)M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* Draw j of stream (seed, worker, round, tag): word j mod 4 of
 * Philox4x64-10 at counter (j div 4, round, tag, 0) under key (seed, worker). */
uint64_t orc_draw(uint64_t seed, uint32_t worker, uint32_t round, uint32_t tag,
                  uint64_t j) {
  uint64_t ctr[4] = {j >> 2, (uint64_t)round, (uint64_t)tag, 0};
  uint64_t key[2] = {seed, (uint64_t)worker};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[j & 3u];
}

/* floor(r * m / 2^64): a 64-bit uniform word mapped onto {0, ..., m-1}. */
static uint64_t orc_scale_word(uint64_t r, uint64_t m) {
  return (uint64_t)(((orc_u128)r * (orc_u128)m) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Sampling (§3; Algorithms 3-5, first line of the worker loop): S_w is a
 * random sample of size s drawn from X.  Reading: with replacement, row i of
 * the sample is X[floor(r_i * n / 2^64)], r_i = draw i of the SAMPLE stream. */
int orc_draw_sample(const float *X, int64_t n, int32_t d, uint64_t seed,
                    uint32_t worker, uint32_t round, int64_t s, float *S,
                    int64_t *idx) {
  if (d < 1 || s < 0 || (s > 0 && n < 1)) return ORC_ERR_ARG;
  for (int64_t i = 0; i < s; ++i) {
    uint64_t r = orc_draw(seed, worker, round, ORC_TAG_SAMPLE, (uint64_t)i);
    int64_t row = (int64_t)orc_scale_word(r, (uint64_t)n);
    memcpy(S + i * (int64_t)d, X + row * (int64_t)d, sizeof(float) * (size_t)d);
    if (idx) idx[i] = row;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 distances.  ||x - c||^2 in double precision, direct form. */
static double orc_dist64(const float *x, const float *c, int32_t d) {
  double acc = 0.0;
  for (int32_t t = 0; t < d; ++t) {
    double diff = (double)x[t] - (double)c[t];
    acc += diff * diff;
  }
  return acc;
}

/* The kernel-precision squared distance used where the GPU must reproduce an
 * integer decision bit for bit (K-means++): float difference, then one fused
 * multiply-add per dimension, in dimension order. */
float orc_dist32(const float *x, const float *c, int32_t d) {
  float acc = 0.0f;
  for (int32_t t = 0; t < d; ++t) {
    float diff = x[t] - c[t];
    acc = fmaf(diff, diff, acc);
  }
  return acc;
}

/* Nearest live centroid of every row (Eq. 1 inner min; Algorithm 1 "assign
 * each x to the nearest centroid").  Ties go to the lowest index; centroids
 * flagged degenerate take no part.  Writes the label, the nearest distance d1
 * and the second-nearest distance d2 (+inf with one live centroid) per row,
 * and returns f = sum of d1 in row order (NaN when no centroid is live).
 * Rows are processed in chunks so the per-row distances of a chunk can be
 * computed in parallel and then summed sequentially. */
double orc_assign(const float *S, int64_t s, int32_t d, const float *C,
                  int32_t k, const uint8_t *degenerate, int32_t *labels,
                  double *d1_out, double *d2_out) {
  int any_live = 0;
  for (int32_t j = 0; j < k; ++j)
    if (!degenerate || !degenerate[j]) any_live = 1;
  if (!any_live) {
    for (int64_t i = 0; i < s; ++i) {
      if (labels) labels[i] = -1;
      if (d1_out) d1_out[i] = NAN;
      if (d2_out) d2_out[i] = NAN;
    }
    return NAN;
  }
  const int64_t chunk = 1 << 20;
  double *d1 = (double *)malloc(sizeof(double) * (size_t)(s < chunk ? (s > 0 ? s : 1) : chunk));
  double f = 0.0;
  for (int64_t base = 0; base < s; base += chunk) {
    int64_t m = s - base < chunk ? s - base : chunk;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < m; ++ii) {
      int64_t i = base + ii;
      const float *x = S + i * (int64_t)d;
      double best = INFINITY, second = INFINITY;
      int32_t bj = -1;
      for (int32_t j = 0; j < k; ++j) {
        if (degenerate && degenerate[j]) continue;
        double v = orc_dist64(x, C + (int64_t)j * d, d);
        if (v < best) {
          second = best;
          best = v;
          bj = j;
        } else if (v < second) {
          second = v;
        }
      }
      d1[ii] = best;
      if (labels) labels[i] = bj;
      if (d1_out) d1_out[i] = best;
      if (d2_out) d2_out[i] = second;
    }
    for (int64_t ii = 0; ii < m; ++ii) f += d1[ii];
  }
  free(d1);
  return f;
}

/* Centroid update (Algorithm 1 "update each c_i to the mean of the points
 * assigned to c_i").  Sums in double, the mean rounded once to float.  A
 * centroid with no members is flagged degenerate and keeps its old value
 * (§3: degenerate clusters are re-initialised by K-means++ later). */
int orc_update(const float *S, int64_t s, int32_t d, const int32_t *labels,
               int32_t k, float *C, uint8_t *degenerate) {
  double *sums = (double *)calloc((size_t)k * (size_t)d, sizeof(double));
  int64_t *counts = (int64_t *)calloc((size_t)k, sizeof(int64_t));
  if (!sums || !counts) {
    free(sums);
    free(counts);
    return ORC_ERR_NOMEM;
  }
  for (int64_t i = 0; i < s; ++i) {
    int32_t j = labels[i];
    if (j < 0) continue;
    counts[j] += 1;
    for (int32_t t = 0; t < d; ++t)
      sums[(int64_t)j * d + t] += (double)S[i * (int64_t)d + t];
  }
  for (int32_t j = 0; j < k; ++j) {
    if (counts[j] == 0) {
      degenerate[j] = 1;
      continue;
    }
    for (int32_t t = 0; t < d; ++t)
      C[(int64_t)j * d + t] = (float)(sums[(int64_t)j * d + t] / (double)counts[j]);
  }
  free(sums);
  free(counts);
  return ORC_OK;
}

/* Lloyd's K-means (Algorithm 1's iterative part) with the stop rule of §6.5:
 * stop after max_iter updates, or when the improvement between two
 * consecutive objectives is below rel_tol relative to the previous one.
 * A zero objective also stops (Algorithm 1: the centroids can no longer
 * change).  The returned centroids are the ones last assigned, so *f_out is
 * exactly f(C_out, S) and labels are their nearest-centroid labels.
 * *iters_out counts the updates performed.  f_trace (nullable, max_iter+1
 * entries) receives the objective of every assignment. */
int orc_lloyd(const float *S, int64_t s, int32_t d, int32_t k, float *C,
              uint8_t *degenerate, int32_t max_iter, double rel_tol,
              int32_t *labels, double *f_out, int32_t *iters_out,
              double *f_trace) {
  if (s < 1 || d < 1 || k < 1 || max_iter < 0) return ORC_ERR_ARG;
  int any_live = 0;
  for (int32_t j = 0; j < k; ++j)
    if (!degenerate[j]) any_live = 1;
  if (!any_live) return ORC_ERR_DEGENERATE_ALL;
  int32_t *lab = labels ? labels : (int32_t *)malloc(sizeof(int32_t) * (size_t)s);
  double f = 0.0, f_prev = 0.0;
  int32_t it = 0;
  for (;; ++it) {
    f = orc_assign(S, s, d, C, k, degenerate, lab, NULL, NULL);
    if (f_trace) f_trace[it] = f;
    if (it > 0 && (f_prev == 0.0 || (f_prev - f) < rel_tol * f_prev)) break;
    if (it == max_iter) break;
    int rc = orc_update(S, s, d, lab, k, C, degenerate);
    if (rc) {
      if (!labels) free(lab);
      return rc;
    }
    f_prev = f;
  }
  if (f_out) *f_out = f;
  if (iters_out) *iters_out = it;
  if (!labels) free(lab);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* K-means++ D^2 seeding (§3 and §6.5: each new centroid is the best of three
 * candidates drawn with probability proportional to D(x)^2).
 *
 * Reading of the draw: the weight D(x)^2 of row i is w_i (a float, see
 * orc_dist32).  With M = max w_i, e = the exponent with 2^(e-1) <= M < 2^e
 * and B = the bit length of s, the weights are put on the fixed-point grid
 * 2^-F, F = 62 - B - e: q_i = floor(w_i * 2^F) < 2^(62-B), so Q = sum q_i
 * < 2^62 is exact.  A 64-bit word r selects target t = floor(r*Q/2^64) and
 * the row is the first i whose running sum q_0 + ... + q_i exceeds t, so
 * row i is drawn with probability q_i / Q. */
static int orc_bit_length(int64_t s) {
  int b = 0;
  while (b < 63 && (s >> b) != 0) ++b;
  return b;
}

int orc_fixed_scale(float M, int64_t s) {
  int e;
  frexpf(M, &e);
  return 62 - orc_bit_length(s) - e;
}

int64_t orc_quant(float w, int F) { return (int64_t)ldexp((double)w, F); }

/* Index drawn by word r from weights w[0..s) (returns -1 if all are zero). */
int64_t orc_d2_pick(const float *w, int64_t s, uint64_t r) {
  float M = 0.0f;
  for (int64_t i = 0; i < s; ++i)
    if (w[i] > M) M = w[i];
  if (!(M > 0.0f)) return -1;
  int F = orc_fixed_scale(M, s);
  uint64_t Q = 0;
  for (int64_t i = 0; i < s; ++i) Q += (uint64_t)orc_quant(w[i], F);
  uint64_t target = orc_scale_word(r, Q);
  uint64_t run = 0;
  for (int64_t i = 0; i < s; ++i) {
    run += (uint64_t)orc_quant(w[i], F);
    if (run > target) return i;
  }
  return -1; /* not reached: target < Q */
}

/* Seeds every centroid flagged degenerate, in index order, leaving live
 * centroids untouched (§3: degenerate clusters are re-initialised with
 * K-means++ on the current sample; Algorithm 3's inner loop).
 *
 * If no centroid is live, the lowest degenerate slot takes the row
 * floor(r_0 * s / 2^64) (draw 0 of the SEED stream): the uniform first pick.
 * Each further slot draws L candidate rows with the D^2 rule (draws
 * 1 + t*L + l, t = number of slots already seeded this way, l < L), scores
 * each by its potential phi = sum_i q(min(w_i, D(x_i, cand)^2)) on the same
 * fixed-point grid, keeps the smallest (first drawn on ties), and lowers the
 * weights to the new nearest distance.  If every weight is zero (every row
 * sits on a live centroid) the remaining slots stay degenerate.
 *
 * cand_out / phi_out (nullable, k*L entries each) record, per slot j, the
 * drawn candidates and their potentials (-1 where the slot was not seeded by
 * the D^2 rule). */
int orc_kmeanspp(const float *S, int64_t s, int32_t d, int32_t k, float *C,
                 uint8_t *degenerate, int32_t L, uint64_t seed, uint32_t worker,
                 uint32_t round, int64_t *cand_out, int64_t *phi_out) {
  if (s < 1 || d < 1 || k < 1 || L < 1) return ORC_ERR_ARG;
  if (cand_out)
    for (int64_t i = 0; i < (int64_t)k * L; ++i) cand_out[i] = -1;
  if (phi_out)
    for (int64_t i = 0; i < (int64_t)k * L; ++i) phi_out[i] = -1;
  float *w = (float *)malloc(sizeof(float) * (size_t)s);
  float *dc = (float *)malloc(sizeof(float) * (size_t)s * (size_t)L);
  int64_t *cand = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
  if (!w || !dc || !cand) {
    free(w);
    free(dc);
    free(cand);
    return ORC_ERR_NOMEM;
  }
  int any_live = 0;
  for (int32_t j = 0; j < k; ++j)
    if (!degenerate[j]) any_live = 1;
  if (!any_live) {
    uint64_t r = orc_draw(seed, worker, round, ORC_TAG_SEED, 0);
    int64_t i0 = (int64_t)orc_scale_word(r, (uint64_t)s);
    memcpy(C, S + i0 * (int64_t)d, sizeof(float) * (size_t)d);
    degenerate[0] = 0;
  }
  /* D(x)^2 to the nearest live centroid. */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s; ++i) {
    float best = INFINITY;
    for (int32_t j = 0; j < k; ++j) {
      if (degenerate[j]) continue;
      float v = orc_dist32(S + i * (int64_t)d, C + (int64_t)j * d, d);
      if (v < best) best = v;
    }
    w[i] = best;
  }
  int64_t t = 0;
  for (int32_t j = 0; j < k; ++j) {
    if (!degenerate[j]) continue;
    float M = 0.0f;
    for (int64_t i = 0; i < s; ++i)
      if (w[i] > M) M = w[i];
    if (!(M > 0.0f)) break; /* no row is away from the live centroids */
    int F = orc_fixed_scale(M, s);
    uint64_t Q = 0;
    for (int64_t i = 0; i < s; ++i) Q += (uint64_t)orc_quant(w[i], F);
    int64_t best_l = -1;
    uint64_t best_phi = 0;
    for (int32_t l = 0; l < L; ++l) {
      uint64_t r = orc_draw(seed, worker, round, ORC_TAG_SEED,
                            1u + (uint64_t)t * (uint64_t)L + (uint64_t)l);
      uint64_t target = orc_scale_word(r, Q);
      uint64_t run = 0;
      int64_t ci = -1;
      for (int64_t i = 0; i < s; ++i) {
        run += (uint64_t)orc_quant(w[i], F);
        if (run > target) {
          ci = i;
          break;
        }
      }
      cand[l] = ci;
      float *dl = dc + (int64_t)l * s;
      const float *xc = S + ci * (int64_t)d;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < s; ++i) dl[i] = orc_dist32(S + i * (int64_t)d, xc, d);
      uint64_t phi = 0;
      for (int64_t i = 0; i < s; ++i)
        phi += (uint64_t)orc_quant(dl[i] < w[i] ? dl[i] : w[i], F);
      if (cand_out) cand_out[(int64_t)j * L + l] = ci;
      if (phi_out) phi_out[(int64_t)j * L + l] = (int64_t)phi;
      if (best_l < 0 || phi < best_phi) {
        best_l = l;
        best_phi = phi;
      }
    }
    memcpy(C + (int64_t)j * d, S + cand[best_l] * (int64_t)d, sizeof(float) * (size_t)d);
    degenerate[j] = 0;
    const float *dl = dc + best_l * s;
    for (int64_t i = 0; i < s; ++i)
      if (dl[i] < w[i]) w[i] = dl[i];
    ++t;
  }
  free(w);
  free(dc);
  free(cand);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Full-data objective f(C, X) of Eq. 1 over the live centroids, with the
 * optional final assignment Y (§3, last step; Algorithms 3-5, last line). */
double orc_objective(const float *X, int64_t n, int32_t d, const float *C,
                     int32_t k, const uint8_t *degenerate, int32_t *labels) {
  if (n == 0) return 0.0;
  return orc_assign(X, n, d, C, k, degenerate, labels, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* One round of HPClust for W workers (one pass of the while-loop body of
 * Algorithm 3 or 4, every worker once).
 *
 * Worker w: draw S_w (size s[w]) with the SAMPLE stream of (seed, w, round);
 * take the base centroids — its own C_w (competitive, Algorithm 3) or those
 * of the worker with the smallest incumbent objective among the workers of
 * its group (cooperative, Algorithm 4; snapshot at the start of the round,
 * lowest worker index on ties); re-seed the degenerate base centroids with
 * K-means++ on S_w; run Lloyd from them; and if the new sample objective per
 * sample point is strictly below fhat[w] (Algorithm 3's incumbent test,
 * normalised by s_w because workers may draw samples of different sizes),
 * replace C_w, its degenerate flags and fhat[w].
 *
 * C_pool holds every worker's k[w] x d centroids at float offset C_off[w];
 * deg_pool the matching flags at offset K_off[w].  f_new_out / iters_out /
 * accepted_out (nullable) report each worker's Lloyd objective, update count
 * and whether the incumbent was replaced. */
int orc_round(const float *X, int64_t n, int32_t d, int32_t W, const int64_t *s,
              const int32_t *k, const int32_t *group, float *C_pool,
              const int64_t *C_off, uint8_t *deg_pool, const int64_t *K_off,
              double *fhat, int32_t strategy, uint64_t seed, uint32_t round,
              int32_t max_iter, double rel_tol, int32_t L, double *f_new_out,
              int32_t *iters_out, uint8_t *accepted_out, int32_t n_competitive,
              int32_t worker0) {
  /* worker0: the index of this set's first worker among all the workers of
   * the run, so that worker w draws from its own stream (seed, worker0 + w)
   * however the workers are split between processes (Section 5.3: one
   * independent random stream per worker). */
  if (W < 1 || d < 1 || n < 1 || worker0 < 0) return ORC_ERR_ARG;
  /* Algorithm 5 runs its phases in order over the round counter t_w (the
   * same for every worker here): the competitive phase while
   * t_w < n_competitive, the cooperative phase after it. */
  if (strategy == ORC_STRAT_HYBRID)
    strategy = (int64_t)round < (int64_t)n_competitive ? ORC_STRAT_COMPETITIVE : ORC_STRAT_COOPERATIVE;
  int64_t pool_f = 0, pool_k = 0;
  for (int32_t w = 0; w < W; ++w) {
    if (s[w] < 1 || k[w] < 1) return ORC_ERR_ARG;
    int64_t ef = C_off[w] + (int64_t)k[w] * d, ek = K_off[w] + k[w];
    if (ef > pool_f) pool_f = ef;
    if (ek > pool_k) pool_k = ek;
  }
  /* Round-start snapshot for the cooperative base selection. */
  float *C_snap = (float *)malloc(sizeof(float) * (size_t)pool_f);
  uint8_t *deg_snap = (uint8_t *)malloc((size_t)pool_k);
  double *fhat_snap = (double *)malloc(sizeof(double) * (size_t)W);
  memcpy(C_snap, C_pool, sizeof(float) * (size_t)pool_f);
  memcpy(deg_snap, deg_pool, (size_t)pool_k);
  memcpy(fhat_snap, fhat, sizeof(double) * (size_t)W);
  int rc = ORC_OK;
  for (int32_t w = 0; w < W && rc == ORC_OK; ++w) {
    int32_t kw = k[w];
    float *Sw = (float *)malloc(sizeof(float) * (size_t)s[w] * (size_t)d);
    float *Cn = (float *)malloc(sizeof(float) * (size_t)kw * (size_t)d);
    uint8_t *dn = (uint8_t *)malloc((size_t)kw);
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)s[w]);
    orc_draw_sample(X, n, d, seed, (uint32_t)(worker0 + w), round, s[w], Sw, NULL);
    int32_t b = w;
    if (strategy == ORC_STRAT_COOPERATIVE) {
      for (int32_t v = 0; v < W; ++v) {
        if (group[v] != group[w] || k[v] != kw) continue;
        if (fhat_snap[v] < fhat_snap[b] || (fhat_snap[v] == fhat_snap[b] && v < b)) b = v;
      }
    }
    memcpy(Cn, C_snap + C_off[b], sizeof(float) * (size_t)kw * (size_t)d);
    memcpy(dn, deg_snap + K_off[b], (size_t)kw);
    double f = 0.0;
    int32_t iters = 0;
    rc = orc_kmeanspp(Sw, s[w], d, kw, Cn, dn, L, seed, (uint32_t)(worker0 + w), round, NULL,
                      NULL);
    if (rc == ORC_OK)
      rc = orc_lloyd(Sw, s[w], d, kw, Cn, dn, max_iter, rel_tol, lab, &f, &iters, NULL);
    if (rc == ORC_OK) {
      double per_point = f / (double)s[w];
      uint8_t acc = per_point < fhat[w];
      if (acc) {
        memcpy(C_pool + C_off[w], Cn, sizeof(float) * (size_t)kw * (size_t)d);
        memcpy(deg_pool + K_off[w], dn, (size_t)kw);
        fhat[w] = per_point;
      }
      if (f_new_out) f_new_out[w] = f;
      if (iters_out) iters_out[w] = iters;
      if (accepted_out) accepted_out[w] = acc;
    }
    free(Sw);
    free(Cn);
    free(dn);
    free(lab);
  }
  free(C_snap);
  free(deg_snap);
  free(fhat_snap);
  return rc;
}
