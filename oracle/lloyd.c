/*
 * FP64 CPU oracle for Lloyd's K-means -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the checker the GPU path is compared against.  Only the tests,
 * the smoke entry point and the CPU-baseline leg of the benchmark may load it;
 * the product library never links or calls it.  It shares no code with the
 * CUDA path.
 *
 * Every step follows the paper's statement of the method, in the paper's order:
 *   - Reassignment (section "The Lloyd's algorithm", step 2):
 *       z_i = argmin_k ||x_i - mu_k||_2^2
 *   - Mean calculation (same section, step 3):
 *       mu_k = sum_i 1(z_i = k) x_i / sum_i 1(z_i = k)
 *   - Convergence error (section "Serial Lloyd's algorithm"):
 *       E^2 = sum_k ||mu_k^{t+1} - mu_k^t||_2^2, compared with a tolerance ~1e-6.
 * The objective sum_i ||x_i - mu_{z_i}||^2 is the one stated in the abstract.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes):
 *   - distances are accumulated left to right over the coordinates, in double,
 *     with no fused multiply-add (the file is built with -ffp-contract=off);
 *   - ties in the argmin go to the lowest k;
 *   - a cluster with no points keeps its previous centre (0/0 is undefined);
 *   - the stop test is strict (E < tol) on E = sqrt(E^2) by default, or on the
 *     paper's squared form when e_mode = 1; T counts the steps executed,
 *     including the one whose E passed the test;
 *   - labels are 0..K-1 (the paper writes 1..K).
 *
 * Data layout: X is d x N (paper: X in R^{d x N}); coordinate j of point i is
 * x[j*ld + i], float32.  Centroids are K x d row-major doubles.
 *
 * Per-cluster sums are formed over fixed chunks of ORC_CHUNK points in index
 * order; the chunk partials are then added in chunk order.  The result does
 * not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CHUNK 65536

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ||x_i - mu_k||^2, coordinates in order 0..d-1, no contraction. */
static double orc_sqdist(const float* x, int64_t ld, int64_t i, int32_t d,
                         const double* mu_k) {
  double acc = 0.0;
  for (int32_t j = 0; j < d; ++j) {
    double t = (double)x[(int64_t)j * ld + i] - mu_k[j];
    acc = acc + t * t;
  }
  return acc;
}

/* Reassignment step.  z[i] <- argmin_k D_ik, lowest k on ties.  dmin (may be
 * NULL) receives D_{i z_i}.  Returns 0. */
int orc_assign(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
               const double* mu, int32_t* z, double* dmin) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int32_t best = 0;
    double bestd = orc_sqdist(x, ld, i, d, mu);
    for (int32_t c = 1; c < k; ++c) {
      double dc = orc_sqdist(x, ld, i, d, mu + (int64_t)c * d);
      if (dc < bestd) { bestd = dc; best = c; }
    }
    z[i] = best;
    if (dmin) dmin[i] = bestd;
  }
  return 0;
}

/* Mean-calculation step.  counts[k] = #{i : z_i = k};
 * mu_next[k] = (sum_{z_i = k} x_i) / counts[k], or mu_prev[k] if counts[k] == 0.
 * Returns the number of empty clusters, or -1 on allocation failure. */
int orc_update(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
               const int32_t* z, const double* mu_prev, double* mu_next,
               int64_t* counts) {
  int64_t nchunks = (n + ORC_CHUNK - 1) / ORC_CHUNK;
  if (nchunks == 0) nchunks = 1;
  double* psum = (double*)calloc((size_t)nchunks * k * d, sizeof(double));
  int64_t* pcnt = (int64_t*)calloc((size_t)nchunks * k, sizeof(int64_t));
  if (!psum || !pcnt) { free(psum); free(pcnt); return -1; }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nchunks; ++c) {
    double* s = psum + c * (int64_t)k * d;
    int64_t* m = pcnt + c * (int64_t)k;
    int64_t lo = c * ORC_CHUNK, hi = lo + ORC_CHUNK < n ? lo + ORC_CHUNK : n;
    for (int64_t i = lo; i < hi; ++i) {
      int32_t zi = z[i];
      m[zi] += 1;
      for (int32_t j = 0; j < d; ++j) s[(int64_t)zi * d + j] += (double)x[(int64_t)j * ld + i];
    }
  }
  int empty = 0;
  for (int32_t c = 0; c < k; ++c) {
    int64_t cnt = 0;
    for (int64_t q = 0; q < nchunks; ++q) cnt += pcnt[q * k + c];
    counts[c] = cnt;
    for (int32_t j = 0; j < d; ++j) {
      if (cnt == 0) { mu_next[(int64_t)c * d + j] = mu_prev[(int64_t)c * d + j]; continue; }
      double sum = 0.0;
      for (int64_t q = 0; q < nchunks; ++q) sum += psum[(q * k + c) * (int64_t)d + j];
      mu_next[(int64_t)c * d + j] = sum / (double)cnt;
    }
    if (cnt == 0) ++empty;
  }
  free(psum);
  free(pcnt);
  return empty;
}

/* E^2 = sum_k sum_j (a_kj - b_kj)^2, k then j in order. */
double orc_error2(int32_t k, int32_t d, const double* a, const double* b) {
  double e2 = 0.0;
  for (int64_t q = 0; q < (int64_t)k * d; ++q) {
    double t = a[q] - b[q];
    e2 = e2 + t * t;
  }
  return e2;
}

/* Objective sum_i ||x_i - mu_{z_i}||^2, summed in the same fixed chunk order. */
double orc_objective(const float* x, int64_t ld, int64_t n, int32_t d,
                     const double* mu, const int32_t* z) {
  int64_t nchunks = (n + ORC_CHUNK - 1) / ORC_CHUNK;
  if (nchunks == 0) return 0.0;
  double* part = (double*)calloc((size_t)nchunks, sizeof(double));
  if (!part) return NAN;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nchunks; ++c) {
    int64_t lo = c * ORC_CHUNK, hi = lo + ORC_CHUNK < n ? lo + ORC_CHUNK : n;
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) s += orc_sqdist(x, ld, i, d, mu + (int64_t)z[i] * d);
    part[c] = s;
  }
  double obj = 0.0;
  for (int64_t c = 0; c < nchunks; ++c) obj += part[c];
  free(part);
  return obj;
}

/* One Lloyd step from mu_in: reassignment, mean calculation, error.
 * Writes z, mu_out, counts; returns E^2 (or -1 on allocation failure). */
double orc_step(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
                const double* mu_in, int32_t* z, double* mu_out, int64_t* counts) {
  orc_assign(x, ld, n, d, k, mu_in, z, NULL);
  if (orc_update(x, ld, n, d, k, z, mu_in, mu_out, counts) < 0) return -1.0;
  return orc_error2(k, d, mu_out, mu_in);
}

/* The whole loop (section "Serial Lloyd's algorithm"): iterate steps 2 and 3
 * until the selected error is below tol or max_iter steps have run.
 * e_mode 0: E = sqrt(E^2) is tested; e_mode 1: the paper's squared sum.
 * Returns 0 if converged, 1 if max_iter was reached, -1 on failure. */
int orc_run(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
            const double* mu0, int32_t max_iter, double tol, int32_t e_mode,
            int32_t* z, double* mu_out, int64_t* counts, int32_t* iters,
            double* e_out, double* e2_out, double* obj_out) {
  size_t kd = (size_t)k * d;
  double* cur = (double*)malloc(kd * sizeof(double));
  double* nxt = (double*)malloc(kd * sizeof(double));
  if (!cur || !nxt) { free(cur); free(nxt); return -1; }
  memcpy(cur, mu0, kd * sizeof(double));
  int status = 1;
  int32_t t = 0;
  double e2 = 0.0;
  while (t < max_iter) {
    ++t;
    e2 = orc_step(x, ld, n, d, k, cur, z, nxt, counts);
    if (e2 < 0.0) { status = -1; break; }
    double* tmp = cur; cur = nxt; nxt = tmp;
    double esel = e_mode == 1 ? e2 : sqrt(e2);
    if (esel < tol) { status = 0; break; }
  }
  memcpy(mu_out, cur, kd * sizeof(double));
  *iters = t;
  *e2_out = e2;
  *e_out = sqrt(e2);
  if (obj_out) *obj_out = t > 0 ? orc_objective(x, ld, n, d, cur, z) : NAN;
  free(cur);
  free(nxt);
  return status;
}

/* k-means++ seeding (Arthur & Vassilvitskii, 2007), with the random numbers
 * passed in: u[0] picks the first centre uniformly (index floor(u0 * n)); for
 * c >= 1, u[c] * total picks the first index whose running sum of
 * D^2(i) = min over chosen centres of ||x_i - centre||^2 exceeds it.
 * Running sums are formed in index order.  idx receives the chosen indices. */
int orc_kmeanspp(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
                 const double* u, double* mu_out, int64_t* idx) {
  double* d2 = (double*)malloc((size_t)n * sizeof(double));
  if (!d2 || n <= 0) { free(d2); return -1; }
  int64_t first = (int64_t)floor(u[0] * (double)n);
  if (first >= n) first = n - 1;
  idx[0] = first;
  for (int32_t j = 0; j < d; ++j) mu_out[j] = (double)x[(int64_t)j * ld + first];
  for (int64_t i = 0; i < n; ++i) d2[i] = orc_sqdist(x, ld, i, d, mu_out);
  for (int32_t c = 1; c < k; ++c) {
    double total = 0.0;
    for (int64_t i = 0; i < n; ++i) total += d2[i];
    double target = u[c] * total;
    double run = 0.0;
    int64_t pick = n - 1;
    for (int64_t i = 0; i < n; ++i) {
      run += d2[i];
      if (run > target) { pick = i; break; }
    }
    idx[c] = pick;
    double* mc = mu_out + (int64_t)c * d;
    for (int32_t j = 0; j < d; ++j) mc[j] = (double)x[(int64_t)j * ld + pick];
    for (int64_t i = 0; i < n; ++i) {
      double dc = orc_sqdist(x, ld, i, d, mc);
      if (dc < d2[i]) d2[i] = dc;
    }
  }
  free(d2);
  return 0;
}
