/*
 * kmref -- plain FP64 CPU oracle of one Lloyd k-means iteration (and of the
 * keyed-reduce training and SPADE downsampling sections at the end).
 *
 * TEST INFRASTRUCTURE ONLY. It exists so that tests (and the benchmark's CPU
 * baseline leg) can check the GPU library against an obviously correct
 * reference. No product code path may link, load or call it, and it shares no
 * code, header, helper or constant with the GPU library.
 *
 * What it computes is the textbook definition of a Lloyd iteration
 * (S. P. Lloyd, "Least squares quantization in PCM", IEEE Trans. IT 28(2), 1982),
 * built from the paper's loop patterns:
 *   - the assignment is a collect over the point range whose body runs once per
 *     index in no set order (DeliteOpLoop with a DeliteCollectElem, Sec. 2.4),
 *     with the distance of Sec. 3.4 (dist = norm(v1 - v2), the norm being the
 *     square root of the summed squares). The square root is monotone, so the
 *     argmin is taken over squared distances and never rounds two distinct
 *     distances into a false tie;
 *   - sums and counts are a keyed reduce over the same range (DeliteReduceElem,
 *     Sec. 2.4); fused or not (Sec. 3.5) the result is the same, so the oracle
 *     runs them as separate plain loops;
 *   - the new centroid is the member mean, avg = sum / length (the VectorOpsExp
 *     listing of Sec. 2.1).
 * Everything is FP64. Inputs X are FP32 and promote exactly; C is FP64.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - metric: squared Euclidean distance (Lloyd); the paper's only generated
 *     distance loop (the SPADE example of Sec. 4.1) is L1 and belongs to SPADE;
 *   - ties: the lowest centroid index wins (strict < scan from j = 0);
 *   - empty cluster: keeps its previous centroid, sums = 0, counts = 0;
 *   - objective of a step: J(a^t, C^t) = sum_i D(i, a_i) with the centroids
 *     used for the assignment;
 *   - stop rule of a run with tol > 0: after the first step whose assignment
 *     equals the previous step's, or whose largest centroid shift is <= tol.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the point loops (0 = OpenMP default). Returns the count in effect. */
int kmref_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

static int bad_args(const float* X, int64_t n, int32_t d, const void* C, int32_t k) {
  return !X || !C || n < 1 || d < 1 || k < 1 || (int64_t)k > n;
}

/* Squared Euclidean distance, direct differences, summed in index order (Sec. 3.4). */
static double sqdist(const float* x, const double* c, int32_t d) {
  double s = 0.0;
  for (int32_t t = 0; t < d; ++t) {
    double diff = (double)x[t] - c[t];
    s += diff * diff;
  }
  return s;
}

/*
 * Assignment step. For each point i:
 *   D_ij = sum_t (x_it - c_jt)^2,  a_i = min{ j : D_ij <= D_ij' for all j' }.
 * Optional outputs (NULL to skip): dmin[i] = D_{i,a_i}; second[i] = the index
 * of the second-smallest distance (lowest index among equals, excluding a_i;
 * -1 when k = 1); gap[i] = (D_(2) - D_(1)) / max(D_(2), DBL_MIN), +inf when k = 1.
 */
int kmref_assign(const float* X, int64_t n, int32_t d, const double* C, int32_t k,
                 int32_t* assign, double* dmin, double* gap, int32_t* second) {
  if (bad_args(X, n, d, C, k) || !assign) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const float* x = X + i * (int64_t)d;
    double b1 = HUGE_VAL, b2 = HUGE_VAL;
    int32_t j1 = -1, j2 = -1;
    for (int32_t j = 0; j < k; ++j) {
      double D = sqdist(x, C + (int64_t)j * d, d);
      if (D < b1) {
        b2 = b1; j2 = j1;
        b1 = D; j1 = j;
      } else if (D < b2) {
        b2 = D; j2 = j;
      }
    }
    assign[i] = j1;
    if (dmin) dmin[i] = b1;
    if (second) second[i] = j2;
    if (gap) gap[i] = (k == 1) ? HUGE_VAL : (b2 - b1) / (b2 > DBL_MIN ? b2 : DBL_MIN);
  }
  return 0;
}

/*
 * Update step from a given assignment: counts_j = |{i : a_i = j}|,
 * sums_j = sum_{a_i = j} x_i (index order), Cnew_j = sums_j / counts_j, or
 * Cprev_j when counts_j = 0. sums is k*d, counts is k, Cnew is k*d
 * (Cnew may alias Cprev).
 */
int kmref_update(const float* X, int64_t n, int32_t d, const int32_t* assign, int32_t k,
                 const double* Cprev, double* sums, int64_t* counts, double* Cnew) {
  if (!X || !assign || !Cprev || !sums || !counts || !Cnew || n < 1 || d < 1 || k < 1) return -1;
  memset(sums, 0, sizeof(double) * (size_t)k * (size_t)d);
  memset(counts, 0, sizeof(int64_t) * (size_t)k);
  for (int64_t i = 0; i < n; ++i) {
    int32_t j = assign[i];
    if (j < 0 || j >= k) return -2;
    counts[j] += 1;
    double* s = sums + (int64_t)j * d;
    const float* x = X + i * (int64_t)d;
    for (int32_t t = 0; t < d; ++t) s[t] += (double)x[t];
  }
  for (int32_t j = 0; j < k; ++j) {
    double* c = Cnew + (int64_t)j * d;
    const double* cp = Cprev + (int64_t)j * d;
    const double* s = sums + (int64_t)j * d;
    for (int32_t t = 0; t < d; ++t) c[t] = counts[j] > 0 ? s[t] / (double)counts[j] : cp[t];
  }
  return 0;
}

/* Objective J = sum_i D(i, a_i) for the given centroids and assignment. */
double kmref_objective(const float* X, int64_t n, int32_t d, const double* C, int32_t k,
                       const int32_t* assign) {
  if (bad_args(X, n, d, C, k) || !assign) return NAN;
  double J = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t j = assign[i];
    if (j < 0 || j >= k) return NAN;
    J += sqdist(X + i * (int64_t)d, C + (int64_t)j * d, d);
  }
  return J;
}

/* Largest centroid shift max_j ||a_j - b_j||_2. */
static double max_shift(const double* a, const double* b, int32_t k, int32_t d) {
  double m = 0.0;
  for (int32_t j = 0; j < k; ++j) {
    double s = 0.0;
    for (int32_t t = 0; t < d; ++t) {
      double e = a[(int64_t)j * d + t] - b[(int64_t)j * d + t];
      s += e * e;
    }
    if (sqrt(s) > m) m = sqrt(s);
  }
  return m;
}

/*
 * One Lloyd step: assignment with C, then update. C (k*d, FP64) is replaced by
 * the new centroids. objective (optional) receives J(a, C_old); shift
 * (optional) receives the largest centroid shift.
 */
int kmref_step(const float* X, int64_t n, int32_t d, double* C, int32_t k, int32_t* assign,
               double* sums, int64_t* counts, double* objective, double* shift) {
  if (bad_args(X, n, d, C, k) || !assign || !sums || !counts) return -1;
  double* Cold = (double*)malloc(sizeof(double) * (size_t)k * (size_t)d);
  if (!Cold) return -3;
  memcpy(Cold, C, sizeof(double) * (size_t)k * (size_t)d);
  int rc = kmref_assign(X, n, d, Cold, k, assign, NULL, NULL, NULL);
  if (rc == 0) rc = kmref_update(X, n, d, assign, k, Cold, sums, counts, C);
  if (rc == 0 && objective) *objective = kmref_objective(X, n, d, Cold, k, assign);
  if (rc == 0 && shift) *shift = max_shift(C, Cold, k, d);
  free(Cold);
  return rc;
}

/*
 * Up to `iters` Lloyd steps from C. tol <= 0: exactly `iters` steps. tol > 0:
 * stop after the first step whose assignment equals the previous step's or
 * whose largest centroid shift is <= tol. obj_hist (optional, length iters)
 * receives J of each step; *iters_done (optional) the number of steps run.
 */
int kmref_run(const float* X, int64_t n, int32_t d, double* C, int32_t k, int32_t* assign,
              double* sums, int64_t* counts, int32_t iters, double tol, double* obj_hist,
              int32_t* iters_done) {
  if (bad_args(X, n, d, C, k) || !assign || !sums || !counts || iters < 0) return -1;
  int32_t* prev = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!prev) return -3;
  int32_t done = 0;
  int rc = 0;
  for (int32_t t = 0; t < iters; ++t) {
    if (t > 0) memcpy(prev, assign, sizeof(int32_t) * (size_t)n);
    double J = 0.0, shift = 0.0;
    rc = kmref_step(X, n, d, C, k, assign, sums, counts, &J, &shift);
    if (rc) break;
    if (obj_hist) obj_hist[t] = J;
    done = t + 1;
    if (tol > 0.0) {
      int same = t > 0 && memcmp(prev, assign, sizeof(int32_t) * (size_t)n) == 0;
      if (same || shift <= tol) break;
    }
  }
  if (iters_done) *iters_done = done;
  free(prev);
  return rc;
}

/*
 * Keyed-reduce training of the paper's two GPU classifiers, naive Bayes (NB)
 * and Gaussian discriminant analysis (GDA) (the GPU results of Sec. 5): both
 * reduce labelled rows keyed by class (DeliteReduceElem, Sec. 2.4), the same
 * pattern as the k-means sums with the label in place of the assignment.
 * FP64, rows in index order. y_i must lie in [0, ncls).
 *
 * Readings where the paper gives no formula (also in the design notes):
 *   - GDA: shared covariance for any number of classes,
 *       phi_c = n_c / n,  mu_c = (1 / n_c) sum_{y_i = c} x_i  (0 when n_c = 0),
 *       Sigma = (1 / n) sum_i (x_i - mu_{y_i}) (x_i - mu_{y_i})^T;
 *   - NB: multinomial with add-one (Laplace) smoothing over d features,
 *       prior_c = n_c / n,  S_cj = sum_{y_i = c} x_ij,
 *       theta_cj = (S_cj + 1) / (sum_j S_cj + d).
 */

/* n_c and the class sums S_c (ncls x d), index order. */
static int class_sums(const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls, double* sums,
                      int64_t* counts) {
  if (!X || !y || !sums || !counts || n < 1 || d < 1 || ncls < 1) return -1;
  memset(sums, 0, sizeof(double) * (size_t)ncls * (size_t)d);
  memset(counts, 0, sizeof(int64_t) * (size_t)ncls);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t c = y[i];
    if (c < 0 || c >= ncls) return -2;
    counts[c] += 1;
    double* s = sums + (int64_t)c * d;
    const float* x = X + i * (int64_t)d;
    for (int32_t t = 0; t < d; ++t) s[t] += (double)x[t];
  }
  return 0;
}

/* GDA: phi (ncls), mu (ncls x d), sigma (d x d, row-major, symmetric). */
int kmref_gda(const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls, double* phi, double* mu,
              double* sigma) {
  if (!phi || !mu || !sigma) return -1;
  int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncls);
  double* c = (double*)malloc(sizeof(double) * (size_t)d);
  if (!counts || !c) {
    free(counts);
    free(c);
    return -3;
  }
  int rc = class_sums(X, n, d, y, ncls, mu, counts);
  if (rc == 0) {
    for (int32_t k = 0; k < ncls; ++k) {
      phi[k] = (double)counts[k] / (double)n;
      for (int32_t t = 0; t < d; ++t)
        mu[(int64_t)k * d + t] = counts[k] > 0 ? mu[(int64_t)k * d + t] / (double)counts[k] : 0.0;
    }
    memset(sigma, 0, sizeof(double) * (size_t)d * (size_t)d);
    for (int64_t i = 0; i < n; ++i) {
      const float* x = X + i * (int64_t)d;
      const double* m = mu + (int64_t)y[i] * d;
      for (int32_t t = 0; t < d; ++t) c[t] = (double)x[t] - m[t];
      for (int32_t a = 0; a < d; ++a)
        for (int32_t b = a; b < d; ++b) sigma[(int64_t)a * d + b] += c[a] * c[b];
    }
    for (int32_t a = 0; a < d; ++a)
      for (int32_t b = a; b < d; ++b) {
        const double v = sigma[(int64_t)a * d + b] / (double)n;
        sigma[(int64_t)a * d + b] = v;
        sigma[(int64_t)b * d + a] = v;
      }
  }
  free(counts);
  free(c);
  return rc;
}

/* NB: prior (ncls), theta (ncls x d). */
int kmref_nb(const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls, double* prior, double* theta) {
  if (!prior || !theta) return -1;
  int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncls);
  if (!counts) return -3;
  int rc = class_sums(X, n, d, y, ncls, theta, counts);
  if (rc == 0) {
    for (int32_t k = 0; k < ncls; ++k) {
      prior[k] = (double)counts[k] / (double)n;
      double* s = theta + (int64_t)k * d;
      double total = 0.0;
      for (int32_t t = 0; t < d; ++t) total += s[t];
      for (int32_t t = 0; t < d; ++t) s[t] = (s[t] + 1.0) / (total + (double)d);
    }
  }
  free(counts);
  return rc;
}

/* ------------------------------------------------------------------------
 * SPADE density downsampling (Sec. 4.1, "Downsampling in Bioinformatics").
 *
 * The paper's loop over the rows of a distance Stream: a row whose density is
 * still 0 is evaluated, i.e. its distances to every row are formed, the rows
 * within apprx_width are found and the rows within kernel_width are counted
 * (find and count fused into one pass), and every found row's density is set
 * to that count; rows with a density already set are skipped. Distances are
 * L1 in FP64 (the generated code's inner loop: difference, absolute value,
 * running sum over the columns in order; the Stream holds Doubles).
 *
 * Readings (each also listed in the design notes):
 *   - order: the loop runs as if sequentially over i = 0..n-1 (the C++
 *     snippet's OpenMP loop races on the skip test; its sequential reading is
 *     the one the generated code has);
 *   - policy 0 (the generated OptiML code): c = #{j : D(i,j) < kernel_width},
 *     and the bulk update overwrites every found row's density;
 *   - policy 1 (the C++ snippet): c also counts D < apprx_width (its else-if),
 *     a found row's density is set only while it is still 0 (the
 *     compare-and-swap), and the row's own density is set to c.
 * ------------------------------------------------------------------------ */

/* D(i, j): the generated code's L1 loop in FP64, columns in increasing order. */
static double l1dist(const float* x, const float* y, int32_t d) {
  double s = 0.0;
  for (int32_t t = 0; t < d; ++t) s += fabs((double)x[t] - (double)y[t]);
  return s;
}

/* #{j : D(i, j) < width} over all n rows (row i itself included). */
int64_t spaderef_count(const float* X, int64_t n, int32_t d, int64_t i, double width) {
  if (!X || n < 1 || d < 1 || i < 0 || i >= n) return -1;
  const float* xi = X + i * (int64_t)d;
  int64_t c = 0;
#pragma omp parallel for reduction(+ : c) schedule(static)
  for (int64_t j = 0; j < n; ++j) c += l1dist(xi, X + j * (int64_t)d, d) < width;
  return c;
}

/* The downsampling loop. dens[n]: the final densities. counts[n]: c of every
 * evaluated row, -1 for skipped rows. processed[n]: 1 for evaluated rows.
 * Requires apprx_width > 0 and kernel_width > 0 (every evaluated row then
 * finds itself, so its density becomes nonzero). */
int spaderef_densities(const float* X, int64_t n, int32_t d, double apprx, double kernel, int32_t policy,
                       int32_t* dens, int32_t* counts, uint8_t* processed) {
  if (!X || !dens || !counts || !processed || n < 1 || d < 1 || !(apprx > 0.0) || !(kernel > 0.0) ||
      (policy != 0 && policy != 1))
    return -1;
  uint8_t* found = (uint8_t*)malloc((size_t)n);
  if (!found) return -2;
  for (int64_t i = 0; i < n; ++i) {
    dens[i] = 0;
    counts[i] = -1;
    processed[i] = 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (dens[i] != 0) continue;  /* the skip test */
    processed[i] = 1;
    const float* xi = X + i * (int64_t)d;
    int64_t c = 0;
    /* one fused pass over the row: find (< apprx) and count (< kernel) */
#pragma omp parallel for reduction(+ : c) schedule(static)
    for (int64_t j = 0; j < n; ++j) {
      const double D = l1dist(xi, X + j * (int64_t)d, d);
      found[j] = D < apprx;
      c += policy == 0 ? (D < kernel) : (D < apprx || D < kernel);
    }
    /* the bulk update of the found rows */
    for (int64_t j = 0; j < n; ++j) {
      if (!found[j]) continue;
      if (policy == 0 || dens[j] == 0) dens[j] = (int32_t)c;
    }
    if (policy == 1) dens[i] = (int32_t)c;
    counts[i] = (int32_t)c;
  }
  free(found);
  return 0;
}

/* For row i and a given evaluated-row set: the lowest and highest evaluated
 * row j with D(i, j) < apprx (-1 when there is none). Used to check a result
 * at sizes where the whole loop is too slow to rerun. */
int spaderef_cover(const float* X, int64_t n, int32_t d, int64_t i, double apprx, const uint8_t* processed,
                   int64_t* first, int64_t* last) {
  if (!X || !processed || !first || !last || n < 1 || d < 1 || i < 0 || i >= n) return -1;
  const float* xi = X + i * (int64_t)d;
  int64_t lo = INT64_MAX, hi = -1;
#pragma omp parallel for reduction(min : lo) reduction(max : hi) schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    if (!processed[j]) continue;
    if (l1dist(xi, X + j * (int64_t)d, d) < apprx) {
      if (j < lo) lo = j;
      if (j > hi) hi = j;
    }
  }
  *first = hi < 0 ? -1 : lo;
  *last = hi;
  return 0;
}
