/*
 * Seeded synthetic inputs for the Lloyd k-means workloads: isotropic Gaussian
 * mixtures drawn with a counter-based generator, so every element is a pure
 * function of (seed, stream, index) and any subset of rows can be regenerated
 * independently of thread count or order.
 *
 * This module holds none of the k-means arithmetic. It is shared by the FP64
 * oracle's tests and by the GPU path's tests and benchmark, and by nothing
 * else.
 *
 * Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014). The i-th output for a key K is
 * mix(K + (i+1)*0x9E3779B97F4A7C15) with the published mixing function.
 * Normals: Box-Muller on pairs of uniforms in (0,1).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

enum { STREAM_MEANS = 1, STREAM_COMP = 2, STREAM_NOISE = 3, STREAM_META = 4 };

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Key of an independent stream: SplitMix64 output #stream for the seed. */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed + (stream + 1) * GOLDEN);
}

static inline uint64_t draw(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1) * GOLDEN);
}

/* Uniform in the open interval (0,1): 53 random bits, centred in their cell. */
static inline double u01(uint64_t key, uint64_t ctr) {
  return ((double)(draw(key, ctr) >> 11) + 0.5) * 0x1.0p-53;
}

static inline double normal(uint64_t key, uint64_t e) {
  uint64_t p = e >> 1;
  double u1 = u01(key, 2 * p), u2 = u01(key, 2 * p + 1);
  double r = sqrt(-2.0 * log(u1));
  double th = 6.283185307179586476925286766559 * u2;
  return (e & 1) ? r * sin(th) : r * cos(th);
}

/* Output #i of a plain SplitMix64 generator started from `state`. */
uint64_t synth_splitmix64(uint64_t state, uint64_t i) {
  return draw(state, i);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return draw(stream_key(seed, stream), ctr);
}

double synth_u01(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return u01(stream_key(seed, stream), ctr);
}

double synth_normal(uint64_t seed, uint64_t stream, uint64_t e) {
  return normal(stream_key(seed, stream), e);
}

/* Component means: mu[c*d + t] = -R + 2R*U(c*d + t), c < m. */
void synth_means(uint64_t seed, int64_t m, int64_t d, double R, double* mu) {
  uint64_t km = stream_key(seed, STREAM_MEANS);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m * d; ++e) mu[e] = -R + 2.0 * R * u01(km, (uint64_t)e);
}

/* Component of point i: floor(U(i) * m), equal weights. */
static inline int64_t comp_of(uint64_t kc, int64_t i, int64_t m) {
  int64_t c = (int64_t)(u01(kc, (uint64_t)i) * (double)m);
  return c < m ? c : m - 1;
}

/*
 * Rows [row0, row0+rows) of the mixture: x_i = mu_{comp(i)} + sigma * N(0, I),
 * rounded to FP32. `mu` must hold synth_means(seed, m, d, R). `comp` may be
 * NULL. Rows are independent of which other rows are generated.
 */
void synth_mixture_rows(uint64_t seed, int64_t row0, int64_t rows, int64_t d,
                        int64_t m, const double* mu, double sigma, float* X,
                        int32_t* comp) {
  uint64_t kc = stream_key(seed, STREAM_COMP), kn = stream_key(seed, STREAM_NOISE);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rows; ++r) {
    int64_t i = row0 + r;
    int64_t c = comp_of(kc, i, m);
    if (comp) comp[r] = (int32_t)c;
    const double* mc = mu + c * d;
    float* xr = X + r * d;
    for (int64_t t = 0; t < d; ++t)
      xr[t] = (float)(mc[t] + sigma * normal(kn, (uint64_t)(i * d + t)));
  }
}

/*
 * Shape of instance b of the batched workload (seed = base + b):
 * n log-uniform in [1e3, 2e5], d uniform in {8, 32, 64, 128},
 * k log-uniform in [4, 512] (clamped to n).
 */
void synth_instance_shape(uint64_t seed, int64_t* n, int32_t* d, int32_t* k) {
  static const int32_t dims[4] = {8, 32, 64, 128};
  uint64_t km = stream_key(seed, STREAM_META);
  double un = u01(km, 0), ud = u01(km, 1), uk = u01(km, 2);
  *n = (int64_t)llround(exp(log(1e3) + un * (log(2e5) - log(1e3))));
  int di = (int)(ud * 4.0);
  *d = dims[di > 3 ? 3 : di];
  int64_t kk = (int64_t)llround(exp(log(4.0) + uk * (log(512.0) - log(4.0))));
  if (kk > *n) kk = *n;
  *k = (int32_t)kk;
}
