// Keyed-reduce training of the paper's GPU classifiers (Sec. 5): shared-
// covariance Gaussian discriminant analysis (GDA) and multinomial naive Bayes
// (NB). Both are the keyed reduce of a Lloyd step (Sec. 2.4) keyed by a class
// label instead of the assignment: the count / scan / scatter / segmented-sum
// stages of km_reduce.cu produce n_c and the class sums S_c (FP32 Kahan runs
// combined in FP64); the kernels here finish them.
//
//   GDA: phi_c = n_c / n, mu_c = S_c / n_c (0 for an empty class),
//        Sigma = (1/n) sum_i (x_i - mu_{y_i}) (x_i - mu_{y_i})^T;
//   NB:  prior_c = n_c / n, theta_cj = (S_cj + 1) / (sum_j S_cj + d).
//
// Sigma is a sum of n outer products (a d x d reduction over the rows). Each
// CTA owns one 64 x 64 tile of its upper triangle and a contiguous range of
// rows; it stages 32 centred rows at a time in shared memory (x - mu_{y_i}
// with the FP32 class mean: centring with the rounded mean changes Sigma only
// to second order, since sum_i (x_i - mu_{y_i}) vanishes per class), forms the
// 32-row partial of every entry with FP32 FMAs (relative error <= 33u of the
// partial's sum of |terms|), adds the partial to an FP64 register accumulator,
// and adds its accumulators to the FP64 result once at the end.
#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kCovT = 64;  // Sigma tile edge
constexpr int kCovR = 32;  // rows per FP32 partial

// Flags a label outside [0, ncls); the later stages then return at entry.
__global__ void check_classes_kernel(const int32_t* __restrict__ y, int64_t n, int ncls, Ctl* ctl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = y[i];
    if (c < 0 || c >= ncls) {
      ctl->done = 1;
      ctl->error = KM_EINVAL;
    }
  }
}

// GDA: phi and mu from the class sums (one warp per class, FP64 division).
__global__ void __launch_bounds__(256)
gda_means_kernel(const double* __restrict__ sums64, const int32_t* __restrict__ counts, int64_t n, int d, int ncls,
                 float* __restrict__ phi, float* __restrict__ mu, const Ctl* ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < ncls; c += nw) {
    const int cnt = counts[c];
    for (int t = lane; t < d; t += 32)
      mu[(int64_t)c * d + t] = cnt > 0 ? (float)(sums64[(int64_t)c * d + t] / (double)cnt) : 0.f;
    if (lane == 0) phi[c] = (float)((double)cnt / (double)n);
  }
}

// NB: prior and the smoothed class feature distributions (one warp per class).
__global__ void __launch_bounds__(256)
nb_theta_kernel(const double* __restrict__ sums64, const int32_t* __restrict__ counts, int64_t n, int d, int ncls,
                float* __restrict__ prior, float* __restrict__ theta, const Ctl* ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < ncls; c += nw) {
    const double* s = sums64 + (int64_t)c * d;
    double total = 0.0;
    for (int t = lane; t < d; t += 32) total += s[t];
#pragma unroll
    for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    const double den = total + (double)d;
    for (int t = lane; t < d; t += 32) theta[(int64_t)c * d + t] = (float)((s[t] + 1.0) / den);
    if (lane == 0) prior[c] = (float)((double)counts[c] / (double)n);
  }
}

// One 64 x 64 tile (ta <= tb) of the upper triangle of sum_i c_i c_i^T over a
// contiguous row range; 256 threads, 4 x 4 entries each.
__global__ void __launch_bounds__(256)
gda_cov_kernel(const float* __restrict__ X, int64_t n, int d, const int32_t* __restrict__ y,
               const float* __restrict__ mu, const int2* __restrict__ tiles, int nsplit,
               double* __restrict__ sigma64, const Ctl* ctl) {
  if (halted(ctl)) return;
  __shared__ __align__(16) float Ca[kCovR][kCovT + 4], Cb[kCovR][kCovT + 4];
  const int2 tile = tiles[blockIdx.x / nsplit];
  const int split = blockIdx.x % nsplit;
  const int a0 = tile.x * kCovT, b0 = tile.y * kCovT;
  const int64_t r0 = n * split / nsplit, r1 = n * (split + 1) / nsplit;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dacc[i][j] = 0.0;
  for (int64_t rb = r0; rb < r1; rb += kCovR) {
    const int rows = (int)min((int64_t)kCovR, r1 - rb);
    // stage the centred a- and b-columns of up to 32 rows (zero past the rows and past d)
    for (int e = tid; e < kCovR * 2 * kCovT; e += 256) {
      const int r = e / (2 * kCovT), col = e % (2 * kCovT);
      const int t = col < kCovT ? a0 + col : b0 + col - kCovT;
      float v = 0.f;
      if (r < rows && t < d) {
        const int64_t i = rb + r;
        v = __fsub_rn(X[i * d + t], mu[(int64_t)y[i] * d + t]);
      }
      if (col < kCovT) Ca[r][col] = v;
      else Cb[r][col - kCovT] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int r = 0; r < kCovR; ++r) {
      const float4 av = *reinterpret_cast<const float4*>(&Ca[r][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Cb[r][tx * 4]);
      const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) dacc[i][j] += (double)acc[i][j];
    __syncthreads();  // every thread is done with the stage before it is refilled
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx * 4 + j;
      if (a < d && b < d && dacc[i][j] != 0.0) atomicAdd(sigma64 + (int64_t)a * d + b, dacc[i][j]);
    }
  }
}

// Sigma = sum / n in FP32, both triangles (an entry in a lower tile is read from its mirror).
__global__ void __launch_bounds__(256)
gda_cov_finish_kernel(const double* __restrict__ sigma64, int d, int64_t n, float* __restrict__ sigma,
                      const Ctl* ctl) {
  if (halted(ctl)) return;
  const int64_t dd = (int64_t)d * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < dd; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / d), b = (int)(e % d);
    const bool upper = a / kCovT <= b / kCovT;
    sigma[e] = (float)(sigma64[upper ? e : (int64_t)b * d + a] / (double)n);
  }
}

}  // namespace

cudaError_t launch_check_classes(const int32_t* y, int64_t n, int ncls, Ctl* ctl, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  check_classes_kernel<<<(int)blocks, 256, 0, s>>>(y, n, ncls, ctl);
  return cudaGetLastError();
}

cudaError_t launch_gda_means(const double* sums64, const int32_t* counts, int64_t n, int d, int ncls, float* phi,
                             float* mu, const Ctl* ctl, cudaStream_t s) {
  const int blocks = (ncls + 7) / 8 < num_sms() * 4 ? (ncls + 7) / 8 : num_sms() * 4;
  gda_means_kernel<<<blocks, 256, 0, s>>>(sums64, counts, n, d, ncls, phi, mu, ctl);
  return cudaGetLastError();
}

cudaError_t launch_nb_theta(const double* sums64, const int32_t* counts, int64_t n, int d, int ncls, float* prior,
                            float* theta, const Ctl* ctl, cudaStream_t s) {
  const int blocks = (ncls + 7) / 8 < num_sms() * 4 ? (ncls + 7) / 8 : num_sms() * 4;
  nb_theta_kernel<<<blocks, 256, 0, s>>>(sums64, counts, n, d, ncls, prior, theta, ctl);
  return cudaGetLastError();
}

// Upper-triangle tiles of a d x d matrix in 64 x 64 tiles.
int gda_cov_tiles(int d) {
  const int t = (d + kCovT - 1) / kCovT;
  return t * (t + 1) / 2;
}

// tiles: device array of gda_cov_tiles(d) int2 (filled here by the host copy);
// sigma64: d x d FP64 accumulators, zero on entry.
cudaError_t launch_gda_cov(const float* X, int64_t n, int d, const int32_t* y, const float* mu, int2* tiles_dev,
                           double* sigma64, float* sigma, const Ctl* ctl, cudaStream_t s) {
  const int tdim = (d + kCovT - 1) / kCovT, nt = gda_cov_tiles(d);
  int2 host[64];  // d <= 256: at most 10 tiles
  int q = 0;
  for (int ta = 0; ta < tdim; ++ta)
    for (int tb = ta; tb < tdim; ++tb) host[q++] = make_int2(ta, tb);
  cudaError_t e = cudaMemcpyAsync(tiles_dev, host, sizeof(int2) * nt, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  // about eight CTAs per SM in all, each with at least 32 rows
  int64_t nsplit = (int64_t)num_sms() * 8 / nt;
  if (nsplit < 1) nsplit = 1;
  if (nsplit > (n + kCovR - 1) / kCovR) nsplit = (n + kCovR - 1) / kCovR;
  gda_cov_kernel<<<(int)(nt * nsplit), 256, 0, s>>>(X, n, d, y, mu, tiles_dev, (int)nsplit, sigma64, ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t dd = (int64_t)d * d;
  int64_t blocks = (dd + 255) / 256;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  gda_cov_finish_kernel<<<(int)blocks, 256, 0, s>>>(sigma64, d, n, sigma, ctl);
  return cudaGetLastError();
}

}  // namespace km
