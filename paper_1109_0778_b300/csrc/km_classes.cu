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
// 64-row partial of every entry with FP32 FMAs (relative error <= 65u of the
// partial's sum of |terms|) and Kahan-adds the partials in FP32 (<= ~2u more).
// Each CTA writes its tile partial in FP64; a second kernel sums the partials
// of an entry in a fixed order (so Sigma is reproducible bit for bit) and
// divides by n.
#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kCovT = 64;  // Sigma tile edge
constexpr int kCovR = 64;  // rows per FP32 partial

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
// contiguous row range; 256 threads, 4 x 4 entries each (paired FMAs along b).
// Thread t stages rows t / 8 and t / 8 + 32 of each 64-row chunk, columns
// 16 (t % 8) .. +15 of the a- then b-range, and loads the next chunk while the
// current one is multiplied. The tile partial goes to part[blockIdx.x][64 x 64]
// (FP64).
__global__ void __launch_bounds__(256)
gda_cov_kernel(const float* __restrict__ X, int64_t n, int d, const int32_t* __restrict__ y,
               const float* __restrict__ mu, const int2* __restrict__ tiles, int nsplit,
               double* __restrict__ part, const Ctl* ctl) {
  if (halted(ctl)) return;
  __shared__ __align__(16) float Cs[2][kCovR][kCovT + 4];  // [0]: a-columns, [1]: b-columns
  const int2 tile = tiles[blockIdx.x / nsplit];
  const int split = blockIdx.x % nsplit;
  const int a0 = tile.x * kCovT, b0 = tile.y * kCovT;
  const int64_t r0 = n * split / nsplit, r1 = n * (split + 1) / nsplit;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int sr = tid >> 3, sg = tid & 7;                  // staged rows sr, sr + 32; 16-column group
  const int side = sg >> 2, c0 = (sg & 3) * 16;           // a or b range, first column in it
  const int t0 = (side ? b0 : a0) + c0;                   // first matrix column of the group
  // rows start on 16-byte boundaries (d a multiple of 4, X and the class means 16-byte aligned)
  const bool v4 = (d & 3) == 0 && (((uintptr_t)X | (uintptr_t)mu) & 15) == 0;
  float stage[2][16];
  auto load_row = [&](int64_t i, float (&st)[16]) {  // centred values of row i, columns t0 .. t0 + 15
    if (i < r1) {
      const float* x = X + i * d;
      const float* m = mu + (int64_t)y[i] * d;
      if (v4 && t0 + 16 <= d) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 xv = *reinterpret_cast<const float4*>(x + t0 + 4 * q);
          const float4 mv = *reinterpret_cast<const float4*>(m + t0 + 4 * q);
          st[4 * q] = __fsub_rn(xv.x, mv.x);
          st[4 * q + 1] = __fsub_rn(xv.y, mv.y);
          st[4 * q + 2] = __fsub_rn(xv.z, mv.z);
          st[4 * q + 3] = __fsub_rn(xv.w, mv.w);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) st[q] = t0 + q < d ? __fsub_rn(x[t0 + q], m[t0 + q]) : 0.f;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) st[q] = 0.f;
    }
  };
  auto load = [&](int64_t rb) {
    load_row(rb + sr, stage[0]);
    load_row(rb + sr + 32, stage[1]);
  };
  float2 acc[4][2];
  float ks[4][4], kc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ks[i][j] = kc[i][j] = 0.f;
  if (r0 < r1) load(r0);
  for (int64_t rb = r0; rb < r1; rb += kCovR) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 16; q += 4)
        *reinterpret_cast<float4*>(&Cs[side][sr + 32 * h][c0 + q]) =
            make_float4(stage[h][q], stage[h][q + 1], stage[h][q + 2], stage[h][q + 3]);
    __syncthreads();
    if (rb + kCovR < r1) load(rb + kCovR);  // in flight while this chunk is multiplied
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int r = 0; r < kCovR; ++r) {
      const float4 av = *reinterpret_cast<const float4*>(&Cs[0][r][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Cs[1][r][tx * 4]);
      const float a[4] = {av.x, av.y, av.z, av.w};
      const float2 b01 = make_float2(bv.x, bv.y), b23 = make_float2(bv.z, bv.w);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 ai = make_float2(a[i], a[i]);
        acc[i][0] = __ffma2_rn(ai, b01, acc[i][0]);
        acc[i][1] = __ffma2_rn(ai, b23, acc[i][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      kahan_add(ks[i][0], kc[i][0], acc[i][0].x);
      kahan_add(ks[i][1], kc[i][1], acc[i][0].y);
      kahan_add(ks[i][2], kc[i][2], acc[i][1].x);
      kahan_add(ks[i][3], kc[i][3], acc[i][1].y);
    }
    __syncthreads();  // every thread is done with the stage before it is refilled
  }
  double* out = part + (int64_t)blockIdx.x * kCovT * kCovT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kCovT + tx * 4 + j] = (double)ks[i][j] - (double)kc[i][j];
}

// Sigma_ab = (sum of the tile partials of (a, b)) / n, in FP32, both
// triangles (an entry of a lower tile is read from its mirror). One warp per
// entry: lane l sums splits l, l + 32, ..., then a fixed butterfly, so the
// order (and Sigma) is the same on every run.
__global__ void __launch_bounds__(256)
gda_cov_finish_kernel(const double* __restrict__ part, int d, int64_t n, int nsplit, float* __restrict__ sigma,
                      const Ctl* ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int tdim = (d + kCovT - 1) / kCovT;
  const int64_t dd = (int64_t)d * d;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = gw; e < dd; e += nw) {
    int a = (int)(e / d), b = (int)(e % d);
    if (a / kCovT > b / kCovT) {
      const int t = a;
      a = b;
      b = t;
    }
    const int ta = a / kCovT, tb = b / kCovT;
    const int tile = ta * tdim - ta * (ta - 1) / 2 + (tb - ta);  // row-major index among the upper tiles
    const double* p = part + ((int64_t)tile * nsplit) * kCovT * kCovT + (a - ta * kCovT) * kCovT + (b - tb * kCovT);
    double v = 0.0;
    for (int sp = lane; sp < nsplit; sp += 32) v += p[(int64_t)sp * kCovT * kCovT];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sigma[e] = (float)(v / (double)n);
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

// Row splits per tile: about four CTAs per SM in all, each with at least 64 rows.
int gda_cov_splits(int64_t n, int d) {
  int64_t ns = (int64_t)num_sms() * 4 / gda_cov_tiles(d);
  if (ns < 1) ns = 1;
  if (ns > (n + kCovR - 1) / kCovR) ns = (n + kCovR - 1) / kCovR;
  return (int)ns;
}

// FP64 scratch of the tile partials, in bytes.
size_t gda_cov_scratch_bytes(int64_t n, int d) {
  return (size_t)gda_cov_tiles(d) * gda_cov_splits(n, d) * kCovT * kCovT * sizeof(double);
}

// tiles_dev: device array of gda_cov_tiles(d) int2 (filled here); part: the scratch.
cudaError_t launch_gda_cov(const float* X, int64_t n, int d, const int32_t* y, const float* mu, int2* tiles_dev,
                           double* part, float* sigma, const Ctl* ctl, cudaStream_t s) {
  const int tdim = (d + kCovT - 1) / kCovT, nt = gda_cov_tiles(d), nsplit = gda_cov_splits(n, d);
  int2 host[64];  // d <= 256: at most 10 tiles
  int q = 0;
  for (int ta = 0; ta < tdim; ++ta)
    for (int tb = ta; tb < tdim; ++tb) host[q++] = make_int2(ta, tb);
  cudaError_t e = cudaMemcpyAsync(tiles_dev, host, sizeof(int2) * nt, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  gda_cov_kernel<<<nt * nsplit, 256, 0, s>>>(X, n, d, y, mu, tiles_dev, nsplit, part, ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t dd = (int64_t)d * d;
  int64_t blocks = (dd + 7) / 8;  // one warp per entry
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  gda_cov_finish_kernel<<<(int)blocks, 256, 0, s>>>(part, d, n, nsplit, sigma, ctl);
  return cudaGetLastError();
}

}  // namespace km
