// Per-call and per-iteration preparation stages.
//
// Code motion (Sec. 3.1): everything that does not depend on the point being
// processed is computed once, outside the point loop -- the half squared norm
// h_j of every centroid, the centroid-norm maxima that size the error bound,
// and (once per call, since X does not change between iterations) an upper
// bound of every point norm.
#include "km_internal.cuh"

namespace km {

// ||x_i|| upper bound and the finiteness check of X. One warp per point.
// The squared norm is summed in FP32; every term is non-negative, so its
// relative error is below gamma_{d+1}, and sqrt halves it. The stored value is
// sqrt rounded up, scaled by (1 + (d + 8) u) and rounded up again.
__global__ void xnorm_kernel(const float* __restrict__ X, int64_t n, int d,
                             float* __restrict__ xnorm, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const float slack = 1.0f + (float)(d + 8) * kU;
  for (int64_t i = warp; i < n; i += nwarps) {
    const float* x = X + i * d;
    float s = 0.f;
    for (int t = lane; t < d; t += 32) s = fmaf(x[t], x[t], s);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (!isfinite(s)) ctl->nonfinite = 1;
      xnorm[i] = __fmul_ru(__fsqrt_ru(s), slack);
    }
  }
}

cudaError_t launch_xnorm(const Problem& p, const Work& w, cudaStream_t s) {
  int64_t warps_needed = p.n;
  int blocks = (int)((warps_needed + 7) / 8);
  int cap = num_sms() * 16;
  if (blocks > cap) blocks = cap;
  xnorm_kernel<<<blocks, 256, 0, s>>>(p.X, p.n, p.d, w.xnorm, w.ctl);
  return cudaGetLastError();
}

// Centroid preparation: h_j = RN32(||c_j||^2 / 2) from an FP64 norm,
// ||c_j|| rounded up, and their maxima over j. One warp per centroid.
// Also clears counts (the histogram of this iteration).
__global__ void prep_kernel(const float* __restrict__ C, int k, int d, float* __restrict__ chalf,
                            float* __restrict__ cnorm, int32_t* __restrict__ counts, Ctl* ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < k; j += nwarps) {
    const float* c = C + (int64_t)j * d;
    double s = 0.0;
    for (int t = lane; t < d; t += 32) s = fma((double)c[t], (double)c[t], s);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      float h = __double2float_rn(0.5 * s);
      float cn = __double2float_ru(sqrt(s) * (1.0 + 1e-13));  // covers the FP64 sum error
      if (!isfinite(h) || !isfinite(cn)) ctl->nonfinite = 1;
      chalf[j] = h;
      cnorm[j] = cn;
      counts[j] = 0;
      atomic_max_nonneg(&ctl->hmax_bits, h);
      atomic_max_nonneg(&ctl->cmax_bits, cn);
    }
  }
}

cudaError_t launch_prep(const Problem& p, const Work& w, cudaStream_t s) {
  int blocks = (p.k + 7) / 8;
  int cap = num_sms() * 8;
  if (blocks > cap) blocks = cap;
  prep_kernel<<<blocks, 256, 0, s>>>(p.C, p.k, p.d, w.chalf, w.cnorm, p.counts, w.ctl);
  return cudaGetLastError();
}

}  // namespace km
