// Quantisation stages of the tensor-core path.
//
// X is quantised once per call (it does not change between iterations, Sec.
// 3.1 code motion) and C once per step. Codes: BF16 round-to-nearest with
// scale 1, or E4M3 round-to-nearest, saturating, of v / s with a power-of-two
// row scale s = 2^ceil(log2(amax / 448)), so that v / s and s * code are exact.
// Every row also gets upper bounds of ||v~||, of the residual ||v~ - v|| (each
// residual v~_t - v_t is exact in FP32) and of ||v||, which size the
// assignment error bound. Codes are stored K-major with Kp >= d columns
// (zero padded) so that TMA boxes of 128 bytes tile them.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"

namespace km {

namespace {

__device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  const float m = frexpf(amax / 448.f, &e);  // amax / 448 = m 2^e, m in [0.5, 1)
  return ldexpf(1.f, m == 0.5f ? e - 1 : e);
}

// One quantised element: stores the code, returns the dequantised value.
template <int FP8>
__device__ __forceinline__ float quantise(float v, float sc, uint8_t* dst) {
  if constexpr (FP8) {
    __nv_fp8_e4m3 q(v / sc);  // RN, satfinite
    *dst = q.__x;
    return (float)q * sc;
  } else {
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(dst) = q;
    return __bfloat162float(q);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// sqrt of an FP32 sum of m non-negative terms, rounded up and widened to cover
// the sum's rounding (relative error < gamma_m).
__device__ __forceinline__ float norm_bound(float sumsq, int m) {
  return __fmul_ru(__fsqrt_ru(sumsq), 1.f + (float)(m + 8) * kU);
}

template <int FP8>
__global__ void __launch_bounds__(256)
quant_x_kernel(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ Xq,
               float4* __restrict__ xs, Ctl* ctl) {
  constexpr int ESZ = FP8 ? 1 : 2;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const float* x = X + i * d;
    float amax = 0.f;
    if (FP8)
      for (int t = lane; t < d; t += 32) amax = fmaxf(amax, fabsf(x[t]));
    const float sc = FP8 ? pow2_scale(warp_max(amax)) : 1.f;
    float sxx = 0.f, sqq = 0.f, sdd = 0.f;
    uint8_t* row = Xq + i * (int64_t)Kp * ESZ;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? x[t] : 0.f;
      const float vq = quantise<FP8>(v, sc, row + t * ESZ);
      const float r = vq - v;
      sxx = fmaf(v, v, sxx);
      sqq = fmaf(vq, vq, sqq);
      sdd = fmaf(r, r, sdd);
    }
    sxx = warp_sum(sxx);
    sqq = warp_sum(sqq);
    sdd = warp_sum(sdd);
    if (lane == 0) {
      if (!isfinite(sxx) || !isfinite(sqq)) ctl->nonfinite = 1;
      xs[i] = make_float4(sc, norm_bound(sqq, d), norm_bound(sdd, d), norm_bound(sxx, d));
    }
  }
}

template <int FP8>
__global__ void __launch_bounds__(256)
quant_c_kernel(const float* __restrict__ C, int k, int kp, int d, int Kp, uint8_t* __restrict__ Cq,
               float2* __restrict__ hsc, int32_t* __restrict__ counts, Ctl* ctl) {
  constexpr int ESZ = FP8 ? 1 : 2;
  if (ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < kp; j += nwarps) {
    uint8_t* row = Cq + (int64_t)j * Kp * ESZ;
    if (j >= k) {  // padding centroid: zero codes, score +inf
      for (int t = lane; t < Kp * ESZ; t += 32) row[t] = 0;
      if (lane == 0) hsc[j] = make_float2(INFINITY, 1.f);
      continue;
    }
    const float* c = C + (int64_t)j * d;
    double s2 = 0.0;
    float amax = 0.f;
    for (int t = lane; t < d; t += 32) {
      s2 = fma((double)c[t], (double)c[t], s2);
      amax = fmaxf(amax, fabsf(c[t]));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const float sc = FP8 ? pow2_scale(warp_max(amax)) : 1.f;
    float sqq = 0.f, sdd = 0.f;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? c[t] : 0.f;
      const float vq = quantise<FP8>(v, sc, row + t * ESZ);
      const float r = vq - v;
      sqq = fmaf(vq, vq, sqq);
      sdd = fmaf(r, r, sdd);
    }
    sqq = warp_sum(sqq);
    sdd = warp_sum(sdd);
    if (lane == 0) {
      const float h = __double2float_rn(0.5 * s2);
      const float cn = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
      const float qn = norm_bound(sqq, d), dn = norm_bound(sdd, d);
      if (!isfinite(h) || !isfinite(cn) || !isfinite(qn)) ctl->nonfinite = 1;
      hsc[j] = make_float2(h, sc);
      counts[j] = 0;
      atomic_max_nonneg(&ctl->hmax_bits, h);
      atomic_max_nonneg(&ctl->cmax_bits, cn);
      atomic_max_nonneg(&ctl->qcmax_bits, qn);
      atomic_max_nonneg(&ctl->dcmax_bits, dn);
    }
  }
}

}  // namespace

cudaError_t launch_quant_x(const Problem& p, const Work& w, int fp8, int Kp, uint8_t* Xq, float4* xs,
                           cudaStream_t s) {
  int64_t blocks = (p.n + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (fp8) quant_x_kernel<1><<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, w.ctl);
  else quant_x_kernel<0><<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_quant_c(const Problem& p, const Work& w, int fp8, int kp, int Kp, uint8_t* Cq, float2* hsc,
                           cudaStream_t s) {
  int blocks = (kp + 7) / 8;
  const int cap = num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (fp8) quant_c_kernel<1><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hsc, p.counts, w.ctl);
  else quant_c_kernel<0><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hsc, p.counts, w.ctl);
  return cudaGetLastError();
}

}  // namespace km
