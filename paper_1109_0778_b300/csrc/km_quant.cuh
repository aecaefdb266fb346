// Device helpers of the quantisation stages (single-instance and batched):
// power-of-two row scales, one quantised element, warp reductions, and norm
// upper bounds. See km_quant.cu for the scheme.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"

namespace km {

// Centring of the quantised paths: the codes are those of v = RN(x - mu_t)
// (mu null: v = x), a translation that leaves every distance unchanged. The
// rounding leaves |v - (x - mu_t)| <= kEu |v| (kEu >= u / (1 - u)), which the
// row statistics add to the residual bound: ||v~ - (x - mu)|| <= ||v~ - v|| +
// kEu ||v||, ||x - mu|| <= (1 + kEu) ||v||.
constexpr float kEu = 0x1.000002p-24f;
static __device__ __forceinline__ float centred(float x, const float* __restrict__ mu, int t) {
  return mu ? __fsub_rn(x, __ldg(mu + t)) : x;
}
// Stages the centring vector in shared memory, zeros without one (x - 0 = x
// exactly); every thread of the block calls it.
static __device__ __forceinline__ void stage_mu(float* mus, const float* __restrict__ mu, int d) {
  for (int t = threadIdx.x; t < d; t += blockDim.x) mus[t] = mu ? __ldg(mu + t) : 0.f;
  __syncthreads();
}
// Residual and norm bounds of a centred row from nb(sum v^2) and nb(sum (v~ - v)^2).
static __device__ __forceinline__ float centred_resid(float nbv, float nbd, bool c) {
  return c ? __fmaf_ru(kEu, nbv, nbd) : nbd;
}
static __device__ __forceinline__ float centred_norm(float nbv, bool c) { return c ? __fmul_ru(nbv, 1.f + kEu) : nbv; }

static __device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  int e;
  const float m = frexpf(amax / 448.f, &e);  // amax / 448 = m 2^e, m in [0.5, 1)
  e = m == 0.5f ? e - 1 : e;
  return ldexpf(1.f, e < -126 ? -126 : e);  // a normal power of two: its reciprocal is exact
}

// 1 / sc for a scale from pow2_scale: exact, so v * pow2_inv(sc) == v / sc.
static __device__ __forceinline__ float pow2_inv(float sc) { return __frcp_rn(sc); }

// One quantised element: stores the code, returns the dequantised value.
template <int FP8>
static __device__ __forceinline__ float quantise(float v, float sc, float inv, uint8_t* dst) {
  if constexpr (FP8) {
    __nv_fp8_e4m3 q(v * inv);  // RN, satfinite; inv = 1 / sc exactly
    *dst = q.__x;
    return (float)q * sc;
  } else {
    const __nv_bfloat16 q = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(dst) = q;
    return __bfloat162float(q);
  }
}

// Two-part BF16 split of v: hi = RN(v), lo = RN(v - hi), stored at hi_dst and
// lo_dst. v - hi and v - hi - lo are exact in FP32 (each operand pair is
// within a factor of two, Sterbenz). lo is kept only while |lo| <= u (1 + u)
// |hi| with u = 2^-8, which holds for every normal hi; otherwise (subnormal
// hi) lo = 0 and the residual carries the difference. Returns the residual
// v - hi - lo; hi and lo come back as floats.
static __device__ __forceinline__ float split_bf16(float v, __nv_bfloat16* hi_dst, __nv_bfloat16* lo_dst, float& hi,
                                                   float& lo) {
  const __nv_bfloat16 qh = __float2bfloat16_rn(v);
  hi = __bfloat162float(qh);
  const float r1 = v - hi;
  __nv_bfloat16 ql = __float2bfloat16_rn(r1);
  lo = __bfloat162float(ql);
  if (!(fabsf(lo) <= fabsf(hi) * (0x1p-8f + 0x1p-16f))) {  // exact product: a power-of-two sum times hi
    ql = __float2bfloat16_rn(0.f);
    lo = 0.f;
  }
  *hi_dst = qh;
  *lo_dst = ql;
  return r1 - lo;
}

// The per-row slice of a folded E4M3 contraction: BF16 [1/s, 1/s, 1/s, 0 x 13]
// (1/s exact: s is a power of two), two 16-byte words of a 32-byte row.
static __device__ __forceinline__ void store_row_slice(uint4* dst, float s) {
  const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(__frcp_rn(s)));
  dst[0] = make_uint4(b | (b << 16), b, 0u, 0u);
  dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

static __device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

static __device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Reduce-scatter over the warp: v[0..NV) (NV = 16 or 32) summed over the 32
// lanes; lane l returns the total of value l >> 1 (NV = 16; lanes l and l ^ 1
// hold the same total) or l (NV = 32). Each level sends half of the remaining
// values to the partner lane and keeps the other half, so NV values cost NV - 1
// shuffles instead of 5 NV. (Any summation tree gives the norm bounds their
// guarantee: a sum of m non-negative terms has relative error < gamma_m.)
template <int NV>
static __device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane) {
#pragma unroll
  for (int o = 16, c = NV; c > 1; o >>= 1, c >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < c / 2; ++i) {
      const float send = up ? v[i] : v[i + c / 2];
      const float keep = up ? v[i + c / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  if (NV == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}

// sqrt of an FP32 sum of m non-negative terms, rounded up and widened to cover
// the sum's rounding (relative error < gamma_m).
static __device__ __forceinline__ float norm_bound(float sumsq, int m) {
  return __fmul_ru(__fsqrt_ru(sumsq), 1.f + (float)(m + 8) * kU);
}


}  // namespace km
