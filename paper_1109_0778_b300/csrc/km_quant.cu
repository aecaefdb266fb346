// Quantisation stages of the tensor-core path.
//
// Code modes: 0 BF16, 1 E4M3, 2 two-part BF16 (split_bf16; rows of 2 Kp
// codes, hi then lo).
//
// X is quantised once per call (it does not change between iterations, Sec.
// 3.1 code motion) and C once per step. Codes: BF16 round-to-nearest with
// scale 1, or E4M3 round-to-nearest, saturating, of v / s with a power-of-two
// scale s = 2^ceil(log2(amax / 448)), so that v / s and s * code are exact:
// one scale per point row (amax over the row), and one for all centroids of
// the step (amax over C), so that a score needs a single per-row factor.
// Every row also gets upper bounds of ||v~||, of the residual ||v~ - v|| (each
// residual v~_t - v_t is exact in FP32) and of ||v||, which size the
// assignment error bound. Codes are stored K-major with Kp >= d columns
// (zero padded) so that TMA boxes of 128 bytes tile them.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"
#include "km_quant.cuh"

namespace km {

namespace {

// Xh (E4M3 with -h_j folded into the contraction; null otherwise): row i's
// [1/s_i, 1/s_i, 1/s_i, 0, ...] slice (store_row_slice).
template <int FP8>
__global__ void __launch_bounds__(256)
quant_x_kernel(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ Xq,
               float4* __restrict__ xs, uint4* __restrict__ Xh, Ctl* ctl) {
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
    const float inv = FP8 ? pow2_inv(sc) : 1.f;
    float sxx = 0.f, sqq = 0.f, sdd = 0.f;
    uint8_t* row = Xq + i * (int64_t)Kp * ESZ;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? x[t] : 0.f;
      const float vq = quantise<FP8>(v, sc, inv, row + t * ESZ);
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
      if (FP8 && Xh) store_row_slice(Xh + 2 * i, sc);
    }
  }
}

// Two-part BF16 codes (split_bf16): row i holds hi in columns [0, Kp) and lo
// in [Kp, 2 Kp). Statistics: (1, ||hi|| + ||lo||, ||v - hi - lo||, ||v||),
// norms rounded up.
__global__ void __launch_bounds__(256)
quant_x_split_kernel(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ Xq,
                     float4* __restrict__ xs, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const float* x = X + i * d;
    float sxx = 0.f, shh = 0.f, sll = 0.f, sdd = 0.f;
    __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(Xq) + i * 2 * (int64_t)Kp;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? x[t] : 0.f;
      float hi, lo;
      const float r = split_bf16(v, row + t, row + Kp + t, hi, lo);
      sxx = fmaf(v, v, sxx);
      shh = fmaf(hi, hi, shh);
      sll = fmaf(lo, lo, sll);
      sdd = fmaf(r, r, sdd);
    }
    sxx = warp_sum(sxx);
    shh = warp_sum(shh);
    sll = warp_sum(sll);
    sdd = warp_sum(sdd);
    if (lane == 0) {
      if (!isfinite(sxx) || !isfinite(shh)) ctl->nonfinite = 1;
      xs[i] = make_float4(1.f, __fadd_ru(norm_bound(shh, d), norm_bound(sll, d)), norm_bound(sdd, d),
                          norm_bound(sxx, d));
    }
  }
}

// BF16 codes and statistics for a cold first step, plus the E4M3 row scale and
// statistics the later E4M3 steps use (their codes are written by the reduce
// stage in sorted order).
__global__ void __launch_bounds__(256)
quant_x_dual_kernel(const float* __restrict__ X, int64_t n, int d, int Kp16, uint8_t* __restrict__ Xq,
                    float4* __restrict__ xs16, float4* __restrict__ xs8, Ctl* ctl) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const float* x = X + i * d;
    float amax = 0.f;
    for (int t = lane; t < d; t += 32) amax = fmaxf(amax, fabsf(x[t]));
    const float sc8 = pow2_scale(warp_max(amax));
    const float inv8 = pow2_inv(sc8);
    float sxx = 0.f, sqq16 = 0.f, sdd16 = 0.f, sqq8 = 0.f, sdd8 = 0.f;
    uint8_t* row = Xq + i * (int64_t)Kp16 * 2;
    for (int t = lane; t < Kp16; t += 32) {
      const float v = t < d ? x[t] : 0.f;
      const float q16 = quantise<0>(v, 1.f, 1.f, row + t * 2);
      uint8_t dummy;
      const float q8 = quantise<1>(v, sc8, inv8, &dummy);
      sxx = fmaf(v, v, sxx);
      sqq16 = fmaf(q16, q16, sqq16);
      sdd16 = fmaf(q16 - v, q16 - v, sdd16);
      sqq8 = fmaf(q8, q8, sqq8);
      sdd8 = fmaf(q8 - v, q8 - v, sdd8);
    }
    sxx = warp_sum(sxx);
    sqq16 = warp_sum(sqq16);
    sdd16 = warp_sum(sdd16);
    sqq8 = warp_sum(sqq8);
    sdd8 = warp_sum(sdd8);
    if (lane == 0) {
      if (!isfinite(sxx) || !isfinite(sqq16) || !isfinite(sqq8)) ctl->nonfinite = 1;
      const float xn = norm_bound(sxx, d);
      xs16[i] = make_float4(1.f, norm_bound(sqq16, d), norm_bound(sdd16, d), xn);
      xs8[i] = make_float4(sc8, norm_bound(sqq8, d), norm_bound(sdd8, d), xn);
    }
  }
}

// max_{j,t} |c_jt| of the step's centroids into ctl->camax_bits.
__global__ void __launch_bounds__(256) camax_kernel(const float* __restrict__ C, int64_t kd, Ctl* ctl) {
  if (halted(ctl)) return;
  float m = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(C[e]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomic_max_nonneg(&ctl->camax_bits, m);
}

// MODE 0: BF16, 1: E4M3, 2: two-part BF16 (hi in columns [0, Kp), lo in
// [Kp, 2 Kp); the code norm statistic is ||hi|| + ||lo||).
// Hc (BF16 "folded" scores; null otherwise): row j of the [kp][16] BF16 array
// holds -h_j as three BF16 parts (-h1, -h2, -h3; h1 = RN(h), h2 = RN(h - h1),
// h3 = RN(h - h1 - h2), each remainder exact by Sterbenz's lemma,
// |h - h1 - h2 - h3| <= 2^-27 h) and zeros, so that the contraction against a
// slice of ones yields x.c_j - h_j in the accumulator; a padding row holds
// -inf there (score +inf).
// cst[j] = (h_j, ||c~_j||, ||c_j||, ||c~_j - c_j||): the per-centroid terms of
// the assignment's error bound, the same values whose maxima the step records
// (h_j as the scores use it, the norms rounded up); zeros for padding rows.
template <int MODE>
__global__ void __launch_bounds__(256)
quant_c_kernel(const float* __restrict__ C, int k, int kp, int d, int Kp, uint8_t* __restrict__ Cq,
               __nv_bfloat16* __restrict__ Hc, float* __restrict__ hq, float* __restrict__ scq,
               float4* __restrict__ cst, int32_t* __restrict__ counts, Ctl* ctl, int stats16) {
  constexpr int FP8 = MODE == 1;
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int W = MODE == 2 ? 2 : 1;  // code parts per element
  if (halted(ctl)) return;
  const bool fold = MODE != 2 && Hc != nullptr;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < kp; j += nwarps) {
    uint8_t* row = Cq + (int64_t)j * W * Kp * ESZ;
    if (j >= k) {  // padding centroid: zero codes, score +inf
      for (int t = lane; t < W * Kp * ESZ; t += 32) row[t] = 0;
      if (fold && lane < 16) Hc[(int64_t)j * 16 + lane] = __float2bfloat16_rn(lane == 0 ? -INFINITY : 0.f);
      if (lane == 0) {
        hq[j] = INFINITY;
        scq[j] = 1.f;
        cst[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    const float* c = C + (int64_t)j * d;
    double s2 = 0.0;
    for (int t = lane; t < d; t += 32) s2 = fma((double)c[t], (double)c[t], s2);
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const float sc = FP8 ? pow2_scale(__uint_as_float(ctl->camax_bits)) : 1.f;  // one scale for all centroids
    const float inv = FP8 ? pow2_inv(sc) : 1.f;
    float sqq = 0.f, sll = 0.f, sdd = 0.f;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? c[t] : 0.f;
      if constexpr (MODE == 2) {
        __nv_bfloat16* r16 = reinterpret_cast<__nv_bfloat16*>(row);
        float hi, lo;
        const float r = split_bf16(v, r16 + t, r16 + Kp + t, hi, lo);
        sqq = fmaf(hi, hi, sqq);
        sll = fmaf(lo, lo, sll);
        sdd = fmaf(r, r, sdd);
      } else {
        const float vq = quantise<FP8>(v, sc, inv, row + t * ESZ);
        const float r = vq - v;
        sqq = fmaf(vq, vq, sqq);
        sdd = fmaf(r, r, sdd);
      }
    }
    sqq = warp_sum(sqq);
    if (MODE == 2) sll = warp_sum(sll);
    sdd = warp_sum(sdd);
    if (fold) {  // -h_j (E4M3: -h_j / s_c, exact) as three BF16 parts (every lane computes h alike)
      const float h = __double2float_rn(0.5 * s2) * inv;
      const __nv_bfloat16 h1 = __float2bfloat16_rn(h);
      const float r1 = h - __bfloat162float(h1);
      const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(h2);
      const __nv_bfloat16 h3 = __float2bfloat16_rn(r2);
      if (lane < 16)
        Hc[(int64_t)j * 16 + lane] =
            lane == 0 ? __hneg(h1) : lane == 1 ? __hneg(h2) : lane == 2 ? __hneg(h3) : __float2bfloat16_rn(0.f);
    }
    if (lane == 0) {
      const float h = __double2float_rn(0.5 * s2);
      const float cn = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
      const float qn = MODE == 2 ? __fadd_ru(norm_bound(sqq, d), norm_bound(sll, d)) : norm_bound(sqq, d);
      const float dn = norm_bound(sdd, d);
      if (!isfinite(h) || !isfinite(cn) || !isfinite(qn)) ctl->nonfinite = 1;
      hq[j] = h;
      scq[j] = sc;
      cst[j] = make_float4(h, qn, cn, dn);
      if (counts) counts[j] = 0;
      atomic_max_nonneg(&ctl->hmax_bits, h);
      if (h >= 0.f && h < INFINITY) atomicMax(&ctl->hmin_neg, 0x7f800000u - __float_as_uint(h));
      atomic_max_nonneg(&ctl->cmax_bits, cn);
      atomic_max_nonneg(stats16 ? &ctl->qcmax16_bits : &ctl->qcmax_bits, qn);
      atomic_max_nonneg(stats16 ? &ctl->dcmax16_bits : &ctl->dcmax_bits, dn);
    }
  }
}

}  // namespace

cudaError_t launch_quant_x(const Problem& p, const Work& w, int mode, int Kp, uint8_t* Xq, float4* xs,
                           cudaStream_t s) {
  int64_t blocks = (p.n + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  uint4* xh = reinterpret_cast<uint4*>(w.Xh);
  if (mode == 2) quant_x_split_kernel<<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, w.ctl);
  else if (mode == 1) quant_x_kernel<1><<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, xh, w.ctl);
  else quant_x_kernel<0><<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, nullptr, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_quant_x_dual(const Problem& p, const Work& w, int Kp16, uint8_t* Xq, float4* xs16, float4* xs8,
                                cudaStream_t s) {
  int64_t blocks = (p.n + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  quant_x_dual_kernel<<<(int)blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp16, Xq, xs16, xs8, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_quant_c(const Problem& p, const Work& w, int mode, int kp, int Kp, uint8_t* Cq, void* Hc, float* h,
                           float* sc, float4* cst, cudaStream_t s, bool stats16) {
  __nv_bfloat16* hc = mode != 2 ? reinterpret_cast<__nv_bfloat16*>(Hc) : nullptr;
  int32_t* counts = stats16 ? nullptr : p.counts;  // the re-check codes leave the counts alone
  int blocks = (kp + 7) / 8;
  const int cap = num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (mode == 2) {
    quant_c_kernel<2><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, counts, w.ctl, stats16);
  } else if (mode == 1) {
    const int64_t kd = (int64_t)p.k * p.d;
    int mb = (int)((kd + 255) / 256);
    if (mb > num_sms() * 4) mb = num_sms() * 4;
    camax_kernel<<<mb, 256, 0, s>>>(p.C, kd, w.ctl);
    quant_c_kernel<1><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, counts, w.ctl, stats16);
  } else {
    quant_c_kernel<0><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, counts, w.ctl, stats16);
  }
  return cudaGetLastError();
}

}  // namespace km
