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

// Rows of X a warp of the point quantisation loads at once (their loads in
// flight together). The kernels take V = lane slices of one code row
// (Kp <= 32 V, a power of two up to kMaxD / 32), so that a row of d <= 128
// holds no registers for the columns it does not have.
constexpr int kQU = 4;

// xv[u][v] = x[i0 + u][v 32 + lane] (0 past d or past the last row).
template <int V>
__device__ __forceinline__ void load_rows(const float* __restrict__ X, int64_t n, int d, int64_t i0, int lane,
                                          float (&xv)[kQU][V]) {
#pragma unroll
  for (int u = 0; u < kQU; ++u) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = v * 32 + lane;
      xv[u][v] = (i0 + u < n && t < d) ? __ldg(X + (i0 + u) * d + t) : 0.f;
    }
  }
}

// Xh (E4M3 with -h_j folded into the contraction; null otherwise): row i's
// [1/s_i, 1/s_i, 1/s_i, 0, ...] slice (store_row_slice).
// mu (null: no centring): the codes and statistics are those of the centred
// rows (km_quant.cuh); xnorm[i] gets the bound of the uncentred ||x_i|| (the
// FP32 consumers: re-check screen, deterministic grid).
template <int FP8, int V>
__global__ void __launch_bounds__(256, V <= 4 ? 4 : 2)
quant_x_kernel(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ Xq,
               float4* __restrict__ xs, uint4* __restrict__ Xh, const float* __restrict__ mu,
               float* __restrict__ xnorm, Ctl* ctl) {
  static_assert(kQU == 4, "four rows of four statistics: one 16-value reduce-scatter");
  constexpr int ESZ = FP8 ? 1 : 2;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ float mus[kMaxD];
  stage_mu(mus, mu, d);
  for (int64_t i0 = warp * kQU; i0 < n; i0 += nwarps * kQU) {
    float xv[kQU][V];
    load_rows(X, n, d, i0, lane, xv);
    float red[4 * kQU];  // row u's lane partials of sum v^2, sum v~^2, sum (v~ - v)^2, sum x^2 at 4 u + s
    float scs[kQU];
#pragma unroll
    for (int u = 0; u < kQU; ++u) {
      const int64_t i = i0 + u;
      float amax = 0.f;
      if (FP8)
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (v * 32 + lane < d) amax = fmaxf(amax, fabsf(__fsub_rn(xv[u][v], mus[v * 32 + lane])));
      const float sc = FP8 ? pow2_scale(warp_max(amax)) : 1.f;
      const float inv = FP8 ? pow2_inv(sc) : 1.f;
      float sxx = 0.f, sqq = 0.f, sdd = 0.f, sraw = 0.f;
      if (i < n) {
        uint8_t* row = Xq + i * (int64_t)Kp * ESZ;
#pragma unroll
        for (int sl = 0; sl < V; ++sl) {
          const int t = sl * 32 + lane;
          if (t >= Kp) break;
          const float xt = xv[u][sl];
          const float v = t < d ? __fsub_rn(xt, mus[t]) : 0.f;
          const float vq = quantise<FP8>(v, sc, inv, row + t * ESZ);
          const float r = vq - v;
          sxx = fmaf(v, v, sxx);
          sqq = fmaf(vq, vq, sqq);
          sdd = fmaf(r, r, sdd);
          sraw = fmaf(xt, xt, sraw);
        }
      }
      red[4 * u] = sxx;
      red[4 * u + 1] = sqq;
      red[4 * u + 2] = sdd;
      red[4 * u + 3] = sraw;
      scs[u] = sc;
    }
    // lane l holds statistic (l >> 1) & 3 of row l >> 3; its bound, then the row's four in lane 8 u
    const float tot = warp_reduce_scatter<16>(red, lane);
    const float nb = norm_bound(tot, d);
    const float nb1 = __shfl_down_sync(0xffffffffu, nb, 2), nb2 = __shfl_down_sync(0xffffffffu, nb, 4);
    const float nb3 = __shfl_down_sync(0xffffffffu, nb, 6);
    const float t1 = __shfl_down_sync(0xffffffffu, tot, 2), t3 = __shfl_down_sync(0xffffffffu, tot, 6);
    const int u = lane >> 3;
    const int64_t i = i0 + u;
    if ((lane & 7) == 0 && i < n) {
      const float sc = u == 0 ? scs[0] : (u == 1 ? scs[1] : (u == 2 ? scs[2] : scs[3]));
      if (!isfinite(tot) || !isfinite(t1) || !isfinite(t3)) ctl->nonfinite = 1;
      xs[i] = make_float4(sc, nb1, centred_resid(nb, nb2, mu), centred_norm(nb, mu));
      if (xnorm) xnorm[i] = nb3;
      if (FP8 && Xh) store_row_slice(Xh + 2 * i, sc);
    }
  }
}

// Two-part BF16 codes (split_bf16): row i holds hi in columns [0, Kp) and lo
// in [Kp, 2 Kp). Statistics: (1, ||hi|| + ||lo||, ||v - hi - lo||, ||v||),
// norms rounded up.
template <int V>
__global__ void __launch_bounds__(256, V <= 2 ? 4 : (V <= 4 ? 3 : 2))
quant_x_split_kernel(const float* __restrict__ X, int64_t n, int d, int Kp, uint8_t* __restrict__ Xq,
                     float4* __restrict__ xs, const float* __restrict__ mu, float* __restrict__ xnorm, Ctl* ctl) {
  static_assert(kQU == 4, "four rows of eight (five used) statistics: one 32-value reduce-scatter");
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ float mus[kMaxD];
  stage_mu(mus, mu, d);
  for (int64_t i0 = warp * kQU; i0 < n; i0 += nwarps * kQU) {
    float xv[kQU][V];
    load_rows(X, n, d, i0, lane, xv);
    float red[8 * kQU];  // row u's lane partials at 8 u + s: sum v^2, hi^2, lo^2, (v - hi - lo)^2, x^2
#pragma unroll
    for (int u = 0; u < kQU; ++u) {
      const int64_t i = i0 + u;
      float sxx = 0.f, shh = 0.f, sll = 0.f, sdd = 0.f, sraw = 0.f;
      if (i < n) {
        __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(Xq) + i * 2 * (int64_t)Kp;
#pragma unroll
        for (int sl = 0; sl < V; ++sl) {
          const int t = sl * 32 + lane;
          if (t >= Kp) break;
          const float xt = xv[u][sl];
          const float v = t < d ? __fsub_rn(xt, mus[t]) : 0.f;
          float hi, lo;
          const float r = split_bf16(v, row + t, row + Kp + t, hi, lo);
          sxx = fmaf(v, v, sxx);
          shh = fmaf(hi, hi, shh);
          sll = fmaf(lo, lo, sll);
          sdd = fmaf(r, r, sdd);
          sraw = fmaf(xt, xt, sraw);
        }
      }
      red[8 * u] = sxx;
      red[8 * u + 1] = shh;
      red[8 * u + 2] = sll;
      red[8 * u + 3] = sdd;
      red[8 * u + 4] = sraw;
      red[8 * u + 5] = 0.f;
      red[8 * u + 6] = 0.f;
      red[8 * u + 7] = 0.f;
    }
    // lane l holds statistic l & 7 of row l >> 3; its bound, then the row's five in lane 8 u
    const float tot = warp_reduce_scatter<32>(red, lane);
    const float nb = norm_bound(tot, d);
    float nbs[5], tots[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
      nbs[s] = __shfl_down_sync(0xffffffffu, nb, s);
      tots[s] = __shfl_down_sync(0xffffffffu, tot, s);
    }
    const int64_t i = i0 + (lane >> 3);
    if ((lane & 7) == 0 && i < n) {
      if (!isfinite(tots[0]) || !isfinite(tots[1]) || !isfinite(tots[4])) ctl->nonfinite = 1;
      const float nbv = nbs[0];
      xs[i] = make_float4(1.f, __fadd_ru(nbs[1], nbs[2]), centred_resid(nbv, nbs[3], mu), centred_norm(nbv, mu));
      if (xnorm) xnorm[i] = nbs[4];
    }
  }
}

// BF16 codes and statistics for a cold first step, plus the E4M3 row scale and
// statistics the later E4M3 steps use (their codes are written by the reduce
// stage in sorted order).
template <int V>
__global__ void __launch_bounds__(256, V <= 4 ? 4 : 2)
quant_x_dual_kernel(const float* __restrict__ X, int64_t n, int d, int Kp16, uint8_t* __restrict__ Xq,
                    float4* __restrict__ xs16, float4* __restrict__ xs8, const float* __restrict__ mu,
                    float* __restrict__ xnorm, Ctl* ctl) {
  static_assert(kQU == 4, "four rows of eight (six used) statistics: one 32-value reduce-scatter");
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  __shared__ float mus[kMaxD];
  stage_mu(mus, mu, d);
  for (int64_t i0 = warp * kQU; i0 < n; i0 += nwarps * kQU) {
    float xv[kQU][V];
    load_rows(X, n, d, i0, lane, xv);
    // row u's lane partials at 8 u + s: sum v^2, BF16 sum q^2 and (q - v)^2, E4M3 the same, sum x^2
    float red[8 * kQU];
    float scs[kQU];
#pragma unroll
    for (int u = 0; u < kQU; ++u) {
      const int64_t i = i0 + u;
      float amax = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (v * 32 + lane < d) amax = fmaxf(amax, fabsf(__fsub_rn(xv[u][v], mus[v * 32 + lane])));
      const float sc8 = pow2_scale(warp_max(amax));
      const float inv8 = pow2_inv(sc8);
      float sxx = 0.f, sqq16 = 0.f, sdd16 = 0.f, sqq8 = 0.f, sdd8 = 0.f, sraw = 0.f;
      if (i < n) {
        uint8_t* row = Xq + i * (int64_t)Kp16 * 2;
#pragma unroll
        for (int sl = 0; sl < V; ++sl) {
          const int t = sl * 32 + lane;
          if (t >= Kp16) break;
          const float xt = xv[u][sl];
          sraw = fmaf(xt, xt, sraw);
          const float v = t < d ? __fsub_rn(xt, mus[t]) : 0.f;
          const float q16 = quantise<0>(v, 1.f, 1.f, row + t * 2);
          uint8_t dummy;
          const float q8 = quantise<1>(v, sc8, inv8, &dummy);
          sxx = fmaf(v, v, sxx);
          sqq16 = fmaf(q16, q16, sqq16);
          sdd16 = fmaf(q16 - v, q16 - v, sdd16);
          sqq8 = fmaf(q8, q8, sqq8);
          sdd8 = fmaf(q8 - v, q8 - v, sdd8);
        }
      }
      red[8 * u] = sxx;
      red[8 * u + 1] = sqq16;
      red[8 * u + 2] = sdd16;
      red[8 * u + 3] = sqq8;
      red[8 * u + 4] = sdd8;
      red[8 * u + 5] = sraw;
      red[8 * u + 6] = 0.f;
      red[8 * u + 7] = 0.f;
      scs[u] = sc8;
    }
    // lane l holds statistic l & 7 of row l >> 3; its bound, then the row's six in lane 8 u
    const float tot = warp_reduce_scatter<32>(red, lane);
    const float nb = norm_bound(tot, d);
    float nbs[6], tots[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      nbs[s] = __shfl_down_sync(0xffffffffu, nb, s);
      tots[s] = __shfl_down_sync(0xffffffffu, tot, s);
    }
    const int u = lane >> 3;
    const int64_t i = i0 + u;
    if ((lane & 7) == 0 && i < n) {
      const float sc8 = u == 0 ? scs[0] : (u == 1 ? scs[1] : (u == 2 ? scs[2] : scs[3]));
      if (!isfinite(tots[0]) || !isfinite(tots[1]) || !isfinite(tots[3]) || !isfinite(tots[5])) ctl->nonfinite = 1;
      const float nbv = nbs[0], xn = centred_norm(nbv, mu);
      xs16[i] = make_float4(1.f, nbs[1], centred_resid(nbv, nbs[2], mu), xn);
      xs8[i] = make_float4(sc8, nbs[3], centred_resid(nbv, nbs[4], mu), xn);
      if (xnorm) xnorm[i] = nbs[5];
    }
  }
}

// max_{j,t} |c_jt| of the step's centroids into ctl->camax_bits.
__global__ void __launch_bounds__(256) camax_kernel(const float* __restrict__ C, int64_t kd, int d,
                                                    const float* __restrict__ mu, Ctl* ctl) {
  if (halted(ctl)) return;
  __shared__ float mus[kMaxD];
  stage_mu(mus, mu, d);
  float m = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(mu ? __fsub_rn(C[e], mus[e % d]) : C[e]));
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
// mu (null: no centring): codes, h_j (hq, Hc), cst and the maxima hmax_c /
// cmax_c / qcmax / dcmax are those of c_j - mu (h_j from the exact FP64
// differences); chalf[j] (j < k) and hmax / cmax keep the uncentred h_j and
// ||c_j|| bound for the FP32 consumers (re-check screen, deterministic grid).
template <int MODE>
__global__ void __launch_bounds__(256)
quant_c_kernel(const float* __restrict__ C, int k, int kp, int d, int Kp, uint8_t* __restrict__ Cq,
               __nv_bfloat16* __restrict__ Hc, float* __restrict__ hq, float* __restrict__ scq,
               float4* __restrict__ cst, const float* __restrict__ mu, float* __restrict__ chalf,
               int32_t* __restrict__ counts, Ctl* ctl, int stats16) {
  constexpr int FP8 = MODE == 1;
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int W = MODE == 2 ? 2 : 1;  // code parts per element
  if (halted(ctl)) return;
  const bool fold = MODE != 2 && Hc != nullptr;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  __shared__ float mus[kMaxD];
  stage_mu(mus, mu, d);
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
    double s2 = 0.0, s2r = 0.0;  // ||c_j - mu||^2 (exact differences), ||c_j||^2
    for (int t = lane; t < d; t += 32) {
      const double e = (double)c[t] - (double)mus[t];
      s2 = fma(e, e, s2);
      s2r = fma((double)c[t], (double)c[t], s2r);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      s2r += __shfl_xor_sync(0xffffffffu, s2r, o);
    }
    const float sc = FP8 ? pow2_scale(__uint_as_float(ctl->camax_bits)) : 1.f;  // one scale for all centroids
    const float inv = FP8 ? pow2_inv(sc) : 1.f;
    float sqq = 0.f, sll = 0.f, sdd = 0.f, svv = 0.f;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? __fsub_rn(c[t], mus[t]) : 0.f;
      svv = fmaf(v, v, svv);
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
    svv = warp_sum(svv);
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
      const float hr = __double2float_rn(0.5 * s2r);
      const float cnr = __double2float_ru(sqrt(s2r) * (1.0 + 1e-13));
      const float qn = MODE == 2 ? __fadd_ru(norm_bound(sqq, d), norm_bound(sll, d)) : norm_bound(sqq, d);
      const float dn = centred_resid(norm_bound(svv, d), norm_bound(sdd, d), mu);
      if (!isfinite(h) || !isfinite(cn) || !isfinite(qn) || !isfinite(hr) || !isfinite(cnr)) ctl->nonfinite = 1;
      hq[j] = h;
      scq[j] = sc;
      cst[j] = make_float4(h, qn, cn, dn);
      chalf[j] = hr;
      if (counts) counts[j] = 0;
      atomic_max_nonneg(&ctl->hmax_bits, hr);
      atomic_max_nonneg(&ctl->cmax_bits, cnr);
      atomic_max_nonneg(&ctl->hmax_c_bits, h);
      atomic_max_nonneg(&ctl->cmax_c_bits, cn);
      if (h >= 0.f && h < INFINITY) atomicMax(&ctl->hmin_neg, 0x7f800000u - __float_as_uint(h));
      atomic_max_nonneg(stats16 ? &ctl->qcmax16_bits : &ctl->qcmax_bits, qn);
      atomic_max_nonneg(stats16 ? &ctl->dcmax16_bits : &ctl->dcmax_bits, dn);
    }
  }
}

constexpr int kCentreThreads = 512;

// The centring vector of a call (one block): mu_t = the mean of column t of
// the call's initial centroids, kept only when it pays -- when the centred
// centroids' largest norm is at most half the uncentred one (a common offset of
// the data dominates its spread); otherwise mu = 0 (the codes of x itself).
// Any fixed vector keeps every distance, so mu need not be the exact mean: FP32
// sums in a fixed order (per warp over its rows, then the warps in order) make
// it a deterministic function of C at FP32 speed.
__global__ void __launch_bounds__(kCentreThreads) centre_kernel(const float* __restrict__ C, int k, int d,
                                                                float* __restrict__ mu) {
  constexpr int NW = kCentreThreads / 32, V = kMaxD / 32;
  __shared__ float part[NW][kMaxD];  // per-warp column sums, added in warp order
  __shared__ float mus[kMaxD];
  __shared__ float mx[2][NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.f;
  for (int j = warp; j < k; j += NW) {  // warp w: rows w, w + NW, ...; lane: columns lane + 32 v
    const float* c = C + (int64_t)j * d;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = v * 32 + lane;
      if (t < d) acc[v] += __ldg(c + t);
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) part[warp][v * 32 + lane] = acc[v];
  __syncthreads();
  for (int t = tid; t < d; t += kCentreThreads) {
    float s = 0.f;
    for (int w = 0; w < NW; ++w) s += part[w][t];
    mus[t] = s / (float)k;
  }
  __syncthreads();
  float m0 = 0.f, m1 = 0.f;  // max_j ||c_j||^2, max_j ||c_j - mu||^2
  for (int j = warp; j < k; j += NW) {
    const float* c = C + (int64_t)j * d;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = v * 32 + lane;
      if (t < d) {
        const float x = __ldg(c + t), e = x - mus[t];
        a = fmaf(x, x, a);
        b = fmaf(e, e, b);
      }
    }
    a = warp_sum(a);
    b = warp_sum(b);
    m0 = fmaxf(m0, a);
    m1 = fmaxf(m1, b);
  }
  if (lane == 0) {
    mx[0][warp] = m0;
    mx[1][warp] = m1;
  }
  __syncthreads();
  float M0 = mx[0][0], M1 = mx[1][0];
  for (int w = 1; w < NW; ++w) {
    M0 = fmaxf(M0, mx[0][w]);
    M1 = fmaxf(M1, mx[1][w]);
  }
  const bool keep = M1 <= 0.25f * M0;
  for (int t = tid; t < d; t += kCentreThreads) mu[t] = keep ? mus[t] : 0.f;
}

}  // namespace

cudaError_t launch_centre(const Problem& p, const Work& w, cudaStream_t s) {
  if (!w.mu) return cudaSuccess;
  centre_kernel<<<1, kCentreThreads, 0, s>>>(p.C, p.k, p.d, w.mu);
  return cudaGetLastError();
}

// Blocks of the point quantisation: one warp per kQU rows, at most 16 blocks per SM.
int quant_x_blocks(int64_t n) {
  int64_t blocks = (n + 8 * kQU - 1) / (8 * kQU);
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  return (int)(blocks > 0 ? blocks : 1);
}

template <int V>
void launch_quant_x_v(const Problem& p, const Work& w, int mode, int Kp, uint8_t* Xq, float4* xs, cudaStream_t s) {
  const int blocks = quant_x_blocks(p.n);
  uint4* xh = reinterpret_cast<uint4*>(w.Xh);
  if (mode == 2) quant_x_split_kernel<V><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, w.mu, w.xnorm, w.ctl);
  else if (mode == 1)
    quant_x_kernel<1, V><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, xh, w.mu, w.xnorm, w.ctl);
  else quant_x_kernel<0, V><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp, Xq, xs, nullptr, w.mu, w.xnorm, w.ctl);
}

// Lane slices of a code row of Kp columns (a power of two, d <= Kp <= kMaxD).
int quant_slices(int Kp) {
  const int v = (Kp + 31) / 32;
  return v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : 8;
}

cudaError_t launch_quant_x(const Problem& p, const Work& w, int mode, int Kp, uint8_t* Xq, float4* xs,
                           cudaStream_t s) {
  switch (quant_slices(Kp)) {
    case 1: launch_quant_x_v<1>(p, w, mode, Kp, Xq, xs, s); break;
    case 2: launch_quant_x_v<2>(p, w, mode, Kp, Xq, xs, s); break;
    case 4: launch_quant_x_v<4>(p, w, mode, Kp, Xq, xs, s); break;
    default: launch_quant_x_v<8>(p, w, mode, Kp, Xq, xs, s); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_quant_x_dual(const Problem& p, const Work& w, int Kp16, uint8_t* Xq, float4* xs16, float4* xs8,
                                cudaStream_t s) {
  const int blocks = quant_x_blocks(p.n);
  switch (quant_slices(Kp16)) {
    case 1: quant_x_dual_kernel<1><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp16, Xq, xs16, xs8, w.mu, w.xnorm, w.ctl); break;
    case 2: quant_x_dual_kernel<2><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp16, Xq, xs16, xs8, w.mu, w.xnorm, w.ctl); break;
    case 4: quant_x_dual_kernel<4><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp16, Xq, xs16, xs8, w.mu, w.xnorm, w.ctl); break;
    default:
      quant_x_dual_kernel<8><<<blocks, 256, 0, s>>>(p.X, p.n, p.d, Kp16, Xq, xs16, xs8, w.mu, w.xnorm, w.ctl);
  }
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
    quant_c_kernel<2><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, w.mu, w.chalf, counts, w.ctl,
                                             stats16);
  } else if (mode == 1) {
    const int64_t kd = (int64_t)p.k * p.d;
    int mb = (int)((kd + 255) / 256);
    if (mb > num_sms() * 4) mb = num_sms() * 4;
    camax_kernel<<<mb, 256, 0, s>>>(p.C, kd, p.d, w.mu, w.ctl);
    quant_c_kernel<1><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, w.mu, w.chalf, counts, w.ctl,
                                             stats16);
  } else {
    quant_c_kernel<0><<<blocks, 256, 0, s>>>(p.C, p.k, kp, p.d, Kp, Cq, hc, h, sc, cst, w.mu, w.chalf, counts, w.ctl,
                                             stats16);
  }
  return cudaGetLastError();
}

}  // namespace km
