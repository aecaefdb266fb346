// Device helpers of the exact re-check (km_recheck.cu, km_batched.cu).
//
// A flagged point is settled by compensated FP32 distances
//   D_j = sum_t (x_t - c_jt)^2
// (each difference and square rounded once: <= 3u per term; the lanes' sums
// merged across the warp with TwoSum: <= u). Within a lane the terms are added
// with Kahan compensation (the all-centroid path: <= 2u, D_j within about 5u
// D_j of the exact value, u = 2^-24) or, for the short lists, by pairwise trees
// of at most 16 terms (depth <= 4: <= 4u), two of them joined exactly by TwoSum
// when d > 128: within 8u D_j. Either way two distances whose relative gap is
// at least 1e-6 (> 16u = 9.5e-7) are always ordered correctly; equal computed
// distances go to the lower index.
//
// When the assignment stage could not narrow the candidates (more than seven
// within its margin, or an FP32 SIMT flag), the re-check first screens all k
// centroids with plain FP32 scores s_j = h_j - x.c_j. With H = max h_j,
// Cmax >= max ||c_j|| and nx >= ||x||, every computed score is within
//   E = 3u H + gamma_{d+1} nx Cmax,   gamma_m = m u / (1 - m u),
// of its exact value (the bound of the FP32 assignment stage), so the true
// nearest centroid is among {j : s_j <= min_j s_j + 2E}. Each lane keeps its
// three best scores; when no lane's third is inside that window the window's
// members (at most two per lane) are the complete candidate list and only they
// get compensated distances. Otherwise every centroid does.
#pragma once

#include "km_internal.cuh"

namespace km {

// Compensated squared distance of x (lane slice xv) to one centroid, reduced
// across the warp with TwoSum; every lane returns the same value.
template <int V>
__device__ __forceinline__ float warp_sqdist(const float (&xv)[V], const float* __restrict__ c, int d, int lane) {
  float s = 0.f, comp = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int t = v * 32 + lane;
    if (t < d) {
      const float diff = __fsub_rn(xv[v], c[t]);
      kahan_add(s, comp, __fmul_rn(diff, diff));
    }
  }
  float hi = s, lo = -comp;  // lane value s - comp as a (hi, lo) pair
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
    const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
    float sh, e;
    two_sum(hi, ohi, sh, e);
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
    hi = sh;
  }
  return __fadd_rn(hi, lo);
}

// Settles one point in a group of G lanes (G a power of two, the group
// aligned to G lanes; sub = lane % G) between nc >= 1 candidates (indices
// cand[0..nc), any order), d <= 4 G F. Lane sub holds coordinates 4 (f G + sub)
// .. + 3 for f < F (a group's loads cover 16 G contiguous bytes) of the point
// in registers; the candidates are taken NQ at a time (four, or two when the
// slices are long), all their slices loaded before any arithmetic, so a short
// list costs about one round trip to memory per NQ candidates. For every coordinate the difference and its
// square are rounded once each; a lane's 4F squares are added by pairwise
// trees of at most 16 (depth <= 4), two of them joined exactly by TwoSum when
// F > 4 (error ~8u of the sum in all), and the G lane sums are combined with
// TwoSum. ncw = the largest nc
// over the warp (the loop bound, so that every lane takes part in the
// shuffles). Equal distances go to the lower index. Every lane of the group
// returns the same index.
template <int G, int F, int NQ = (F <= 4 ? 4 : 2)>
__device__ __forceinline__ int group_settle(const float* __restrict__ x, const float* __restrict__ C, int d, int nc,
                                            int ncw, const int (&cand)[kMaxCand], int sub) {
  const bool vec = (d & 3) == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(C)) & 15) == 0;
  auto load4 = [&](const float* p, int t, bool ok) -> float4 {
    if (!ok || t >= d) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec) return __ldg(reinterpret_cast<const float4*>(p + t));
    return make_float4(__ldg(p + t), t + 1 < d ? __ldg(p + t + 1) : 0.f, t + 2 < d ? __ldg(p + t + 2) : 0.f,
                       t + 3 < d ? __ldg(p + t + 3) : 0.f);
  };
  float4 xv[F];
#pragma unroll
  for (int f = 0; f < F; ++f) xv[f] = load4(x, 4 * (f * G + sub), true);
  float best = INFINITY;
  int jb = cand[0];
  for (int q0 = 0; q0 < ncw; q0 += NQ) {
    int jq[NQ];
    float4 cv[NQ][F];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      jq[u] = cand[0];
#pragma unroll
      for (int a = 0; a < kMaxCand; ++a)
        if (a == q0 + u) jq[u] = cand[a];
      const float* c = C + (int64_t)jq[u] * d;
#pragma unroll
      for (int f = 0; f < F; ++f) cv[u][f] = load4(c, 4 * (f * G + sub), q0 + u < nc);
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      // the lane's squares: one pairwise tree of depth <= 4 over f < 4 (at most 16
      // squares, error <= 4u of that part) and, for F > 4, a second over f >= 4,
      // the two added exactly by TwoSum; the lane's sum as (hi, lo)
      float part[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const float a = __fsub_rn(xv[f].x, cv[u][f].x), b = __fsub_rn(xv[f].y, cv[u][f].y);
        const float c = __fsub_rn(xv[f].z, cv[u][f].z), e = __fsub_rn(xv[f].w, cv[u][f].w);
        part[f] = __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fadd_rn(__fmul_rn(c, c), __fmul_rn(e, e)));
      }
      auto tree = [&](int f0, int m) {  // m = 1 .. 4 partials from f0
        if (m == 1) return part[f0];
        if (m == 2) return __fadd_rn(part[f0], part[f0 + 1]);
        if (m == 3) return __fadd_rn(__fadd_rn(part[f0], part[f0 + 1]), part[f0 + 2]);
        return __fadd_rn(__fadd_rn(part[f0], part[f0 + 1]), __fadd_rn(part[f0 + 2], part[f0 + 3]));
      };
      float hi, lo = 0.f;
      if constexpr (F <= 4) {
        hi = tree(0, F);
      } else {
        static_assert(F <= 8, "at most two trees of 16 squares per lane");
        two_sum(tree(0, 4), tree(4, F - 4), hi, lo);
      }
#pragma unroll
      for (int o = G >> 1; o; o >>= 1) {
        const float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        const float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, ohi, sh, e);
        lo = __fadd_rn(__fadd_rn(lo, olo), e);
        hi = sh;
      }
      const float D = __fadd_rn(hi, lo);
      if (q0 + u < nc && (D < best || (D == best && jq[u] < jb))) {  // equal distances: the lower index
        best = D;
        jb = jq[u];
      }
    }
  }
  return jb;
}

// Index of the n-th (0-based) set bit of m, or -1.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  for (int i = 0; i < n && m; ++i) m &= m - 1;
  return m ? __ffs(m) - 1 : -1;
}

// Keeps a lane's three smallest (score, index) pairs; indices arrive in
// increasing order, so strict comparisons keep the lower index first.
struct Top3 {
  float v0, v1, v2;
  int j0, j1, j2;
  __device__ __forceinline__ void init() {
    v0 = v1 = v2 = INFINITY;
    j0 = j1 = j2 = -1;
  }
  __device__ __forceinline__ void add(float v, int j) {
    if (v < v2) {
      if (v < v1) {
        v2 = v1;
        j2 = j1;
        if (v < v0) {
          v1 = v0;
          j1 = j0;
          v0 = v;
          j0 = j;
        } else {
          v1 = v;
          j1 = j;
        }
      } else {
        v2 = v;
        j2 = j;
      }
    }
  }
};

// Index of the nearest centroid of x among all k (same value on every lane).
// xv: the lane's slice of x (x_t at t = 32 v + lane); xsh: 32 V floats of
// shared memory private to the warp; h: h_j = RN(||c_j||^2 / 2); H, Cmax: the
// step's maxima of h_j and ||c_j||.
template <int V>
__device__ int nearest_all(const float (&xv)[V], float* xsh, const float* __restrict__ C,
                           const float* __restrict__ h, int k, int d, int lane, float H, float Cmax) {
  float sxx = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    xsh[v * 32 + lane] = xv[v];
    sxx = fmaf(xv[v], xv[v], sxx);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
  __syncwarp();
  // ||x|| rounded up: the sum of d squares has relative error below gamma_d
  const float kUf = 0x1p-24f;
  const float gd = (float)d * kUf / (1.f - (float)d * kUf);
  const float nx = __fmul_ru(__fsqrt_ru(__fmul_ru(sxx, 1.f + gd)), 1.f + 2.f * kUf);
  const float g = (float)(d + 1) * kUf / (1.f - (float)(d + 1) * kUf);
  const float E = __fadd_ru(__fmul_ru(3.f * kUf, H), __fmul_ru(__fmul_ru(g, nx), Cmax));
  const float margin = __fmul_ru(2.f * E, 1.f + 0x1p-10f);

  // screen: plain FP32 scores, lanes over centroids
  Top3 t3;
  t3.init();
  const bool vec4 = (d & 3) == 0 && ((uintptr_t)C & 15) == 0;  // centroid rows on 16-byte boundaries
  for (int j = lane; j < k; j += 32) {
    const float* c = C + (int64_t)j * d;
    float dot = 0.f;
    if (vec4) {
      for (int t = 0; t < d; t += 4) {
        const float4 cv = __ldg(reinterpret_cast<const float4*>(c + t));
        dot = fmaf(xsh[t], cv.x, dot);
        dot = fmaf(xsh[t + 1], cv.y, dot);
        dot = fmaf(xsh[t + 2], cv.z, dot);
        dot = fmaf(xsh[t + 3], cv.w, dot);
      }
    } else {
      for (int t = 0; t < d; ++t) dot = fmaf(xsh[t], __ldg(c + t), dot);
    }
    t3.add(__fsub_rn(__ldg(h + j), dot), j);
  }
  float mn = t3.v0;
#pragma unroll
  for (int o = 16; o; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  const float lim = __fadd_ru(mn, margin);
  const bool overflow = __any_sync(0xffffffffu, t3.v2 <= lim) || !(lim < INFINITY);

  float best = INFINITY;
  int jb = k;
  if (!overflow) {
    // compensated distances of the window's members
    unsigned m0 = __ballot_sync(0xffffffffu, t3.v0 <= lim);
    const unsigned m1 = __ballot_sync(0xffffffffu, t3.v1 <= lim);
    for (int pass = 0; pass < 2; ++pass) {
      unsigned m = pass ? m1 : m0;
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const int j = __shfl_sync(0xffffffffu, pass ? t3.j1 : t3.j0, src);
        const float D = warp_sqdist<V>(xv, C + (int64_t)j * d, d, lane);
        if (lex_less(D, j, best, jb)) {
          best = D;
          jb = j;
        }
      }
    }
  } else {
    // every centroid, lanes over centroids (x from shared memory)
    for (int j = lane; j < k; j += 32) {
      const float* c = C + (int64_t)j * d;
      float s = 0.f, comp = 0.f;
      for (int t = 0; t < d; ++t) {
        const float diff = __fsub_rn(xsh[t], __ldg(c + t));
        kahan_add(s, comp, __fmul_rn(diff, diff));
      }
      const float D = __fsub_rn(s, comp);
      if (D < best) {  // this lane's centroids arrive in increasing index order
        best = D;
        jb = j;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, jb, o);
      if (lex_less(ob, oj, best, jb)) {
        best = ob;
        jb = oj;
      }
    }
  }
  __syncwarp();
  return jb >= k ? 0 : jb;  // k: every distance was NaN
}

}  // namespace km
