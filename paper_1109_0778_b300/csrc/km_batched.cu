// Batched Lloyd steps: many independent instances (each with its own n, d, k)
// advance together, one launch per stage for the whole batch.
//
// Every per-instance array lives at an offset in one flattened array of the
// batch workspace; a stage walks the flattened rows (or centroids, or tiles)
// and finds the instance of an element by binary search over the offsets. A
// finished instance (its stop rule fired) is skipped element by element. The
// arithmetic of each stage is the single-instance one (km_quant.cu,
// km_recheck.cu, km_reduce.cu): the same codes, error bounds, compensated
// sums and FP64 divide, so every instance gets the same accuracy contract.
#include "km_internal.cuh"
#include "km_quant.cuh"
#include "km_recheck.cuh"
#include "km_gather.cuh"
#include "km_scatter.cuh"

namespace km {

namespace {

constexpr int kMaxV = 4;   // d <= 128 in batched runs: 4 floats per lane

__global__ void b_reset_kernel(Ctl* ctls, int nb, unsigned long long* flag_slots) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *flag_slots = 0;
  if (b < nb) {
    unsigned int* w = reinterpret_cast<unsigned int*>(ctls + b);
    for (size_t e = 0; e < kCtlIterBytes / 4; ++e) w[e] = 0;
  }
}

// Copies every instance's centroids to (restore = 0) or from (restore = 1) the
// batch's saved copy, which holds instance b's k x d floats at its sums offset.
// Grid row y takes instances y, y + gridDim.y, ..., grid-strided over their floats.
__global__ void b_copy_c_kernel(const BInst* __restrict__ inst, int nb, float* __restrict__ csave, int restore) {
  for (int b = blockIdx.y; b < nb; b += gridDim.y) {
    const BInst& I = inst[b];
    const int64_t m = (int64_t)I.k * I.d;
    float* save = csave + I.sum_off;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
      if (restore) I.C[e] = save[e];
      else save[e] = I.C[e];
    }
  }
}

// Sum and maximum over the DP lanes of an aligned lane group (DP a power of two).
template <int DP>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = DP >> 1; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int DP>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
  for (int o = DP >> 1; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Codes and statistics of flattened rows [p, pend) of instance q with Kp <= 32 V:
// four rows at a time with their loads in flight together, lanes over the code
// columns. (Warp-uniform.)
template <int FP8, int V>
__device__ __forceinline__ void bq_rows(const BWork& W, int q, int64_t p, int64_t pend, int lane) {
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int U = 4;
  const BInst& I = W.inst[q];
  const int d = I.d, Kp = I.Kp;
  for (; p < pend; p += U) {
    const int64_t i0 = p - I.row_off;
    const int rows = (int)min((int64_t)U, pend - p);
    float xv[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float* x = I.X + (i0 + u) * d;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int t = v * 32 + lane;
        xv[u][v] = (u < rows && t < d) ? x[t] : 0.f;
      }
    }
    float red[4 * U];  // row u's lane partials at 4 u + s: sum x^2, sum x~^2, sum (x~ - x)^2, 0
    float scs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float amax = 0.f;
      if (FP8) {
#pragma unroll
        for (int v = 0; v < V; ++v) amax = fmaxf(amax, fabsf(xv[u][v]));
      }
      const float sc = FP8 ? pow2_scale(warp_max(amax)) : 1.f;
      const float inv = FP8 ? pow2_inv(sc) : 1.f;
      float sxx = 0.f, sqq = 0.f, sdd = 0.f;
      if (u < rows) {
        uint8_t* row = W.Xq + I.xq_off + (i0 + u) * (int64_t)Kp * ESZ;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int t = v * 32 + lane;
          if (t < Kp) {
            const float xt = xv[u][v];
            const float vq = quantise<FP8>(xt, sc, inv, row + t * ESZ);
            sxx = fmaf(xt, xt, sxx);
            sqq = fmaf(vq, vq, sqq);
            sdd = fmaf(vq - xt, vq - xt, sdd);
          }
        }
      }
      red[4 * u] = sxx;
      red[4 * u + 1] = sqq;
      red[4 * u + 2] = sdd;
      red[4 * u + 3] = 0.f;
      scs[u] = sc;
    }
    // lane l holds statistic (l >> 1) & 3 of row l >> 3 (warp_reduce_scatter); the row's lane 8 u stores
    const float tot = warp_reduce_scatter<16>(red, lane);
    const float nb = norm_bound(tot, d);
    const float nb1 = __shfl_down_sync(0xffffffffu, nb, 2), nb2 = __shfl_down_sync(0xffffffffu, nb, 4);
    const float t1 = __shfl_down_sync(0xffffffffu, tot, 2);
    const int u = lane >> 3;
    if ((lane & 7) == 0 && u < rows) {
      const float sc = u == 0 ? scs[0] : (u == 1 ? scs[1] : (u == 2 ? scs[2] : scs[3]));
      if (!isfinite(tot) || !isfinite(t1)) W.ctls[q].nonfinite = 1;
      W.xs[p + u] = make_float4(sc, nb1, nb2, nb);
    }
  }
}

// The same for rows of d <= DP <= 16 (DP a power of two): a group of DP lanes
// per row, 32 / DP rows per warp step, four steps with their loads in flight
// together; lane s of a group holds coordinate s and writes code columns s,
// s + DP, ... < Kp (zero past d). (Warp-uniform.)
template <int FP8, int DP>
__device__ __forceinline__ void bq_packed(const BWork& W, int q, int64_t p, int64_t pend, int lane) {
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int RPW = 32 / DP, U = 4;
  const BInst& I = W.inst[q];
  const int d = I.d, Kp = I.Kp;
  const int g = lane / DP, s = lane % DP;
  for (; p < pend; p += RPW * U) {
    float xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t pr = p + u * RPW + g;
      xv[u] = (pr < pend && s < d) ? I.X[(pr - I.row_off) * d + s] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t pr = p + u * RPW + g;
      const bool live = pr < pend;
      const float sc = FP8 ? pow2_scale(group_max<DP>(fabsf(xv[u]))) : 1.f;
      const float inv = FP8 ? pow2_inv(sc) : 1.f;
      float sxx = 0.f, sqq = 0.f, sdd = 0.f;
      if (live) {
        uint8_t* row = W.Xq + I.xq_off + (pr - I.row_off) * (int64_t)Kp * ESZ;
        for (int t = s; t < Kp; t += DP) {
          const float xt = t == s ? xv[u] : 0.f;
          const float vq = quantise<FP8>(xt, sc, inv, row + t * ESZ);
          sxx = fmaf(xt, xt, sxx);
          sqq = fmaf(vq, vq, sqq);
          sdd = fmaf(vq - xt, vq - xt, sdd);
        }
      }
      sxx = group_sum<DP>(sxx);
      sqq = group_sum<DP>(sqq);
      sdd = group_sum<DP>(sdd);
      if (live && s == 0) {
        if (!isfinite(sxx) || !isfinite(sqq)) W.ctls[q].nonfinite = 1;
        W.xs[pr] = make_float4(sc, norm_bound(sqq, d), norm_bound(sdd, d), norm_bound(sxx, d));
      }
    }
  }
}

// Codes and row statistics of every point of the batch. Each warp walks one
// contiguous range of the flattened rows (instances found by walking forward
// from one search), each instance's part with the row loop for its width.
template <int FP8>
__global__ void __launch_bounds__(256) b_quant_x_kernel(BWork W) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t P0 = W.R * gw / nw, P1 = W.R * (gw + 1) / nw;
  int q = P0 < P1 ? find_block(W.row_off, W.nb, P0) : 0;
  for (int64_t p = P0; p < P1;) {
    while (W.row_off[q + 1] <= p) ++q;
    const int64_t pend = min(W.row_off[q + 1], P1);
    const int d = W.inst[q].d, Kp = W.inst[q].Kp;
    if (d <= 1) bq_packed<FP8, 1>(W, q, p, pend, lane);
    else if (d <= 2) bq_packed<FP8, 2>(W, q, p, pend, lane);
    else if (d <= 4) bq_packed<FP8, 4>(W, q, p, pend, lane);
    else if (d <= 8) bq_packed<FP8, 8>(W, q, p, pend, lane);
    else if (d <= 16) bq_packed<FP8, 16>(W, q, p, pend, lane);
    else if (Kp <= 32) bq_rows<FP8, 1>(W, q, p, pend, lane);
    else if (Kp <= 64) bq_rows<FP8, 2>(W, q, p, pend, lane);
    else bq_rows<FP8, kMaxV>(W, q, p, pend, lane);
    p = pend;
  }
}

// max_{j,t} |c_jt| of every instance (one block per instance) for its E4M3 centroid scale.
__global__ void __launch_bounds__(256) b_camax_kernel(BWork W) {
  const int b = blockIdx.x;
  if (halted(W.ctls + b)) return;
  const BInst& I = W.inst[b];
  const int64_t kd = (int64_t)I.k * I.d;
  float m = 0.f;
  for (int64_t e = threadIdx.x; e < kd; e += blockDim.x) m = fmaxf(m, fabsf(I.C[e]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomic_max_nonneg(&W.ctls[b].camax_bits, m);
}

template <int FP8>
__global__ void __launch_bounds__(256) b_quant_c_kernel(BWork W) {
  constexpr int ESZ = FP8 ? 1 : 2;
  const int lane = threadIdx.x & 31;
  // one warp per padded centroid; its instance from the table
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < W.KP;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int b = __ldg(W.kp_inst + g);
    Ctl* ctl = W.ctls + b;
    if (halted(ctl)) continue;
    const BInst& I = W.inst[b];
    const int j = (int)(g - I.kp_off);
    const int d = I.d, Kp = I.Kp;
    uint8_t* row = W.Cq + I.cq_off + (int64_t)j * Kp * ESZ;
    if (j >= I.k) {  // padding centroid: zero codes, score +inf
      for (int t = lane; t < Kp * ESZ; t += 32) row[t] = 0;
      if (lane == 0) {
        W.hq[g] = INFINITY;
        W.scq[g] = 1.f;
        W.cst[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      continue;
    }
    const float* c = I.C + (int64_t)j * d;
    double s2 = 0.0;
    for (int t = lane; t < d; t += 32) s2 = fma((double)c[t], (double)c[t], s2);
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const float sc = FP8 ? pow2_scale(__uint_as_float(ctl->camax_bits)) : 1.f;  // one scale per instance
    const float inv = FP8 ? pow2_inv(sc) : 1.f;
    float sqq = 0.f, sdd = 0.f;
    for (int t = lane; t < Kp; t += 32) {
      const float v = t < d ? c[t] : 0.f;
      const float vq = quantise<FP8>(v, sc, inv, row + t * ESZ);
      sqq = fmaf(vq, vq, sqq);
      sdd = fmaf(vq - v, vq - v, sdd);
    }
    sqq = warp_sum(sqq);
    sdd = warp_sum(sdd);
    if (lane == 0) {
      const float h = __double2float_rn(0.5 * s2);
      const float cn = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
      const float qn = norm_bound(sqq, d), dn = norm_bound(sdd, d);
      if (!isfinite(h) || !isfinite(cn) || !isfinite(qn)) ctl->nonfinite = 1;
      W.hq[g] = h;
      W.scq[g] = sc;
      W.cst[g] = make_float4(h, qn, cn, dn);
      I.counts[j] = 0;
      atomic_max_nonneg(&ctl->hmax_bits, h);
      if (h >= 0.f && h < INFINITY) atomicMax(&ctl->hmin_neg, 0x7f800000u - __float_as_uint(h));
      atomic_max_nonneg(&ctl->cmax_bits, cn);
      atomic_max_nonneg(&ctl->hmax_c_bits, h);  // (batched codes are not centred)
      atomic_max_nonneg(&ctl->cmax_c_bits, cn);
      atomic_max_nonneg(&ctl->qcmax_bits, qn);
      atomic_max_nonneg(&ctl->dcmax_bits, dn);
    }
  }
}

// Flagged points of all instances (FlagRec.pad = instance): the re-check of
// km_recheck.cu with lanes over dimensions (d <= 128).
// Settles one flagged point of instance I with V = ceil(d / 32) registers per lane.
template <int V>
__device__ __forceinline__ int b_settle(const BWork& W, const FlagRec& rec, const BInst& I, int b, float* xsh,
                                        int lane) {
  const int d = I.d, k = I.k;
  const float* x = I.X + (int64_t)rec.i * d;
  float xv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int t = v * 32 + lane;
    xv[v] = t < d ? x[t] : 0.f;
  }
  if (rec.nc > 0) {
    float best = INFINITY;
    int jb = rec.cand[0];
    for (int q = 0; q < rec.nc; ++q) {
      const int j = rec.cand[q];
      const float D = warp_sqdist<V>(xv, I.C + (int64_t)j * d, d, lane);
      if (D < best || (D == best && j < jb)) {  // equal distances: the lower index
        best = D;
        jb = j;
      }
    }
    return jb;
  }
  return nearest_all<V>(xv, xsh, I.C, W.hq + I.kp_off, k, d, lane, __uint_as_float(W.ctls[b].hmax_bits),
                        __uint_as_float(W.ctls[b].cmax_bits));
}

// Short candidate lists: groups of G lanes per point (group_settle), 32 / G
// points at a time; 8 lanes with one float4 slice each for d <= 32, four slices
// (d <= 128) above. (Narrower groups for small d measured slower: 0.74 -> 0.83 ms.)
// A round's candidate loop runs to its longest list, so the lists of at most
// two candidates (one load round) are settled first, among themselves.
template <int G, int F>
__device__ __forceinline__ void b_settle_short(const BWork& W, unsigned sl, const FlagRec& r, int lane) {
  const int g = lane / G, sub = lane % G;
  const unsigned sm1 = __ballot_sync(0xffffffffu, ((sl >> lane) & 1u) && r.nc <= 2);
  for (int pass = 0; pass < 2; ++pass) {
  unsigned sm = pass ? sl & ~sm1 : sm1;
  while (sm) {  // warp-uniform
    const int src = nth_set_bit(sm, g);
    const int from = src < 0 ? __ffs(sm) - 1 : src;  // (a group without a point repeats the first one)
    const int ri = __shfl_sync(0xffffffffu, r.i, from), rnc = __shfl_sync(0xffffffffu, r.nc, from);
    const int rold = __shfl_sync(0xffffffffu, r.old, from), b = __shfl_sync(0xffffffffu, r.pad, from);
    int cand[kMaxCand];
#pragma unroll
    for (int a = 0; a < kMaxCand; ++a) cand[a] = __shfl_sync(0xffffffffu, r.cand[a], from);
    const BInst& I = W.inst[b];
    const int ncw = __reduce_max_sync(0xffffffffu, src >= 0 ? rnc : 0);
    const int jb = group_settle<G, F, 2>(I.X + (int64_t)ri * I.d, I.C, I.d, rnc, ncw, cand, sub);
    if (src >= 0 && sub == 0) {
      I.assign[ri] = jb;
      if (rold != jb) atomicAdd(&W.ctls[b].n_changed, 1ull);
    }
    for (int a = 0; a < 32 / G && sm; ++a) sm &= sm - 1;  // the points of this round
  }
  }
}

// A warp takes 32 flags at a time (nwarps apart); lane l loads flag l's record.
// Short lists go to b_settle_short, the points to check against all k are
// settled one at a time by the whole warp (b_settle).
__global__ void __launch_bounds__(256, 3) b_recheck_kernel(BWork W) {
  __shared__ __align__(16) float xs_all[8][kMaxV * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* xsh = xs_all[wib];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const int64_t nflag = min((int64_t)*W.flag_slots, W.R);
  for (int64_t f0 = warp; f0 < nflag; f0 += nwarps * 32) {
    const int64_t fl = f0 + lane * nwarps;
    bool have = fl < nflag;
    FlagRec r;
    r.i = 0;
    r.nc = 0;
    r.old = -1;
    r.pad = 0;
#pragma unroll
    for (int a = 0; a < kMaxCand; ++a) r.cand[a] = 0;
    int d = 0;
    if (have) {
      r = W.flags[fl];
      have = !halted(W.ctls + r.pad);
      d = W.inst[r.pad].d;
    }
    const bool shortl = have && r.nc > 0;
    b_settle_short<8, 1>(W, __ballot_sync(0xffffffffu, shortl && d <= 32), r, lane);
    b_settle_short<8, 4>(W, __ballot_sync(0xffffffffu, shortl && d > 32), r, lane);  // d <= 128
    unsigned todo = __ballot_sync(0xffffffffu, have && !shortl);
    while (todo) {
      const int l = __ffs(todo) - 1;
      todo &= todo - 1;
      const FlagRec rec = W.flags[f0 + l * nwarps];
      const int b = rec.pad;
      const BInst& I = W.inst[b];
      const int jb = I.d <= 32 ? b_settle<1>(W, rec, I, b, xsh, lane)
                               : (I.d <= 64 ? b_settle<2>(W, rec, I, b, xsh, lane)
                                            : b_settle<kMaxV>(W, rec, I, b, xsh, lane));
      if (lane == 0) {
        I.assign[rec.i] = jb;
        if (rec.old != jb) atomicAdd(&W.ctls[b].n_changed, 1ull);
      }
    }
  }
}

// Counts per cluster: each block takes whole row chunks (one instance each),
// counts them in a shared-memory histogram and adds its nonzero bins to the
// instance's counts; instances with more than kBHistMax clusters add warp-
// aggregated global atomics instead.
__global__ void __launch_bounds__(256) b_count_kernel(BWork W) {
  extern __shared__ int hist[];
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < W.nrchunks; c += gridDim.x) {
    const BChunk ch = W.rchunks[c];
    if (halted(W.ctls + ch.b)) continue;  // block-uniform
    const BInst& I = W.inst[ch.b];
    const int k = I.k;
    const int32_t* a = I.assign + (ch.r0 - I.row_off);
    if (k <= kBHistMax) {
      for (int j = threadIdx.x; j < k; j += blockDim.x) hist[j] = 0;
      __syncthreads();
      for (int r = threadIdx.x; r < ch.n; r += blockDim.x) atomicAdd(&hist[__ldg(a + r)], 1);
      __syncthreads();
      for (int j = threadIdx.x; j < k; j += blockDim.x)
        if (hist[j]) atomicAdd(&I.counts[j], hist[j]);
      __syncthreads();
    } else {
      for (int r0 = 0; r0 < ch.n; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        const bool act = r < ch.n;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (act) {
          const int j = __ldg(a + r);
          const unsigned peers = __match_any_sync(m, j);
          if (lane == __ffs(peers) - 1) atomicAdd(&I.counts[j], __popc(peers));
        }
      }
    }
  }
}

// Exclusive scan of one instance's counts per block (k <= 1024 * 64).
__global__ void __launch_bounds__(1024) b_scan_kernel(BWork W) {
  const int b = blockIdx.x;
  if (halted(W.ctls + b)) return;
  const BInst& I = W.inst[b];
  __shared__ int warp_tot[32];
  __shared__ int carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < I.k; base += 1024) {
    const int j = base + threadIdx.x;
    const int v = j < I.k ? I.counts[j] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int excl = carry_s + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (j < I.k) {
      W.offs[I.offs_off + j] = excl;
      W.cursor[I.kp_off + j] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) W.offs[I.offs_off + I.k] = carry_s;
}

// Cluster-sorted order of every instance: each block takes whole row chunks,
// ranks a chunk's points per cluster with shared-memory atomics, reserves one
// range per (chunk, cluster) in the instance's cursors and writes its points
// there (the order within a cluster varies from run to run). Instances with
// more than kBHistMax clusters reserve per warp-aggregated group instead.
constexpr int kBScatterPer = kBRowChunk / 256;  // rows per thread of a chunk
static_assert(kBRowChunk == kScatterChunk, "a row chunk is one sorted-write scatter chunk");

__global__ void __launch_bounds__(256) b_scatter_kernel(BWork W) {
  extern __shared__ int cnt[];  // per-cluster count, then the chunk's base position
  __shared__ int wsum[8];
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < W.nrchunks; c += gridDim.x) {
    const BChunk ch = W.rchunks[c];
    if (halted(W.ctls + ch.b)) continue;  // block-uniform
    const BInst& I = W.inst[ch.b];
    const int k = I.k;
    const int64_t i0 = ch.r0 - I.row_off;  // the chunk's first point within its instance
    const int32_t* a = I.assign + i0;
    int32_t* cur = W.cursor + I.kp_off;
    int32_t* perm = W.perm + I.row_off;
    int32_t* slab = W.lab_sorted + I.row_off;
    if (W.kmax <= kSortedScatterMax) {  // (the launch gave the sorted write's shared memory)
      scatter_chunk_sorted(a, ch.n, i0, k, cur, perm, slab, cnt, wsum);
    } else if (k <= kBHistMax) {
      for (int j = threadIdx.x; j < k; j += blockDim.x) cnt[j] = 0;
      __syncthreads();
      int lab[kBScatterPer], rank[kBScatterPer];
#pragma unroll
      for (int q = 0; q < kBScatterPer; ++q) {
        const int r = q * 256 + threadIdx.x;
        lab[q] = r < ch.n ? __ldg(a + r) : -1;
        rank[q] = lab[q] >= 0 ? atomicAdd(&cnt[lab[q]], 1) : 0;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < k; j += blockDim.x)
        if (cnt[j]) cnt[j] = atomicAdd(&cur[j], cnt[j]);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kBScatterPer; ++q) {
        if (lab[q] >= 0) {
          const int pos = cnt[lab[q]] + rank[q];
          perm[pos] = (int32_t)(i0 + q * 256 + threadIdx.x);
          slab[pos] = lab[q];
        }
      }
      __syncthreads();
    } else {
      for (int r0 = 0; r0 < ch.n; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        const bool act = r < ch.n;
        const unsigned m = __ballot_sync(0xffffffffu, act);
        if (act) {
          const int j = __ldg(a + r);
          const unsigned peers = __match_any_sync(m, j);
          const int leader = __ffs(peers) - 1;
          int pos = 0;
          if (lane == leader) pos = atomicAdd(&cur[j], __popc(peers));
          pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1));
          perm[pos] = (int32_t)(i0 + r);
          slab[pos] = j;
        }
      }
    }
  }
}

// Cluster-sorted copies for the instances whose tiles run in that order
// (gsort: k spans several chunks, where a tile of one previous cluster keeps
// its candidate tracking cheap): sorted row p of the copy holds the codes of
// point perm[p], and the row statistics go to xs_sorted[p]. A warp copies
// 32 / (row bytes / 16) rows per step, a lane one 16-byte piece of a row, and
// takes kPermU steps at a time (their index loads, then their row loads, in
// flight together).
constexpr int kPermU = 8;

__global__ void __launch_bounds__(256) b_permute_kernel(BWork W) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < W.nrchunks; c += gridDim.x) {
    const BChunk ch = W.rchunks[c];
    const BInst& I = W.inst[ch.b];
    if (!I.gsort || halted(W.ctls + ch.b)) continue;  // block-uniform
    const int pieces = (I.nkb * I.rowb) >> 4;  // 16-byte pieces of a code row: 2, 4, 8 or 16
    const int rpw = 32 / pieces, q = lane % pieces;
    const int64_t p0 = ch.r0 - I.row_off;  // sorted position of the chunk's first row
    const int32_t* perm = W.perm + I.row_off;
    const float4* xs = W.xs + I.row_off;
    float4* xss = W.xs_sorted + I.row_off;
    const uint4* src = reinterpret_cast<const uint4*>(W.Xq + I.xq_off);
    uint4* dst = reinterpret_cast<uint4*>(W.Xqs + I.xqs_off);
    for (int r0 = wib * rpw * kPermU + lane / pieces; r0 < ch.n; r0 += 8 * rpw * kPermU) {
      int idx[kPermU];
#pragma unroll
      for (int u = 0; u < kPermU; ++u) {
        const int r = r0 + u * rpw;
        idx[u] = r < ch.n ? __ldg(perm + p0 + r) : -1;
      }
      uint4 v[kPermU];
      float4 st[kPermU];
#pragma unroll
      for (int u = 0; u < kPermU; ++u) {
        if (idx[u] >= 0) {
          v[u] = __ldg(src + (int64_t)idx[u] * pieces + q);
          if (q == 0) st[u] = __ldg(xs + idx[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kPermU; ++u) {
        if (idx[u] >= 0) {
          const int64_t p = p0 + r0 + u * rpw;
          dst[p * pieces + q] = v[u];
          if (q == 0) xss[p] = st[u];
        }
      }
    }
  }
}

// Segmented sums over the cluster-sorted positions of every instance. The
// work items are host-built chunks of one instance's sorted positions (about
// 96 KB of X each, a table as for the count and scatter), which warps take in
// turn; within an item the instance and its row width are fixed, so the row
// loop is specialised for V = ceil(d / 32) slices per lane, or packs 32 / dp
// rows per warp step for d <= 16 (dp the power of two >= d). Rows are gathered
// into shared memory with cp.async one batch ahead (their indices two batches
// ahead), as in km_reduce.cu; each run of a cluster is summed in Kahan FP32 per
// coordinate and added to the FP64 sums with one atomic per coordinate, and
// the objective terms ||x_i - c_j||^2 of the item go to the instance's control
// block with one atomic.
constexpr int kSegStage = 768;                               // floats per stage (6 rows of 128, 24 of 32)
constexpr size_t kSegSmem = (size_t)8 * 2 * kSegStage * 4;   // 8 warps x 2 stages

// One item: sorted positions [it.r0, it.r0 + it.n) of instance it.b, V
// slices of 32 coordinates per lane (16 < d <= 32 V).
template <int V>
__device__ __forceinline__ void seg_item(const BWork& W, const BChunk& it, float* stage0, float* stage1, int lane) {
  constexpr int RB = kSegStage / (32 * V);  // rows per batch (a 3 KB stage)
  constexpr int rs = 32 * V;                           // stage floats per row
  constexpr bool BLK = V == 2 || V == 4;               // a lane owns V contiguous columns (vector loads)
  auto col = [&](int v) { return BLK ? lane * V + v : v * 32 + lane; };
  const BInst& I = W.inst[it.b];
  const int d = I.d;
  const float* __restrict__ X = I.X;
  const float* __restrict__ C = I.C;
  double* sums = W.sums64 + I.sum_off;
  const int32_t* perm = W.perm + it.r0;
  const int32_t* labs = W.lab_sorted + it.r0;
  const int nb = (it.n + RB - 1) / RB;
  auto meta = [&](int bt, int& i, int& j) {  // lane r < RB: row bt RB + r
    const int r = bt * RB + lane;
    i = 0;
    j = -1;
    if (lane < RB && r < it.n) {
      i = __ldg(perm + r);
      j = __ldg(labs + r);
    }
  };
  auto gather = [&](int bt, float* st, int i_lane) {
    gather_rows(st, rs, X, d, min(RB, it.n - bt * RB), (int64_t)i_lane * d, lane);
  };
  float s[V], c[V], cj[V];
#pragma unroll
  for (int v = 0; v < V; ++v) s[v] = c[v] = cj[v] = 0.f;
  float objS = 0.f, objC = 0.f;
  int cur = -1;  // the run being summed
  // this lane's partial sums of run cur into the FP64 sums
  auto flush = [&]() {
    if (cur < 0) return;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = col(v);
      if (t < d) atomicAdd(sums + (int64_t)cur * d + t, (double)s[v] - (double)c[v]);
      s[v] = c[v] = 0.f;
    }
  };
  // columns [d, 32 V) of every row slot hold zeros (the gathers write only
  // [0, d)), so rows are read without a column test
  if (d < rs) {
    for (int e = lane; e < RB * rs; e += 32)
      if (e % rs >= d) stage0[e] = stage1[e] = 0.f;
    __syncwarp();
  }
  // the objective terms are added plainly over RF rows (at most 8 terms per
  // lane: relative error <= 7u of the partial), each partial then Kahan-added
  constexpr int RF = V >= 8 ? 1 : 8 / V;
  float qacc = 0.f;
  int i_c = 0, j_c = -1, i_n = 0, j_n = -1;
  meta(0, i_c, j_c);
  gather(0, stage0, i_c);
  if (nb > 1) meta(1, i_n, j_n);
  for (int bt = 0; bt < nb; ++bt) {
    float* st = (bt & 1) ? stage1 : stage0;
    if (bt + 1 < nb) gather(bt + 1, (bt & 1) ? stage0 : stage1, i_n);
    int i_nn = 0, j_nn = -1;
    if (bt + 2 < nb) meta(bt + 2, i_nn, j_nn);
    if (bt + 1 < nb) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncwarp();
    const int rows = min(RB, it.n - bt * RB);
    {
      // rows that start a run (lane r holds row r's label), found once per batch
      const int jprev = __shfl_up_sync(0xffffffffu, j_c, 1);
      const unsigned starts = __ballot_sync(0xffffffffu, lane < rows && j_c != (lane == 0 ? cur : jprev));
      for (int r = 0; r < rows;) {
        if ((starts >> r) & 1u) {  // the same for every lane
          flush();
          cur = __shfl_sync(0xffffffffu, j_c, r);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int t = col(v);
            cj[v] = t < d ? C[(int64_t)cur * d + t] : 0.f;
          }
        }
        const unsigned later = starts & ~((2u << r) - 1u);  // run starts after row r
        const int rend = later ? __ffs(later) - 1 : rows;
        auto row = [&](int rr) {
          float xv[V];
          if constexpr (V == 2) {
            const float2 a = *reinterpret_cast<const float2*>(st + rr * rs + lane * 2);
            xv[0] = a.x;
            xv[1] = a.y;
          } else if constexpr (V == 4) {
            const float4 a = *reinterpret_cast<const float4*>(st + rr * rs + lane * 4);
            xv[0] = a.x;
            xv[1] = a.y;
            xv[2] = a.z;
            xv[3] = a.w;
          } else {
#pragma unroll
            for (int v = 0; v < V; ++v) xv[v] = st[rr * rs + v * 32 + lane];
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float xr = xv[v];
            kahan_add(s[v], c[v], xr);
            const float df = __fsub_rn(xr, cj[v]);
            qacc = fmaf(df, df, qacc);
          }
        };
        for (; r + RF <= rend; r += RF) {
#pragma unroll
          for (int u = 0; u < RF; ++u) row(r + u);
          kahan_add(objS, objC, qacc);
          qacc = 0.f;
        }
        for (; r < rend; ++r) row(r);
        kahan_add(objS, objC, qacc);
        qacc = 0.f;
      }
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
    i_c = i_n;
    j_c = j_n;
    i_n = i_nn;
    j_n = j_nn;
  }
  flush();
  double o = (double)objS - (double)objC;
#pragma unroll
  for (int off = 16; off; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
  if (lane == 0 && o != 0.0) atomicAdd(&W.ctls[it.b].objective, o);
}

// Packed rows (d <= DP <= 16, DP the power of two >= d): batches of up to 128
// rows (lane l holds the indices of rows l, l + 32, l + 64, l + 96), so that a
// warp keeps a few KB of these short rows in flight; lane group g = lane / DP
// takes row r0 + g of each step, lane t = lane mod DP its column t, and keeps
// its own run (flushed alone). A full batch runs as unrolled steps; the
// objective terms are added plainly over 8 steps (one term per lane each),
// each partial then Kahan-added.
template <int DP>
__device__ __forceinline__ void seg_item_packed(const BWork& W, const BChunk& it, float* stage0, float* stage1,
                                                int lane) {
  constexpr int RB = kSegStage / DP < 128 ? kSegStage / DP : 128;  // rows per batch (a multiple of 32 / DP)
  constexpr int G = 32 / DP;                                       // rows per warp step
  const BInst& I = W.inst[it.b];
  const int d = I.d;
  const float* __restrict__ X = I.X;
  const float* __restrict__ C = I.C;
  double* sums = W.sums64 + I.sum_off;
  const int32_t* perm = W.perm + it.r0;
  const int32_t* labs = W.lab_sorted + it.r0;
  const int nb = (it.n + RB - 1) / RB;
  auto meta = [&](int bt, int (&i)[4], int (&j)[4]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int r = bt * RB + m * 32 + lane;
      i[m] = 0;
      j[m] = -1;
      if (m * 32 < RB && r < it.n) {
        i[m] = __ldg(perm + r);
        j[m] = __ldg(labs + r);
      }
    }
  };
  auto gather = [&](int bt, float* st, const int (&i)[4]) {
    const int rows = min(RB, it.n - bt * RB);
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (m * 32 < rows) gather_rows(st + m * 32 * DP, DP, X, d, min(32, rows - m * 32), (int64_t)i[m] * d, lane, false);
    cp_async_commit();
  };
  const int g = lane / DP, t = lane & (DP - 1);
  // columns [d, DP) of every row slot hold zeros (the gathers write only [0, d))
  if (d < DP) {
    for (int e = lane; e < RB * DP; e += 32)
      if ((e & (DP - 1)) >= d) stage0[e] = stage1[e] = 0.f;
    __syncwarp();
  }
  float s = 0.f, c = 0.f, cj = 0.f, objS = 0.f, objC = 0.f, qacc = 0.f;
  int cur = -1;  // this lane's run
  auto flush = [&]() {
    if (cur < 0) return;
    if (t < d) atomicAdd(sums + (int64_t)cur * d + t, (double)s - (double)c);
    s = c = 0.f;
  };
  // row r of the batch in stage st, label j (every lane of the group)
  auto step = [&](const float* st, int r, int j) {
    if (j != cur) {
      flush();
      cur = j;
      cj = t < d ? C[(int64_t)j * d + t] : 0.f;
    }
    const float xr = st[r * DP + t];
    kahan_add(s, c, xr);
    const float df = __fsub_rn(xr, cj);
    qacc = fmaf(df, df, qacc);
  };
  int i_c[4], j_c[4], i_n[4], j_n[4];
  meta(0, i_c, j_c);
  gather(0, stage0, i_c);
  if (nb > 1) meta(1, i_n, j_n);
  for (int bt = 0; bt < nb; ++bt) {
    float* st = (bt & 1) ? stage1 : stage0;
    if (bt + 1 < nb) gather(bt + 1, (bt & 1) ? stage0 : stage1, i_n);
    int i_nn[4], j_nn[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      i_nn[m] = 0;
      j_nn[m] = -1;
    }
    if (bt + 2 < nb) meta(bt + 2, i_nn, j_nn);
    if (bt + 1 < nb) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncwarp();
    const int rows = min(RB, it.n - bt * RB);
    if (rows == RB) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (m * 32 >= RB) break;
#pragma unroll
        for (int q = 0; q < 32 / G; ++q) {
          if (m * 32 + (q + 1) * G > RB) break;
          step(st, m * 32 + q * G + g, __shfl_sync(0xffffffffu, j_c[m], q * G + g));
          if ((q & 7) == 7) {
            kahan_add(objS, objC, qacc);
            qacc = 0.f;
          }
        }
        kahan_add(objS, objC, qacc);
        qacc = 0.f;
      }
    } else {
      int q8 = 0;
      for (int r0 = 0; r0 < rows; r0 += G) {
        const int m = r0 >> 5;  // the same for every lane (G divides 32)
        const int jm = m == 0 ? j_c[0] : (m == 1 ? j_c[1] : (m == 2 ? j_c[2] : j_c[3]));
        const int r = r0 + g;
        const bool ok = r < rows;
        const int j = __shfl_sync(0xffffffffu, jm, ok ? (r & 31) : 0);
        if (ok) step(st, r, j);
        if (++q8 == 8) {
          kahan_add(objS, objC, qacc);
          qacc = 0.f;
          q8 = 0;
        }
      }
      kahan_add(objS, objC, qacc);
      qacc = 0.f;
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      i_c[m] = i_n[m];
      j_c[m] = j_n[m];
      i_n[m] = i_nn[m];
      j_n[m] = j_nn[m];
    }
  }
  flush();
  double o = (double)objS - (double)objC;
#pragma unroll
  for (int off = 16; off; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
  if (lane == 0 && o != 0.0) atomicAdd(&W.ctls[it.b].objective, o);
}

__global__ void __launch_bounds__(256, 4) b_segsum_kernel(BWork W) {
  extern __shared__ __align__(16) float bseg_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* stage0 = bseg_smem + (size_t)wib * 2 * kSegStage;
  float* stage1 = stage0 + kSegStage;
  const int64_t nw = (int64_t)gridDim.x * 8;
  for (int64_t q = (int64_t)blockIdx.x * 8 + wib; q < W.nsitems; q += nw) {
    const BChunk it = W.sitems[q];
    if (halted(W.ctls + it.b)) continue;
    const int d = W.inst[it.b].d;
    if (d <= 1) seg_item_packed<1>(W, it, stage0, stage1, lane);
    else if (d <= 2) seg_item_packed<2>(W, it, stage0, stage1, lane);
    else if (d <= 4) seg_item_packed<4>(W, it, stage0, stage1, lane);
    else if (d <= 8) seg_item_packed<8>(W, it, stage0, stage1, lane);
    else if (d <= 16) seg_item_packed<16>(W, it, stage0, stage1, lane);
    else if (d <= 32) seg_item<1>(W, it, stage0, stage1, lane);
    else if (d <= 64) seg_item<2>(W, it, stage0, stage1, lane);
    else seg_item<4>(W, it, stage0, stage1, lane);
  }
}

// Divide per centroid of every instance (one warp per centroid, its instance
// from the table). A lane's coordinates t = lane, lane + 32, ... are all loaded
// before any store, so a centroid costs one round trip to memory whatever d.
__global__ void __launch_bounds__(256) b_divide_kernel(BWork W) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < W.KC;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int b = __ldg(W.kc_inst + g);
    Ctl* ctl = W.ctls + b;
    if (halted(ctl)) continue;
    const BInst& I = W.inst[b];
    const int j = (int)(g - I.kc_off), d = I.d;
    float* __restrict__ Cj = I.C + (int64_t)j * d;
    float* __restrict__ Sj = I.sums + (int64_t)j * d;
    double* __restrict__ sp = W.sums64 + I.sum_off + (int64_t)j * d;
    const int cnt = I.counts[j];
    double sv[kMaxV];
    float co[kMaxV];
#pragma unroll
    for (int v = 0; v < kMaxV; ++v) {
      const int t = v * 32 + lane;
      sv[v] = t < d ? sp[t] : 0.0;
      co[v] = t < d ? Cj[t] : 0.f;
    }
    // FP64 quotients: a lane with more than one coordinate divides once, y = RN(1 / cnt), and
    // corrects each quotient (div_by_recip: the same correctly rounded result as a division)
    const bool recip = d > 32 && cnt > 0;
    const double y = recip ? 1.0 / (double)cnt : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int v = 0; v < kMaxV; ++v) {
      const int t = v * 32 + lane;
      if (t < d) {
        sp[t] = 0.0;
        Sj[t] = (float)sv[v];
        const float cn =
            cnt > 0 ? (float)(recip ? div_by_recip(sv[v], (double)cnt, y) : sv[v] / (double)cnt) : co[v];
        Cj[t] = cn;
        const double df = (double)cn - (double)co[v];
        acc = fma(df, df, acc);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      atomic_max_nonneg(&ctl->shift2_bits, acc);
      if (cnt == 0) atomicAdd(&ctl->n_empty, 1);
    }
  }
}

// After the divide: every running instance records its step statistics and
// evaluates its stop rule (one thread per instance).
__global__ void __launch_bounds__(256) b_finish_kernel(BWork W, double tol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= W.nb) return;
  Ctl* ctl = W.ctls + b;
  if (halted(ctl)) return;
  const int it = ctl->iters_done;
  const int64_t h = (int64_t)b * W.iters + it;
  const double shift = sqrt(__longlong_as_double((long long)ctl->shift2_bits));
  const unsigned long long changed = ctl->n_changed;
  W.obj_hist[h] = ctl->objective;
  W.shift_hist[h] = shift;
  W.changed_hist[h] = changed;
  W.flagged_hist[h] = ctl->n_flagged;
  W.full_hist[h] = ctl->n_full;
  W.empty_hist[h] = ctl->n_empty;
  ctl->iters_done = it + 1;
  if (tol > 0.0 && (changed == 0 || shift <= tol)) ctl->done = 1;
}

int grid_for(int64_t work_items, int per_block, int cap_per_sm) {
  int64_t blocks = (work_items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms() * cap_per_sm;
  if (blocks > cap) blocks = cap;
  return (int)(blocks > 0 ? blocks : 1);
}

}  // namespace

cudaError_t launch_b_reset(const BWork& W, cudaStream_t s) {
  b_reset_kernel<<<(W.nb + 255) / 256, 256, 0, s>>>(W.ctls, W.nb, W.flag_slots);
  return cudaGetLastError();
}

cudaError_t launch_b_copy_c(const BInst* inst, int nb, float* csave, int restore, cudaStream_t s) {
  b_copy_c_kernel<<<dim3(8, (unsigned)(nb < 65535 ? nb : 65535)), 256, 0, s>>>(inst, nb, csave, restore);
  return cudaGetLastError();
}

cudaError_t launch_b_quant_x(const BWork& W, int fp8, cudaStream_t s) {
  const int grid = grid_for(W.R, 8, 16);
  if (fp8) b_quant_x_kernel<1><<<grid, 256, 0, s>>>(W);
  else b_quant_x_kernel<0><<<grid, 256, 0, s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_quant_c(const BWork& W, int fp8, cudaStream_t s) {
  const int grid = grid_for(W.KP, 8, 8);
  if (fp8) b_camax_kernel<<<W.nb, 256, 0, s>>>(W);
  if (fp8) b_quant_c_kernel<1><<<grid, 256, 0, s>>>(W);
  else b_quant_c_kernel<0><<<grid, 256, 0, s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_recheck(const BWork& W, cudaStream_t s) {
  b_recheck_kernel<<<num_sms() * 3, 256, 0, s>>>(W);  // every CTA resident (three per SM)
  return cudaGetLastError();
}

static size_t b_hist_bytes(const BWork& W) { return sizeof(int) * (size_t)(W.kmax < kBHistMax ? W.kmax : kBHistMax); }

cudaError_t launch_b_count(const BWork& W, cudaStream_t s) {
  b_count_kernel<<<grid_for(W.nrchunks, 1, 8), 256, b_hist_bytes(W), s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_scan(const BWork& W, cudaStream_t s) {
  b_scan_kernel<<<W.nb, 1024, 0, s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_scatter(const BWork& W, cudaStream_t s) {
  const size_t smem = W.kmax <= kSortedScatterMax ? (size_t)sorted_scatter_ints(W.kmax) * sizeof(int) : b_hist_bytes(W);
  b_scatter_kernel<<<grid_for(W.nrchunks, 1, 8), 256, smem, s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_permute(const BWork& W, cudaStream_t s) {
  b_permute_kernel<<<grid_for(W.nrchunks, 1, 8), 256, 0, s>>>(W);
  return cudaGetLastError();
}

cudaError_t init_batched() {
  return cudaFuncSetAttribute(b_segsum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSegSmem);
}

cudaError_t launch_b_segsum(const BWork& W, cudaStream_t s) {
  int64_t blocks = (W.nsitems + 7) / 8;
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();  // four CTAs of 8 warps per SM
  b_segsum_kernel<<<(int)(blocks > 0 ? blocks : 1), 256, kSegSmem, s>>>(W);
  return cudaGetLastError();
}

cudaError_t launch_b_divide(const BWork& W, double tol, cudaStream_t s) {
  b_divide_kernel<<<grid_for(W.KC, 8, 8), 256, 0, s>>>(W);
  b_finish_kernel<<<(W.nb + 255) / 256, 256, 0, s>>>(W, tol);
  return cudaGetLastError();
}

}  // namespace km
