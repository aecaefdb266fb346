// Exact re-check of flagged near-ties with compensated FP32 distances.
//
// A warp takes 32 flagged points at a time. Each lane settles its own point
// when the assignment stage kept a short candidate list (lane_settle); the
// points it could not narrow are queued for the re-score pass or, failing
// that, screened against all k centroids one at a time by the whole warp
// (nearest_all). The distances, the tie rule and the error argument are those
// of km_recheck.cuh.
#include <functional>

#include "km_quant.cuh"
#include "km_recheck.cuh"

namespace km {

namespace {

// CTAs per SM: three for d <= 128 (up to 85 registers; short lists take two
// candidates per round), two above (the point's longer slices need more).
template <int V>
constexpr int recheck_ctas() { return V <= 4 ? 3 : 2; }

template <int V>
__global__ void __launch_bounds__(256, recheck_ctas<V>())
recheck_kernel(const float* __restrict__ X, int d, const float* __restrict__ C, const float* __restrict__ h, int k,
               const FlagRec* __restrict__ flags, const unsigned long long* nflag_ptr, Ctl* ctl,
               int32_t* __restrict__ assign, int32_t* __restrict__ q_rows, int32_t* __restrict__ q_old,
               int64_t q_cap) {
  if (halted(ctl)) return;
  __shared__ __align__(16) float xs_all[8][V * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* xsh = xs_all[wib];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const int64_t nflag = (int64_t)*nflag_ptr;
  const float H = __uint_as_float(ctl->hmax_bits), Cmax = __uint_as_float(ctl->cmax_bits);
  unsigned int changed = 0;
  // 32 flags per warp step, nwarps apart (few flags still spread one per warp): lane l reads
  // flag f0 + l nwarps's header; the points whose candidates could not be narrowed are queued
  // with one atomic per warp, the others are settled one at a time below
  for (int64_t f0 = warp; f0 < nflag; f0 += nwarps * 32) {
    const int64_t fl = f0 + lane * nwarps;
    const bool have = fl < nflag;
    int nc_l = -1, i_l = 0, old_l = 0;
    int cand_l[kMaxCand];
    if (have) {
      const FlagRec r = flags[fl];
      nc_l = r.nc;
      i_l = r.i;
      old_l = r.old;
#pragma unroll
      for (int a = 0; a < kMaxCand; ++a) cand_l[a] = r.cand[a];
    } else {
#pragma unroll
      for (int a = 0; a < kMaxCand; ++a) cand_l[a] = 0;
    }
    unsigned todo = __ballot_sync(0xffffffffu, have);
    if (q_rows) {
      // all k candidates: queue the point for the tiled FP32 pass while the queue has room
      const unsigned qm = __ballot_sync(0xffffffffu, have && nc_l == 0);
      if (qm) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctl->n_fullq, (unsigned long long)__popc(qm));
        base = __shfl_sync(0xffffffffu, base, 0);
        const unsigned long long slot = base + __popc(qm & ((1u << lane) - 1u));
        const bool queued = ((qm >> lane) & 1u) && slot < (unsigned long long)q_cap;
        if (queued) {
          q_rows[slot] = i_l;
          q_old[slot] = old_l;
        }
        todo &= ~__ballot_sync(0xffffffffu, queued);
      }
    }
    // short candidate lists: a group of G lanes per point, 32 / G points at a time (group_settle);
    // a round's candidate loop runs to its longest list, so the lists of at most NQ candidates
    // (one load round) go first, among themselves, then the longer ones
    const unsigned sl = __ballot_sync(0xffffffffu, ((todo >> lane) & 1u) && nc_l > 0);
    todo &= ~sl;
    constexpr int G = 8;                    // lanes per point: 4 points per round
    constexpr int F = (V * 8 + G - 1) / G;  // float4 slices of the point per lane (4 G F >= 32 V >= d)
    constexpr int NQ = V <= 4 ? 2 : (F <= 4 ? 4 : 2);
    const int g = lane / G, sub = lane % G;
    const unsigned sm1 = __ballot_sync(0xffffffffu, ((sl >> lane) & 1u) && nc_l <= NQ);
    for (int pass = 0; pass < 2; ++pass) {
    unsigned sm = pass ? sl & ~sm1 : sm1;
    while (sm) {  // warp-uniform
      const int src = nth_set_bit(sm, g);
      const int from = src < 0 ? __ffs(sm) - 1 : src;  // (a group without a point repeats the first one)
      const int ri = __shfl_sync(0xffffffffu, i_l, from), rnc = __shfl_sync(0xffffffffu, nc_l, from);
      const int rold = __shfl_sync(0xffffffffu, old_l, from);
      int cand[kMaxCand];
#pragma unroll
      for (int a = 0; a < kMaxCand; ++a) cand[a] = __shfl_sync(0xffffffffu, cand_l[a], from);
      const int ncw = __reduce_max_sync(0xffffffffu, src >= 0 ? rnc : 0);
      const int jb = group_settle<G, F, NQ>(X + (int64_t)ri * d, C, d, rnc, ncw, cand, sub);
      if (src >= 0 && sub == 0) {
        assign[ri] = jb;
        changed += (rold != jb);
      }
      for (int a = 0; a < 32 / G && sm; ++a) sm &= sm - 1;  // the points of this round
    }
    }
    // the rest (all k candidates, not queued): one point at a time, lanes over dimensions
    while (todo) {
      const int l = __ffs(todo) - 1;
      todo &= todo - 1;
      const int ri = __shfl_sync(0xffffffffu, i_l, l), rold = __shfl_sync(0xffffffffu, old_l, l);
      const float* x = X + (int64_t)ri * d;
      float xv[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int t = v * 32 + lane;
        xv[v] = t < d ? x[t] : 0.f;
      }
      const int jb = nearest_all<V>(xv, xsh, C, h, k, d, lane, H, Cmax);
      if (lane == 0) {
        assign[ri] = jb;
        changed += (rold != jb);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) changed += __shfl_xor_sync(0xffffffffu, changed, o);  // (every lane counted its own)
  if (lane == 0 && changed) atomicAdd(&ctl->n_changed, (unsigned long long)changed);
}

// Copies the queued rows into X_sub and their norm bounds (xs.w on the
// quantised paths, xnorm on the FP32 path) into xn_sub; one warp per row.
// With Xq16 (E4M3 runs) it also writes each row's BF16 codes (Kp16 columns,
// zero padded) and their statistics (1, ||x~||, ||x~ - x||, ||x||) for the
// tensor-core re-score, as the BF16 quantisation stage does.
__global__ void __launch_bounds__(256)
gather_queue_kernel(const float* __restrict__ X, int d, const float* __restrict__ xnorm, const Ctl* ctl,
                    const int32_t* __restrict__ q_rows, int64_t q_cap, float* __restrict__ X_sub,
                    float* __restrict__ xn_sub, uint8_t* __restrict__ Xq16, float4* __restrict__ xs16q, int Kp16,
                    const float* __restrict__ mu) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const int64_t nq = min((int64_t)ctl->n_fullq, q_cap);
  for (int64_t r = warp; r < nq; r += nwarps) {
    const int64_t i = q_rows[r];
    const float* x = X + i * d;
    float* y = X_sub + r * d;
    for (int t = lane; t < d; t += 32) y[t] = x[t];
    if (lane == 0) xn_sub[r] = xnorm[i];  // the uncentred norm bound (the FP32 pass scores x itself)
    if (Xq16) {  // the BF16 codes of the centred row, as the quantisation stage forms them
      float sxx = 0.f, sqq = 0.f, sdd = 0.f;
      uint8_t* row = Xq16 + r * (int64_t)Kp16 * 2;
      for (int t = lane; t < Kp16; t += 32) {
        const float v = t < d ? centred(x[t], mu, t) : 0.f;
        const float vq = quantise<0>(v, 1.f, 1.f, row + 2 * t);
        sxx = fmaf(v, v, sxx);
        sqq = fmaf(vq, vq, sqq);
        sdd = fmaf(vq - v, vq - v, sdd);
      }
      sxx = warp_sum(sxx);
      sqq = warp_sum(sqq);
      sdd = warp_sum(sdd);
      if (lane == 0) {
        const float nbv = norm_bound(sxx, d);
        xs16q[r] = make_float4(1.f, norm_bound(sqq, d), centred_resid(nbv, norm_bound(sdd, d), mu),
                               centred_norm(nbv, mu));
      }
    }
  }
}

}  // namespace

template <int V>
cudaError_t recheck_v(const Problem& p, const Work& w, const float* h, const FlagRec* flags,
                      const unsigned long long* nflag, bool queue, cudaStream_t s) {
  const int blocks = num_sms() * recheck_ctas<V>();  // every CTA resident
  recheck_kernel<V><<<blocks, 256, 0, s>>>(p.X, p.d, p.C, h, p.k, flags, nflag, w.ctl, p.assign,
                                           queue ? w.fq_rows : nullptr, queue ? w.fq_old : nullptr,
                                           queue ? w.fq_cap : 0);
  return cudaGetLastError();
}

cudaError_t recheck_pass(const Problem& p, const Work& w, const float* h, const FlagRec* flags,
                         const unsigned long long* nflag, bool queue, cudaStream_t s) {
  switch ((p.d + 31) / 32) {
    case 1: return recheck_v<1>(p, w, h, flags, nflag, queue, s);
    case 2: return recheck_v<2>(p, w, h, flags, nflag, queue, s);
    case 3: return recheck_v<3>(p, w, h, flags, nflag, queue, s);
    case 4: return recheck_v<4>(p, w, h, flags, nflag, queue, s);
    case 5: return recheck_v<5>(p, w, h, flags, nflag, queue, s);
    case 6: return recheck_v<6>(p, w, h, flags, nflag, queue, s);
    case 7: return recheck_v<7>(p, w, h, flags, nflag, queue, s);
    case 8: return recheck_v<8>(p, w, h, flags, nflag, queue, s);
    default: return cudaErrorInvalidValue;
  }
}

// The re-check stage. Short candidate lists are settled directly. Points whose
// candidates could not be narrowed are queued, gathered, and scored again by
// the tiled FP32 kernel (the distances of many points against all centroids,
// each centroid tile read once per 128 points), which this time keeps the best
// two candidates and the third-best score: a point whose third score lies
// outside the margin is settled between its two candidates, the few others by
// compensated distances against all k. E4M3 runs instead re-score the queued
// points with BF16 codes on the tensor cores (tc16: a margin ~16 x tighter
// than E4M3's), then settle the short lists. (The FP32 path's own flags come from
// that kernel's top-two pass, so all of them take this route when d allows the
// slab kernel.)
cudaError_t launch_recheck(const Problem& p, const Work& w, const float* h, int first, cudaStream_t s,
                           const std::function<cudaError_t(cudaStream_t)>& tc16) {
  (void)first;  // the stored old label is -1 in a call's first step
  const bool queue = w.fq_rows != nullptr;
  cudaError_t e = recheck_pass(p, w, h, w.flags, &w.ctl->n_flagged, queue, s);
  if (e != cudaSuccess || !queue) return e;
  gather_queue_kernel<<<num_sms() * 4, 256, 0, s>>>(p.X, p.d, w.xnorm, w.ctl, w.fq_rows, w.fq_cap, w.X_sub, w.xn_sub,
                                                    tc16 ? w.Xq16 : nullptr, w.xs16q, w.Kp16, w.mu);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (tc16) e = tc16(s);  // E4M3 runs: BF16 codes on the tensor cores, then the short lists
  else e = launch_assign_simt_sub(p, w, h, s);
  if (e != cudaSuccess) return e;
  return recheck_pass(p, w, h, w.flags2, &w.ctl->n_flagged2, false, s);
}

}  // namespace km
