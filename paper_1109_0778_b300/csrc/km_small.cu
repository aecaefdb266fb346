// Small problems (n <= 16384, k <= 64, d <= 64, n k d <= 2^23, FP32): every Lloyd
// step of a call in ONE cooperative kernel launch -- the whole loop of the
// paper's fused Lloyd iteration (Sec. 3.5, vertical fusion of the distance,
// argmin, keyed reduce and divide loops) in one kernel, with two grid barriers
// per step. For such sizes a step is a few microseconds of work, and the ~10
// launches per step of the staged path cost more than the arithmetic.
//
// G CTAs of 256 threads (k <= G <= the SM count, all resident: cooperative
// launch). T lanes share a point (T a power of two <= min(32, k), the largest
// with n T <= 256 x SMs), lane r scoring the centroids j = r mod T. Each
// cluster j is owned by S = G / k CTAs, sub-owner s scanning the labels of the
// points [n s / S, n (s+1) / S). Per step, with the accuracy contract of the
// staged FP32 path:
//   assign  -- every CTA holds C and the h_j = RN32(||c_j||^2 / 2) (FP64 norm) in
//              shared memory with their maxima H and Cmax; FP32 scores s_j = h_j -
//              x.c_j (FMA chain), the two smallest by (score, index) merged across
//              the T lanes; final when s2 - s1 > 2 E (1 + 2^-10), E = 3u H +
//              gamma_{d+1} ||x|| Cmax (u = 2^-24), else all k distances are
//              recomputed as compensated sums of rounded squared differences
//              (Kahan; relative error ~5u, so any pair with relative gap >= 1e-6 is
//              ordered exactly, equal values go to the lower index);
//   -- grid barrier --
//   reduce  -- each warp of a sub-owner lists the points of its label range that
//              belong to j (ballots, ascending index) and sums their rows in Kahan
//              FP32 per coordinate, with the objective terms ||x_i - c_j||^2; the
//              warps' partials are added in FP64 in warp order and published;
//   divide  -- the last sub-owner of j to finish (ticket) adds the S partials in
//              FP64 in sub-owner order, writes c_j = RN32(sum_j / count_j) (an
//              empty cluster keeps c_j), sum_j, count_j, the squared shift and
//              the h_j and ||c_j|| bound of the new centroid;
//   -- grid barrier --
//   next    -- every CTA loads the new C and h_j; the largest shift, the stop rule
//              (tol > 0: stop after the first step with no changed label or shift
//              <= tol), and the step's history.
// The sums are taken in a fixed order, so the centroids, sums and objective
// depend only on the inputs. Label changes and re-checks are counted with
// atomics into counters double-buffered by step parity (a step's counters are
// cleared after the next step's first barrier, when every CTA has read them).
// Every grid barrier is a bounded wait: on expiry the kernel records
// KM_ETIMEOUT and every CTA leaves. The per-step history goes to the workspace
// arrays the staged path fills, so the call's statistics are read back the
// same way.
#include "km_internal.cuh"
#include "km_quant.cuh"
#include "km_tc.cuh"

namespace km {

namespace {

constexpr int kSmallThreads = 256;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallMaxK = 64;
constexpr int kListRows = 256;  // labels a warp lists per batch

__host__ __device__ constexpr size_t a16(size_t v) { return (v + 15) / 16 * 16; }

// Global state of one call (in the workspace). The header and the tickets
// start at zero; the rest is written before it is read.
struct SmallScratch {
  unsigned int bar_count, bar_gen;  // grid barrier
  int error;                        // first km_status recorded by any CTA
  unsigned int pad;
  unsigned int changed[2], flagged[2];
};

// Offsets (bytes) of the arrays that follow the header.
struct SmallLayout {
  size_t tick, part, shift2, obj, h, cn, cnt, total;
  __host__ __device__ SmallLayout(int G, int d, int k) {
    size_t o = a16(sizeof(SmallScratch));
    tick = o;   o = a16(o + 4 * (size_t)k);                // [k] arrivals of the sub-owners
    part = o;   o = a16(o + 8 * (size_t)G * (d + 2));      // [G][d+2] a sub-owner's sums, count, objective
    shift2 = o; o = a16(o + 8 * (size_t)k);                // [k] ||c_j^{t+1} - c_j^t||^2
    obj = o;    o = a16(o + 8 * (size_t)k);                // [k] objective terms of cluster j
    h = o;      o = a16(o + 4 * (size_t)k);                // [k] h_j of the new centroids
    cn = o;     o = a16(o + 4 * (size_t)k);                // [k] ||c_j|| rounded up
    cnt = o;    o = a16(o + 4 * (size_t)k);                // [k] cluster sizes
    total = o;
  }
};

struct SmallArgs {
  const float* X;
  int64_t n;
  int d, k;
  float* C;
  int32_t* assign;
  float* sums;
  int32_t* counts;
  int iters;
  double tol;
  int first;    // no previous labels (the first step counts every point as changed)
  int recheck;  // 0: keep the FP32 argmin of the scores
  int T;        // lanes per point
  int stall;    // test knob: the first grid barrier waits for one CTA more than the grid has (it expires)
  Work w;
  char* scr;
};

// Bounded grid barrier over all G resident CTAs. Returns false if the wait
// gave up (~1 s, or another CTA gave up) or an error is recorded.
__device__ __forceinline__ bool grid_barrier(SmallScratch* scr, unsigned nblocks) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &scr->bar_gen;
    volatile int* err = &scr->error;
    const unsigned int g = *gen;
    __threadfence();
    if (atomicAdd(&scr->bar_count, 1u) == nblocks - 1) {
      scr->bar_count = 0u;
      __threadfence();
      atomicAdd(&scr->bar_gen, 1u);
    } else {
      const uint64_t t0 = tc::globaltimer_ns();
      for (uint32_t it = 0; *gen == g; ++it) {
        if ((it & 15u) == 15u) {
          if (*err == (int)KM_ETIMEOUT) break;
          if (tc::globaltimer_ns() - t0 > 1000000000ull) {
            atomicCAS(&scr->error, 0, (int)KM_ETIMEOUT);
            break;
          }
        }
      }
    }
    __threadfence();
    ok_s = *err == 0;
  }
  __syncthreads();
  return ok_s != 0;
}

// Compensated squared distance (rounded differences and squares, Kahan sum).
template <int D>
__device__ __forceinline__ float comp_dist(const float (&x)[D], const float* c, int d) {
  float s = 0.f, cmp = 0.f;
#pragma unroll
  for (int t = 0; t < D; ++t) {
    if (t < d) {
      const float df = __fsub_rn(x[t], c[t]);
      kahan_add(s, cmp, __fmul_rn(df, df));
    }
  }
  return s - cmp;
}

// (a, ja) precedes (b, jb): smaller value, then lower index.
__device__ __forceinline__ bool before(float a, int ja, float b, int jb) { return a < b || (a == b && ja < jb); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int D>
__global__ void __launch_bounds__(kSmallThreads, 1) small_run_kernel(SmallArgs A) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  const int n = (int)A.n, d = A.d, k = A.k, kd = k * d, T = A.T;
  const int G = (int)gridDim.x, S = G / k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, cta = blockIdx.x;
  const int r = lane & (T - 1);  // this lane's share of the centroids: j = r mod T
  const int per_warp = 32 / T, per_cta = kSmallThreads / T;
  float* Cs = reinterpret_cast<float*>(small_smem);  // [k*d] C of this step (16-byte aligned rows when d % 4 == 0)
  float* hs = Cs + kd;                               // [k]
  __shared__ double wsum[kSmallWarps][64], wobj[kSmallWarps];
  __shared__ int wcount[kSmallWarps], wlist[kSmallWarps][kListRows];
  __shared__ unsigned int H_bits, Cmax_bits, nonfinite_s;
  __shared__ int last_s;
  SmallScratch* scr = reinterpret_cast<SmallScratch*>(A.scr);
  const SmallLayout L(G, d, k);
  unsigned int* tick = reinterpret_cast<unsigned int*>(A.scr + L.tick);
  double* part = reinterpret_cast<double*>(A.scr + L.part);
  double* shift2g = reinterpret_cast<double*>(A.scr + L.shift2);
  double* objg = reinterpret_cast<double*>(A.scr + L.obj);
  float* hg = reinterpret_cast<float*>(A.scr + L.h);
  float* cng = reinterpret_cast<float*>(A.scr + L.cn);
  int* cntg = reinterpret_cast<int*>(A.scr + L.cnt);
  Ctl* ctl = A.w.ctl;
  int first = A.first;

  // ---------------------------------------------------------------- C and h_j of the first step
  if (tid == 0) {
    H_bits = 0u;
    Cmax_bits = 0u;
    nonfinite_s = 0u;
  }
  for (int e = tid; e < kd; e += kSmallThreads) Cs[e] = A.C[e];
  __syncthreads();
  for (int j = warp; j < k; j += kSmallWarps) {
    double s2 = 0.0;
    for (int t = lane; t < d; t += 32) s2 = fma((double)Cs[j * d + t], (double)Cs[j * d + t], s2);
    s2 = warp_sum(s2);
    if (lane == 0) {
      const float h = __double2float_rn(0.5 * s2);
      const float cn = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
      if (!isfinite(h) || !isfinite(cn)) nonfinite_s = 1u;
      hs[j] = h;
      atomic_max_nonneg(&H_bits, h);
      atomic_max_nonneg(&Cmax_bits, cn);
    }
  }
  __syncthreads();

  bool ok = true;
  for (int it = 0; it < A.iters; ++it) {
    const int q = it & 1;
    const float H = __uint_as_float(H_bits), Cmax = __uint_as_float(Cmax_bits);
    const float gam = (float)(d + 1) * kU / (1.f - (float)(d + 1) * kU);
    const bool vec4 = (d & 3) == 0;

    // ---------------------------------------------------------------- assign
    unsigned my_changed = 0, my_flagged = 0;
    // point of lane group g of round m: m G per_cta + cta per_cta + warp per_warp + lane / T
    for (int ib = cta * per_cta + warp * per_warp; ib < n; ib += G * per_cta) {  // warp-uniform loop
      const int i = ib + lane / T;
      const bool live = i < n;
      float x[D];
      const float* xr = A.X + (int64_t)(live ? i : 0) * d;
      float xx = 0.f;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        x[t] = (live && t < d) ? xr[t] : 0.f;
        xx = fmaf(x[t], x[t], xx);
      }
      const int old_raw = (live && r == 0 && !first) ? A.assign[i] : -1;
      if (live && !isfinite(xx)) nonfinite_s = 1u;
      float b1 = INFINITY, b2 = INFINITY;
      int label = r;  // (stays in range even if every score is NaN)
      for (int j = r; j < k; j += T) {
        const float* c = Cs + j * d;
        float acc = 0.f;
        if (vec4) {  // four coordinates per shared load
#pragma unroll
          for (int t = 0; t < D; t += 4) {
            if (t < d) {
              const float4 c4 = *reinterpret_cast<const float4*>(c + t);
              acc = fmaf(x[t], c4.x, acc);
              acc = fmaf(x[t + 1], c4.y, acc);
              acc = fmaf(x[t + 2], c4.z, acc);
              acc = fmaf(x[t + 3], c4.w, acc);
            }
          }
        } else {
#pragma unroll
          for (int t = 0; t < D; ++t)
            if (t < d) acc = fmaf(x[t], c[t], acc);
        }
        const float s = hs[j] - acc;
        if (s < b1) {  // j increases within a lane: strict < keeps the lowest index
          b2 = b1;
          b1 = s;
          label = j;
        } else if (s < b2) {
          b2 = s;
        }
      }
      for (int o = T >> 1; o; o >>= 1) {  // merge the T lanes' two smallest
        const float p1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const float p2 = __shfl_xor_sync(0xffffffffu, b2, o);
        const int pj = __shfl_xor_sync(0xffffffffu, label, o);
        if (before(p1, pj, b1, label)) {
          b2 = fminf(b1, p2);
          b1 = p1;
          label = pj;
        } else {
          b2 = fminf(b2, p1);
        }
      }
      if (A.recheck && k > 1) {
        const float E = fmaf(3.f * kU, H, gam * norm_bound(xx, d) * Cmax);
        const bool flag = live && !(__fsub_rn(b2, b1) > 2.f * E * (1.f + 0x1p-10f));
        if (__any_sync(0xffffffffu, flag)) {  // near-tie: exact distances to all k
          float best = INFINITY;
          int jb = r;
          if (flag)
            for (int j = r; j < k; j += T) {
              const float Dj = comp_dist<D>(x, Cs + j * d, d);
              if (Dj < best) {
                best = Dj;
                jb = j;
              }
            }
          for (int o = T >> 1; o; o >>= 1) {
            const float pb = __shfl_xor_sync(0xffffffffu, best, o);
            const int pj = __shfl_xor_sync(0xffffffffu, jb, o);
            if (before(pb, pj, best, jb)) {
              best = pb;
              jb = pj;
            }
          }
          if (flag) {
            label = jb;
            my_flagged += r == 0;
          }
        }
      }
      if (live && r == 0) {
        const int old = (old_raw < 0 || old_raw >= k) ? -1 : old_raw;
        my_changed += (old != label);
        A.assign[i] = label;
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      my_changed += __shfl_xor_sync(0xffffffffu, my_changed, o);
      my_flagged += __shfl_xor_sync(0xffffffffu, my_flagged, o);
    }
    if (lane == 0) {
      if (my_changed) atomicAdd(&scr->changed[q], my_changed);
      if (my_flagged) atomicAdd(&scr->flagged[q], my_flagged);
    }
    __syncthreads();
    if (tid == 0 && nonfinite_s) atomicCAS(&scr->error, 0, (int)KM_ENONFINITE);
    if (!(ok = grid_barrier(scr, G + (it == 0 ? A.stall : 0)))) break;

    // ---------------------------------------------------------------- reduce + divide (owners)
    if (cta == 0 && tid == 0) {  // the previous step's counters (every CTA read them before the barrier)
      scr->changed[1 - q] = 0u;
      scr->flagged[1 - q] = 0u;
    }
    if (cta < k * S) {
      const int j = cta / S, s = cta % S;
      const int64_t lo = (int64_t)n * s / S, hi = (int64_t)n * (s + 1) / S;
      const int w0 = (int)(lo + (hi - lo) * warp / kSmallWarps), w1 = (int)(lo + (hi - lo) * (warp + 1) / kSmallWarps);
      float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, oS = 0.f, oC = 0.f;
      const float cj0 = lane < d ? Cs[j * d + lane] : 0.f;
      const float cj1 = lane + 32 < d ? Cs[j * d + lane + 32] : 0.f;
      int count = 0;
      int* list = wlist[warp];
      for (int base = w0; base < w1; base += kListRows) {
        int lab[kListRows / 32];
#pragma unroll
        for (int c = 0; c < kListRows / 32; ++c) {  // all label loads in flight together
          const int i = base + 32 * c + lane;
          lab[c] = i < w1 ? __ldcg(&A.assign[i]) : -1;
        }
        int m = 0;
#pragma unroll
        for (int c = 0; c < kListRows / 32; ++c) {  // members in ascending index
          const unsigned mask = __ballot_sync(0xffffffffu, lab[c] == j);
          if (lab[c] == j) list[m + __popc(mask & ((1u << lane) - 1u))] = base + 32 * c + lane;
          m += __popc(mask);
        }
        __syncwarp();
        count += m;
        constexpr int RB = D <= 32 ? 32 : 16;  // rows whose loads are in flight together
        for (int r0 = 0; r0 < m; r0 += RB) {
          float xa[RB], xb[D > 32 ? RB : 1];
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const bool okr = r0 + u < m;
            const float* xr = A.X + (int64_t)(okr ? list[r0 + u] : 0) * d;
            xa[u] = okr && lane < d ? xr[lane] : 0.f;
            if constexpr (D > 32) xb[u] = okr && lane + 32 < d ? xr[lane + 32] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            if (r0 + u >= m) break;  // the same for every lane
            const float xbu = D > 32 ? xb[D > 32 ? u : 0] : 0.f;
            kahan_add(s0, c0, xa[u]);
            kahan_add(s1, c1, xbu);
            const float d0 = lane < d ? __fsub_rn(xa[u], cj0) : 0.f;
            const float d1 = lane + 32 < d ? __fsub_rn(xbu, cj1) : 0.f;
            kahan_add(oS, oC, fmaf(d1, d1, d0 * d0));
          }
        }
        __syncwarp();
      }
      wsum[warp][lane] = (double)s0 - (double)c0;
      wsum[warp][lane + 32] = (double)s1 - (double)c1;
      const double ow = warp_sum((double)oS - (double)oC);
      if (lane == 0) {
        wobj[warp] = ow;
        wcount[warp] = count;
      }
      __syncthreads();
      double* mine = part + (size_t)cta * (d + 2);
      if (tid < d) {
        double v = 0.0;
        for (int w2 = 0; w2 < kSmallWarps; ++w2) v += wsum[w2][tid];
        mine[tid] = v;
      } else if (tid == 64) {
        int c = 0;
        double o = 0.0;
        for (int w2 = 0; w2 < kSmallWarps; ++w2) {
          c += wcount[w2];
          o += wobj[w2];
        }
        mine[d] = (double)c;
        mine[d + 1] = o;
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const bool last = atomicAdd(&tick[j], 1u) == (unsigned)(S - 1);
        if (last) {
          tick[j] = 0u;
          __threadfence();
        }
        last_s = last;
      }
      __syncthreads();
      if (last_s && warp == 0) {  // the divide of cluster j, from the S partials in sub-owner order
        const double* pj = part + (size_t)j * S * (d + 2);
        double t0 = 0.0, t1 = 0.0, cnt = 0.0, obj = 0.0;
        for (int s2 = 0; s2 < S; ++s2) {
          const double* p = pj + (size_t)s2 * (d + 2);
          if (lane < d) t0 += __ldcg(p + lane);
          if (lane + 32 < d) t1 += __ldcg(p + lane + 32);
          cnt += __ldcg(p + d);
          obj += __ldcg(p + d + 1);
        }
        const int cn = (int)cnt;
        const float n0 = cn > 0 ? (float)(t0 / cnt) : cj0;
        const float n1 = cn > 0 ? (float)(t1 / cnt) : cj1;
        if (lane < d) {
          A.C[j * d + lane] = n0;
          A.sums[j * d + lane] = (float)t0;
        }
        if (lane + 32 < d) {
          A.C[j * d + lane + 32] = n1;
          A.sums[j * d + lane + 32] = (float)t1;
        }
        const double e0 = (double)n0 - (double)cj0, e1 = (double)n1 - (double)cj1;
        const double sh = warp_sum(fma(e1, e1, e0 * e0));
        const double s2 = warp_sum(fma((double)n1, (double)n1, (double)n0 * (double)n0));
        if (lane == 0) {
          shift2g[j] = sh;
          objg[j] = obj;
          cntg[j] = cn;
          A.counts[j] = cn;
          hg[j] = __double2float_rn(0.5 * s2);
          cng[j] = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
        }
      }
    }
    if (!(ok = grid_barrier(scr, G))) break;

    // ---------------------------------------------------------------- the new C, the stop rule, the history
    if (tid == 0) {
      H_bits = 0u;
      Cmax_bits = 0u;
    }
    __syncthreads();
    for (int e = tid; e < kd; e += kSmallThreads) Cs[e] = __ldcg(&A.C[e]);
    __shared__ double shift2_s;
    __shared__ unsigned int nf_next;
    if (warp == 0) {
      double m = 0.0;
      unsigned nf = 0u;
      for (int j = lane; j < k; j += 32) {
        const float h = __ldcg(&hg[j]), cn = __ldcg(&cng[j]);
        m = fmax(m, __ldcg(&shift2g[j]));
        hs[j] = h;
        nf |= (!isfinite(h) || !isfinite(cn)) ? 1u : 0u;
        atomic_max_nonneg(&H_bits, h);
        atomic_max_nonneg(&Cmax_bits, cn);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        nf |= __shfl_xor_sync(0xffffffffu, nf, o);
      }
      if (lane == 0) {
        shift2_s = m;
        nf_next = nf;
      }
    } else if (cta == 0 && warp == 1 && lane == 0) {
      double o = 0.0;
      int empty = 0;
      for (int j = 0; j < k; ++j) {
        o += __ldcg(&objg[j]);
        empty += __ldcg(&cntg[j]) == 0;
      }
      A.w.obj_hist[it] = o;
      A.w.changed_hist[it] = __ldcg(&scr->changed[q]);
      A.w.flagged_hist[it] = __ldcg(&scr->flagged[q]);
      A.w.full_hist[it] = __ldcg(&scr->flagged[q]);
      A.w.empty_hist[it] = empty;
      A.w.queued_hist[it] = 0ull;
    }
    __syncthreads();
    const double shift = sqrt(shift2_s);
    const unsigned changed = __ldcg(&scr->changed[q]);
    if (cta == 0 && tid == 0) {
      A.w.shift_hist[it] = shift;
      ctl->iters_done = it + 1;
    }
    if (A.tol > 0.0 && (changed == 0u || shift <= A.tol)) break;  // every CTA takes the same decision
    if (nf_next && tid == 0) nonfinite_s = 1u;  // reported by the next step (C^{t+1} has a non-finite norm)
    first = 0;
  }
  if (!ok && cta == 0 && tid == 0) {
    const int err = *(volatile int*)&scr->error;
    if (err == (int)KM_ENONFINITE) ctl->nonfinite = 1;
    else ctl->error = err ? err : (int)KM_ETIMEOUT;
  }
  // C, sums and counts were written by the cluster owners (on an error the caller restores C)
}

size_t small_smem_bytes(int d, int k) { return (size_t)4 * ((size_t)k * d + k); }

// Lanes per point: the largest power of two <= min(32, k) with n T <= 256 x SMs (at least 1).
int small_lanes(int64_t n, int k) {
  int T = 1;
  while (T < 32 && 2 * T <= k && n * 2 * T <= (int64_t)kSmallThreads * num_sms()) T *= 2;
  return T;
}

// CTAs: enough for one lane group per point, and at least one per cluster.
int small_ctas(int64_t n, int k) {
  const int64_t want = std::max<int64_t>((n * small_lanes(n, k) + kSmallThreads - 1) / kSmallThreads, k);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, num_sms()));
}

template <int D>
cudaError_t small_launch(SmallArgs A, int G, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(small_run_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)small_run_kernel<D>, dim3(G), dim3(kSmallThreads), args, smem, s);
}

}  // namespace

bool small_path_fits(int64_t n, int d, int k) {
  return n <= 16384 && k <= kSmallMaxK && d <= 64 && n * (int64_t)k * d <= (int64_t)1 << 23 && k <= num_sms();
}

size_t small_scratch_bytes(int64_t n, int d, int k) { return SmallLayout(small_ctas(n, k), d, k).total; }

cudaError_t launch_small_run(const Problem& p, const Work& w, int iters, double tol, int first, int recheck,
                             cudaStream_t s) {
  const int G = small_ctas(p.n, p.k);
  SmallArgs A{p.X, p.n, p.d, p.k, p.C, p.assign, p.sums, p.counts, iters, tol, first, recheck,
              small_lanes(p.n, p.k), getenv("KM_DEBUG_STALL") ? 1 : 0, w, reinterpret_cast<char*>(w.small)};
  const SmallLayout L(G, p.d, p.k);
  cudaError_t e = cudaMemsetAsync(w.small, 0, L.part, s);  // header and tickets
  if (e != cudaSuccess) return e;
  const size_t smem = small_smem_bytes(p.d, p.k);
  if (p.d <= 8) return small_launch<8>(A, G, smem, s);
  if (p.d <= 16) return small_launch<16>(A, G, smem, s);
  if (p.d <= 32) return small_launch<32>(A, G, smem, s);
  return small_launch<64>(A, G, smem, s);
}

}  // namespace km
