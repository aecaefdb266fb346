// Small problems (n <= 16384, k <= 64, d <= 64, FP32): every Lloyd step of a
// call in ONE kernel launch of one CTA -- the whole loop of the paper's fused
// Lloyd iteration (Sec. 3.5, vertical fusion of the distance, argmin, keyed
// reduce and divide loops) kept on chip, with the centroids, labels and the
// cluster-sorted permutation in shared memory. For such sizes a step is a few
// microseconds of work, and the ~10 launches per step of the general path cost
// more than the arithmetic.
//
// Per step, with the accuracy contract of the general FP32 path:
//   prep    -- h_j = RN32(||c_j||^2 / 2) from an FP64 norm, ||c_j|| rounded up,
//              and their maxima H and Cmax;
//   assign  -- per point the FP32 scores s_j = h_j - x.c_j (FMA chain), the two
//              smallest (strict <: the lowest index wins ties); the point is
//              final when s2 - s1 > 2 E (1 + 2^-10) with E = 3u H + gamma_{d+1}
//              ||x|| Cmax (u = 2^-24), else its distances to all k centroids are
//              recomputed as compensated sums of rounded squared differences
//              (Kahan; relative error ~5u, so any pair with relative gap >= 1e-6
//              is ordered exactly, equal values go to the lower index);
//   reduce  -- counting sort of the points by label in shared memory, then each
//              warp sums a contiguous range of sorted positions in Kahan FP32 runs
//              that are flushed into FP64 cluster sums (one shared atomic per
//              coordinate and run); the objective J(a^t, C^t) per lane the same way;
//   divide  -- c_j = RN32(sum_j / count_j) in FP64, an empty cluster keeps c_j; the
//              largest shift; the stop rule (tol > 0: stop after the first step
//              with no changed label or shift <= tol).
// The per-step history (objective, shift, changes, re-checks, empties) goes to
// the workspace arrays the general path fills, so the call's statistics are
// read back the same way.
#include "km_internal.cuh"
#include "km_quant.cuh"

namespace km {

namespace {

constexpr int kSmallThreads = 512;
constexpr int kSmallWarps = kSmallThreads / 32;

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
  Work w;
};

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

template <int D>
__global__ void __launch_bounds__(kSmallThreads, 1) small_run_kernel(SmallArgs A) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  const int n = (int)A.n, d = A.d, k = A.k, kd = k * d;
  double* sums64 = reinterpret_cast<double*>(small_smem);       // [k*d]
  double* sh2 = sums64 + kd;                                    // [k] squared shift per centroid
  float* Cs = reinterpret_cast<float*>(sh2 + k);                // [k*d]
  float* hs = Cs + kd;                                          // [k]
  int* cnt = reinterpret_cast<int*>(hs + k);                    // [k]
  int* cur = cnt + k;                                           // [k] scatter cursors
  int* lab = cur + k;                                           // [n] labels
  int* perm = lab + n;                                          // [n] point indices by cluster
  __shared__ unsigned int H_bits, Cmax_bits, n_changed, n_flagged, n_empty, nonfinite;
  __shared__ double objective;
  __shared__ int done;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Ctl* ctl = A.w.ctl;

  for (int e = tid; e < kd; e += kSmallThreads) Cs[e] = A.C[e];
  if (tid == 0) {
    done = 0;
    nonfinite = 0;
  }
  __syncthreads();

  for (int it = 0; it < A.iters; ++it) {
    // ---------------------------------------------------------------- prep
    if (tid == 0) {
      H_bits = 0u;
      Cmax_bits = 0u;
      n_changed = 0u;
      n_flagged = 0u;
      n_empty = 0u;
      objective = 0.0;
    }
    for (int e = tid; e < kd; e += kSmallThreads) sums64[e] = 0.0;
    __syncthreads();
    for (int j = warp; j < k; j += kSmallWarps) {
      double s2 = 0.0;
      for (int t = lane; t < d; t += 32) s2 = fma((double)Cs[j * d + t], (double)Cs[j * d + t], s2);
#pragma unroll
      for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) {
        const float h = __double2float_rn(0.5 * s2);
        const float cn = __double2float_ru(sqrt(s2) * (1.0 + 1e-13));
        if (!isfinite(h) || !isfinite(cn)) nonfinite = 1u;
        hs[j] = h;
        cnt[j] = 0;
        sh2[j] = 0.0;
        atomic_max_nonneg(&H_bits, h);
        atomic_max_nonneg(&Cmax_bits, cn);
      }
    }
    __syncthreads();
    if (nonfinite) break;
    const float H = __uint_as_float(H_bits), Cmax = __uint_as_float(Cmax_bits);
    const float gam = (float)(d + 1) * kU / (1.f - (float)(d + 1) * kU);

    // ---------------------------------------------------------------- assign
    unsigned my_changed = 0, my_flagged = 0;
    for (int i = tid; i < n; i += kSmallThreads) {
      float x[D];
      const float* xr = A.X + (int64_t)i * d;
      float xx = 0.f;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        x[t] = t < d ? xr[t] : 0.f;
        xx = fmaf(x[t], x[t], xx);
      }
      if (!isfinite(xx)) nonfinite = 1u;
      float b1 = INFINITY, b2 = INFINITY;
      int j1 = 0;
      for (int j = 0; j < k; ++j) {
        const float* c = Cs + j * d;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < D; ++t)
          if (t < d) acc = fmaf(x[t], c[t], acc);
        const float s = hs[j] - acc;
        if (s < b1) {
          b2 = b1;
          b1 = s;
          j1 = j;
        } else if (s < b2) {
          b2 = s;
        }
      }
      int label = j1;
      if (A.recheck && k > 1) {
        const float E = fmaf(3.f * kU, H, gam * norm_bound(xx, d) * Cmax);
        if (!(__fsub_rn(b2, b1) > 2.f * E * (1.f + 0x1p-10f))) {  // near-tie: exact over all k
          ++my_flagged;
          float best = INFINITY;
          for (int j = 0; j < k; ++j) {
            const float Dj = comp_dist<D>(x, Cs + j * d, d);
            if (Dj < best) {
              best = Dj;
              label = j;
            }
          }
        }
      }
      int old = A.first ? -1 : A.assign[i];
      if (old < 0 || old >= k) old = -1;
      my_changed += (old != label);
      A.assign[i] = label;
      lab[i] = label;
      atomicAdd(&cnt[label], 1);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      my_changed += __shfl_xor_sync(0xffffffffu, my_changed, o);
      my_flagged += __shfl_xor_sync(0xffffffffu, my_flagged, o);
    }
    if (lane == 0) {
      atomicAdd(&n_changed, my_changed);
      atomicAdd(&n_flagged, my_flagged);
    }
    __syncthreads();
    if (nonfinite) break;

    // ---------------------------------------------------------------- counting sort
    if (warp == 0) {  // exclusive scan of the counts into the cursors (k <= 64)
      int carry = 0;
      for (int base = 0; base < k; base += 32) {
        const int j = base + lane;
        const int v = j < k ? cnt[j] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (j < k) cur[j] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += kSmallThreads) perm[atomicAdd(&cur[lab[i]], 1)] = i;
    __syncthreads();

    // ---------------------------------------------------------------- segmented sums + objective
    {
      const int p0 = (int)((int64_t)n * warp / kSmallWarps), p1 = (int)((int64_t)n * (warp + 1) / kSmallWarps);
      float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, oS = 0.f, oC = 0.f;
      int cj = -1;
      auto flush = [&]() {
        if (cj < 0) return;
        if (lane < d) atomicAdd(&sums64[cj * d + lane], (double)s0 - (double)c0);
        if (lane + 32 < d) atomicAdd(&sums64[cj * d + lane + 32], (double)s1 - (double)c1);
        s0 = c0 = s1 = c1 = 0.f;
      };
      for (int p = p0; p < p1; ++p) {
        const int i = perm[p];
        const int j = lab[i];
        if (j != cj) {
          flush();
          cj = j;
        }
        const float* xr = A.X + (int64_t)i * d;
        const float x0 = lane < d ? xr[lane] : 0.f;
        const float x1 = lane + 32 < d ? xr[lane + 32] : 0.f;
        kahan_add(s0, c0, x0);
        kahan_add(s1, c1, x1);
        const float d0 = lane < d ? __fsub_rn(x0, Cs[j * d + lane]) : 0.f;
        const float d1 = lane + 32 < d ? __fsub_rn(x1, Cs[j * d + lane + 32]) : 0.f;
        kahan_add(oS, oC, fmaf(d1, d1, d0 * d0));
      }
      flush();
      double o = (double)oS - (double)oC;
#pragma unroll
      for (int off = 16; off; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
      if (lane == 0 && o != 0.0) atomicAdd(&objective, o);
    }
    __syncthreads();

    // ---------------------------------------------------------------- divide
    for (int e = tid; e < kd; e += kSmallThreads) {
      const int j = e / d;
      const int cn = cnt[j];
      const double sv = sums64[e];
      const float co = Cs[e];
      const float cnew = cn > 0 ? (float)(sv / (double)cn) : co;
      Cs[e] = cnew;
      A.sums[e] = (float)sv;
      const double df = (double)cnew - (double)co;
      if (df != 0.0) atomicAdd(&sh2[j], df * df);
    }
    __syncthreads();
    if (tid == 0) {
      double m = 0.0;
      int empty = 0;
      for (int j = 0; j < k; ++j) {
        m = fmax(m, sh2[j]);
        empty += cnt[j] == 0;
      }
      const double shift = sqrt(m);
      A.w.obj_hist[it] = objective;
      A.w.shift_hist[it] = shift;
      A.w.changed_hist[it] = n_changed;
      A.w.flagged_hist[it] = n_flagged;
      A.w.full_hist[it] = n_flagged;
      A.w.empty_hist[it] = empty;
      A.w.queued_hist[it] = 0ull;
      ctl->iters_done = it + 1;
      if (A.tol > 0.0 && (n_changed == 0u || shift <= A.tol)) done = 1;
    }
    __syncthreads();
    if (done) break;
    A.first = 0;
  }
  if (nonfinite) {
    if (tid == 0) ctl->nonfinite = 1;
    return;  // C keeps its value on entry (the caller restores it from its copy)
  }
  for (int e = tid; e < kd; e += kSmallThreads) A.C[e] = Cs[e];
  for (int j = tid; j < k; j += kSmallThreads) A.counts[j] = cnt[j];
}

size_t small_smem_bytes(int64_t n, int d, int k) {
  return (size_t)8 * ((size_t)k * d + k) + (size_t)4 * ((size_t)k * d + k) + (size_t)4 * (2 * (size_t)k + 2 * (size_t)n);
}

template <int D>
cudaError_t small_attr(size_t smem) {
  return cudaFuncSetAttribute(small_run_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

bool small_path_fits(int64_t n, int d, int k) {
  return n <= 16384 && k <= 64 && d <= 64 && n * (int64_t)k * d <= (int64_t)1 << 23;
}

cudaError_t launch_small_run(const Problem& p, const Work& w, int iters, double tol, int first, int recheck,
                             cudaStream_t s) {
  SmallArgs A{p.X, p.n, p.d, p.k, p.C, p.assign, p.sums, p.counts, iters, tol, first, recheck, w};
  const size_t smem = small_smem_bytes(p.n, p.d, p.k);
  cudaError_t e;
  if (p.d <= 8) {
    if ((e = small_attr<8>(smem))) return e;
    small_run_kernel<8><<<1, kSmallThreads, smem, s>>>(A);
  } else if (p.d <= 16) {
    if ((e = small_attr<16>(smem))) return e;
    small_run_kernel<16><<<1, kSmallThreads, smem, s>>>(A);
  } else if (p.d <= 32) {
    if ((e = small_attr<32>(smem))) return e;
    small_run_kernel<32><<<1, kSmallThreads, smem, s>>>(A);
  } else {
    if ((e = small_attr<64>(smem))) return e;
    small_run_kernel<64><<<1, kSmallThreads, smem, s>>>(A);
  }
  return cudaGetLastError();
}

}  // namespace km
