// Exact re-check of flagged near-ties with compensated FP32 distances.
//
// For a flagged point the candidates (all k centroids, or the short list the
// assignment stage kept) are evaluated as
//   D_j = sum_t (x_t - c_jt)^2,
// each difference and square rounded once and the terms summed with Kahan
// compensation (per lane, then TwoSum across the warp for short lists), so the
// computed D_j is within about 5u D_j of the exact value (u = 2^-24). Two
// distances whose relative gap is at least 1e-6 are therefore always ordered
// correctly (1e-6 > 10u), and equal computed distances go to the lower index.
#include "km_internal.cuh"

namespace km {

namespace {

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

// One warp per flagged point. Short candidate lists are scanned in index
// order with warp-wide distances; a full re-check gives each lane every 32nd
// centroid (its own Kahan chain over d, reading x from shared memory) and
// then takes the warp's lexicographic (distance, index) minimum.
template <int V>
__global__ void __launch_bounds__(256)
recheck_kernel(const float* __restrict__ X, int d, const float* __restrict__ C, int k,
               const FlagRec* __restrict__ flags, Ctl* ctl, int32_t* __restrict__ assign) {
  if (halted(ctl)) return;
  __shared__ __align__(16) float xs_all[8][V * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* xsh = xs_all[wib];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const int64_t nflag = (int64_t)ctl->n_flagged;
  unsigned int changed = 0;
  for (int64_t f = warp; f < nflag; f += nwarps) {
    const FlagRec rec = flags[f];
    const float* x = X + (int64_t)rec.i * d;
    float xv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = v * 32 + lane;
      xv[v] = t < d ? x[t] : 0.f;
    }
    float best = INFINITY;
    int jb;
    if (rec.nc > 0) {
      jb = rec.cand[0];
      for (int q = 0; q < rec.nc; ++q) {
        const int j = rec.cand[q];
        const float D = warp_sqdist<V>(xv, C + (int64_t)j * d, d, lane);
        if (D < best) {  // candidates arrive in increasing index order
          best = D;
          jb = j;
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) xsh[v * 32 + lane] = xv[v];
      __syncwarp();
      jb = k;  // no centroid yet
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
      if (jb >= k) jb = 0;  // every distance was NaN
      __syncwarp();
    }
    if (lane == 0) {
      assign[rec.i] = jb;
      changed += (rec.old != jb);
    }
  }
  if (lane == 0 && changed) atomicAdd(&ctl->n_changed, (unsigned long long)changed);
}

}  // namespace

cudaError_t launch_recheck(const Problem& p, const Work& w, int first, cudaStream_t s) {
  (void)first;  // the stored old label is -1 in a call's first step
  const int blocks = num_sms() * 4;
  const int V = (p.d + 31) / 32;
  switch (V) {
#define KM_CASE(v) case v: recheck_kernel<v><<<blocks, 256, 0, s>>>(p.X, p.d, p.C, p.k, w.flags, w.ctl, p.assign); break;
    KM_CASE(1) KM_CASE(2) KM_CASE(3) KM_CASE(4) KM_CASE(5) KM_CASE(6) KM_CASE(7) KM_CASE(8)
#undef KM_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace km
