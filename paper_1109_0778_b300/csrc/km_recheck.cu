// Exact re-check of flagged near-ties with compensated FP32 distances.
//
// One warp per flagged point. A short candidate list (kept by the assignment
// stage) is evaluated directly; otherwise all k centroids are screened with
// plain FP32 scores and a rigorous bound first (km_recheck.cuh). The
// distances, the tie rule and the error argument are those of km_recheck.cuh.
#include "km_recheck.cuh"

namespace km {

namespace {

template <int V>
__global__ void __launch_bounds__(256)
recheck_kernel(const float* __restrict__ X, int d, const float* __restrict__ C, const float* __restrict__ h, int k,
               const FlagRec* __restrict__ flags, Ctl* ctl, int32_t* __restrict__ assign) {
  if (halted(ctl)) return;
  __shared__ __align__(16) float xs_all[8][V * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* xsh = xs_all[wib];
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
  const int64_t nflag = (int64_t)ctl->n_flagged;
  const float H = __uint_as_float(ctl->hmax_bits), Cmax = __uint_as_float(ctl->cmax_bits);
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
    int jb;
    if (rec.nc > 0) {
      float best = INFINITY;
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
      jb = nearest_all<V>(xv, xsh, C, h, k, d, lane, H, Cmax);
    }
    if (lane == 0) {
      assign[rec.i] = jb;
      changed += (rec.old != jb);
    }
  }
  if (lane == 0 && changed) atomicAdd(&ctl->n_changed, (unsigned long long)changed);
}

}  // namespace

cudaError_t launch_recheck(const Problem& p, const Work& w, const float* h, int first, cudaStream_t s) {
  (void)first;  // the stored old label is -1 in a call's first step
  const int blocks = num_sms() * 4;
  const int V = (p.d + 31) / 32;
  switch (V) {
#define KM_CASE(v) case v: recheck_kernel<v><<<blocks, 256, 0, s>>>(p.X, p.d, p.C, h, p.k, w.flags, w.ctl, p.assign); break;
    KM_CASE(1) KM_CASE(2) KM_CASE(3) KM_CASE(4) KM_CASE(5) KM_CASE(6) KM_CASE(7) KM_CASE(8)
#undef KM_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace km
