// Exact re-check of flagged near-ties with compensated FP32 distances.
//
// For a flagged point the candidates (all k centroids, or the short list the
// assignment stage kept) are scanned in increasing index order with
//   D_j = sum_t (x_t - c_jt)^2,
// each difference and square rounded once, the lane partials summed with
// Kahan compensation and combined across the warp with TwoSum, so the
// computed D_j is within about 5u D_j of the exact value (u = 2^-24). Two
// distances whose relative gap is at least 1e-6 are therefore always ordered
// correctly (1e-6 > 10u), and equal computed distances go to the lower index.
#include "km_internal.cuh"

namespace km {

namespace {

template <int V>
__global__ void __launch_bounds__(256)
recheck_kernel(const float* __restrict__ X, int d, const float* __restrict__ C, int k,
               const FlagRec* __restrict__ flags, Ctl* ctl, int32_t* __restrict__ assign, int first) {
  if (ctl->done) return;
  const int lane = threadIdx.x & 31;
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
      int t = v * 32 + lane;
      xv[v] = t < d ? x[t] : 0.f;
    }
    const int cnt = rec.nc ? rec.nc : k;
    float best = INFINITY;
    int jb = rec.nc ? rec.cand[0] : 0;
    for (int q = 0; q < cnt; ++q) {
      const int j = rec.nc ? rec.cand[q] : q;
      const float* c = C + (int64_t)j * d;
      float s = 0.f, comp = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        int t = v * 32 + lane;
        if (t < d) {
          float diff = __fsub_rn(xv[v], c[t]);
          kahan_add(s, comp, __fmul_rn(diff, diff));
        }
      }
      // lane value is s - comp; combine (hi, lo) pairs across the warp
      float hi = s, lo = -comp;
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        float ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        float olo = __shfl_xor_sync(0xffffffffu, lo, o);
        float sh, e;
        two_sum(hi, ohi, sh, e);
        lo = __fadd_rn(__fadd_rn(lo, olo), e);
        hi = sh;
      }
      const float D = __fadd_rn(hi, lo);
      if (D < best) {
        best = D;
        jb = j;
      }
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
#define KM_CASE(v) case v: recheck_kernel<v><<<blocks, 256, 0, s>>>(p.X, p.d, p.C, p.k, w.flags, w.ctl, p.assign, first); break;
    KM_CASE(1) KM_CASE(2) KM_CASE(3) KM_CASE(4) KM_CASE(5) KM_CASE(6) KM_CASE(7) KM_CASE(8)
#undef KM_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace km
