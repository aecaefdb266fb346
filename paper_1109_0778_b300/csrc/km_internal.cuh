// Internal declarations of the fused Lloyd k-means library: the device control
// block, the workspace layout, the per-stage launchers, and small device
// helpers. Nothing here is part of the C ABI (include/kmeans.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kmeans.h"

namespace km {

constexpr int kMaxD = 256;      // largest supported dimension
constexpr int kMaxCand = 4;     // candidates kept per flagged point
constexpr float kU = 5.9604644775390625e-8f;  // FP32 unit roundoff 2^-24

// Per-run device control block. The first block of fields is per-iteration
// state and is cleared (memset) at the start of every iteration.
struct Ctl {
  // ---- per iteration (cleared) ----
  unsigned long long n_changed;
  unsigned long long n_flagged;    // entries in the flag list
  unsigned long long n_full;       // flagged points that need all k candidates
  double objective;                // J(a^t, C^t)
  unsigned long long shift2_bits;  // max_j ||dc_j||^2 as FP64 bits (>= 0)
  unsigned int cmax_bits;          // max_j ||c_j|| (FP32 bits, rounded up)
  unsigned int hmax_bits;          // max_j h_j = max_j ||c_j||^2 / 2
  unsigned int qcmax_bits;         // max_j ||c~_j|| of the quantised centroids (rounded up)
  unsigned int dcmax_bits;         // max_j ||c~_j - c_j|| (quantisation residual, rounded up)
  int n_empty;
  unsigned int blocks_done;        // last-block detection in the divide stage
  // ---- per run (cleared once) ----
  int done;          // the stop rule fired: every later stage returns at entry
  int iters_done;
  int error;         // km_status set by a device stage, 0 = none
  int nonfinite;     // X or C held a NaN / Inf or an overflowing norm
};
constexpr size_t kCtlIterBytes = offsetof(Ctl, done);

// A point whose top-2 margin is under its error bound. nc = 0: re-check
// against all k centroids; otherwise against cand[0..nc) (increasing order).
struct __align__(16) FlagRec {
  int32_t i;
  int32_t old;
  int32_t nc;
  int32_t pad;
  int32_t cand[kMaxCand];
};

// Device workspace of one call (pointers into one allocation).
struct Work {
  Ctl* ctl;
  float* xnorm;        // [n] upper bound of ||x_i||
  FlagRec* flags;      // [n]
  int32_t* perm;       // [n] point indices sorted by cluster
  int32_t* offs;       // [k+1] cluster segment starts in perm
  int32_t* cursor;     // [k] scatter cursors
  double* sums64;      // [k*d] FP64 sums (zero between iterations)
  float* chalf;        // [k] h_j = ||c_j||^2 / 2 (FP32, from FP64)
  float* cnorm;        // [k] ||c_j|| rounded up
  float* Csave;        // [k*d] C on entry (restored on error)
  double* obj_hist;    // [iters]
  double* shift_hist;  // [iters]
  unsigned long long* changed_hist;  // [iters]
  unsigned long long* flagged_hist;  // [iters]
  unsigned long long* full_hist;     // [iters]
  int* empty_hist;     // [iters]
  // quantised operands of the tensor-core path (null for FP32)
  uint8_t* Xq;         // [n][Kp] point codes (cached for the call)
  float4* xs;          // [n] row scale and norm bounds
  uint8_t* Cq;         // [kp][Kp] centroid codes (per step)
  float2* hsc;         // [kp] (h_j, sc_j)
  float4* state;       // [n] per-row (best, index, second) between centroid slabs (FP32 path)
};

// Tensor-core assignment: quantised operands and launch shape.
struct TcParams {
  const float2* hsc;  // [kp] (h_j, sc_j); h_j = +inf for padding rows j >= k
  const float4* xs;   // [n] (sx_i, ||x~_i||, ||x~_i - x_i||, ||x_i||), norms rounded up
  const uint8_t* Cq;  // [kp][Kp] centroid codes (row stride Kp * element size)
  int32_t* assign;
  FlagRec* flags;
  Ctl* ctl;
  int64_t n;
  int k, Kp, nkb, bn, nchunks, stages, first;
  uint32_t idesc;
  float gam_tc;       // accumulation bound of the tensor-core sum over Kp terms
  float gam_simt;     // accumulation bound of the FP32 SIMT seed over Kp terms
  uint64_t wait_ns;   // bound of every mbarrier wait
};

struct TcLaunch {
  CUtensorMap mapX;   // codes of X: rows n, Kp elements, box (128 B, 128 rows), 128B swizzle
  CUtensorMap mapC;   // codes of C: rows kp, Kp elements, box (128 B, bn rows), 128B swizzle
  int fp8;
};

struct Problem {
  const float* X;
  int64_t n;
  int d;
  float* C;
  int k;
  int32_t* assign;
  float* sums;
  int32_t* counts;
};

// ---- launchers (each returns the launch's cudaError_t) ----
cudaError_t launch_xnorm(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_prep(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_assign_simt(const Problem& p, const Work& w, int first, cudaStream_t s);
cudaError_t launch_recheck(const Problem& p, const Work& w, int first, cudaStream_t s);
cudaError_t launch_count(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_scan(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_scatter(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_segsum(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_divide(const Problem& p, const Work& w, int iter, double tol, cudaStream_t s);
cudaError_t launch_quant_x(const Problem& p, const Work& w, int fp8, int Kp, uint8_t* Xq, float4* xs,
                           cudaStream_t s);
cudaError_t launch_quant_c(const Problem& p, const Work& w, int fp8, int kp, int Kp, uint8_t* Cq, float2* hsc,
                           cudaStream_t s);
cudaError_t launch_assign_tc(const Problem& p, const TcLaunch& L, const TcParams& P, cudaStream_t s);
cudaError_t init_assign_tc();
size_t tc_smem_bytes(int nkb, int bn, int stages);

int num_sms();
void set_last_error(const char* msg);  // message returned by kmeans_last_error()
cudaError_t init_assign_simt();  // one-time kernel attributes (per device)
int simt_slab_width(int d);       // centroids per shared-memory slab of the FP32 kernel (0: streamed)

// ---- device helpers ----
__device__ __forceinline__ void atomic_max_nonneg(unsigned int* addr, float v) {
  atomicMax(addr, __float_as_uint(v));  // non-negative floats order like their bits
}
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated (Kahan) accumulation of one term into (s, c); the running value
// is s - c (c holds the negated low-order part lost by s).
__device__ __forceinline__ void kahan_add(float& s, float& c, float term) {
  float y = __fsub_rn(term, c);
  float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Lexicographic (value, index) order used by every argmin: lower value first,
// then lower index.
__device__ __forceinline__ bool lex_less(float a, int ia, float b, int ib) {
  return a < b || (a == b && ia < ib);
}

}  // namespace km
