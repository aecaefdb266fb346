// Internal declarations of the fused Lloyd k-means library: the device control
// block, the workspace layout, the per-stage launchers, and small device
// helpers. Nothing here is part of the C ABI (include/kmeans.h).
#pragma once

#include <functional>

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kmeans.h"

namespace km {

constexpr int kMaxD = 256;      // largest supported dimension
constexpr int kMaxCand = 8;     // candidates kept per flagged point
constexpr float kU = 5.9604644775390625e-8f;  // FP32 unit roundoff 2^-24

// Per-run device control block. The first block of fields is per-iteration
// state and is cleared (memset) at the start of every iteration.
struct Ctl {
  // ---- per iteration (cleared) ----
  unsigned long long n_changed;
  unsigned long long n_flagged;    // entries in the flag list
  unsigned long long n_full;       // flagged points that need all k candidates
  unsigned long long n_fullq;      // of those, queued for the tiled FP32 pass (re-check stage)
  unsigned long long n_flagged2;   // points the tiled FP32 pass leaves flagged
  double objective;                // J(a^t, C^t)
  unsigned long long shift2_bits;  // max_j ||dc_j||^2 as FP64 bits (>= 0)
  unsigned int cmax_bits;          // max_j ||c_j|| (FP32 bits, rounded up)
  unsigned int hmax_bits;          // max_j h_j = max_j ||c_j||^2 / 2
  unsigned int hmax_c_bits;        // the same two maxima of the centred centroids c_j - mu of the quantised
  unsigned int cmax_c_bits;        //   paths (equal to hmax, cmax without centring)
  unsigned int hmin_neg;           // min_j h_j of the quantised paths as 0x7f800000 - its bits (an atomicMax
                                   // of the complement; 0: none recorded)
  unsigned int qcmax_bits;         // max_j ||c~_j|| of the quantised centroids (rounded up)
  unsigned int dcmax_bits;         // max_j ||c~_j - c_j|| (quantisation residual, rounded up)
  unsigned int camax_bits;         // max_{j,t} |c_jt| (FP32 bits): sets the E4M3 centroid scale
  unsigned int qcmax16_bits;       // the same two maxima for the BF16 codes of an E4M3 run's
  unsigned int dcmax16_bits;       //   re-check pass (queued points re-scored with BF16)
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
// against all k centroids; otherwise against cand[0..nc), in any order (the
// re-check gives exactly equal distances to the lower index).
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
  unsigned long long* queued_hist;   // [iters] points re-scored by the queued pass
  // deterministic reduce (null otherwise): exact fixed-point sums on the grid of *xmax
  int32_t* pcounts;    // [k] counts of a partial step (the caller passes no counts array)
  unsigned int* xmax;  // max_i ||x_i|| upper bound (FP32 bits), computed once per call
  unsigned long long* facc;  // [3][k*d] integer parts of the coordinate sums (two's complement)
  unsigned long long* oacc;  // [3] integer parts of the objective
  // quantised operands of the tensor-core path (null for FP32)
  uint8_t* Xq;         // [n][Kp] point codes (cached for the call)
  float4* xs;          // [n] row scale and norm bounds
  uint8_t* Cq;         // [kp][Kp] centroid codes (per step)
  float* hq;           // [kp] h_j of the quantised path (+inf for padding)
  float* scq;          // [kp] centroid code scales
  float4* cst;         // [kp] per-centroid error-bound terms of the codes (TcParams::cst)
  float* mu;           // [d] centring vector of the quantised paths' codes (null: none)
  void* Hc;            // [kp][16] BF16 -h_j slices (folded contraction), null otherwise
  void* Xh;            // [n][16] BF16 [1/s_i, 1/s_i, 1/s_i, 0...] slices of a folded E4M3 contraction, in the
                       // codes' row order (null otherwise)
  float4* state;       // [n] per-row (best, index, second, second's index) between centroid slabs
  float* state3;       // [fq_cap] third-best score between slabs (re-check passes over gathered rows)
  float4* xs16;        // [n] BF16 statistics of a cold first step of an E4M3 run
  float4* xs_sorted;   // [n] xs in this step's cluster-sorted order (quantised paths)
  int32_t* lab_sorted; // [n] label of each sorted position (scatter stage)
  // points the assignment could not narrow to a short list: gathered and
  // re-scored by the tiled FP32 kernel keeping two candidates and a third score
  // (null when that kernel does not apply)
  int64_t fq_cap;      // rows the queue holds
  int32_t* fq_rows;    // [fq_cap] point index
  int32_t* fq_old;     // [fq_cap] previous label
  float* X_sub;        // [fq_cap][d] gathered rows
  float* xn_sub;       // [fq_cap] ||x|| bounds of the gathered rows
  FlagRec* flags2;     // [fq_cap] points the tiled FP32 pass leaves flagged
  // E4M3 runs re-score the queued points with BF16 codes on the tensor cores
  uint8_t* Xq16;       // [fq_cap][Kp16] BF16 codes of the gathered rows (null: tiled FP32 pass)
  float4* xs16q;       // [fq_cap] their row statistics
  int Kp16;            // BF16 code row width
  void* small;         // state of the one-launch small-problem path (null when it does not apply)
};

// Row map of an FP32 assignment pass over gathered rows: row r of X is point
// rows[r] with previous label old[r]; *n_dev rows; flags go to flags / *nflag.
struct SubRows {
  const int32_t* rows;  // null: row r is point r (the regular pass)
  const int32_t* old;
  const unsigned long long* n_dev;
  unsigned long long* nflag;
  FlagRec* flags;
};

struct BInst;

// Tensor-core assignment: quantised operands and launch shape.
struct TcParams {
  const float* h;     // [kp] h_j = ||c_j||^2 / 2; +inf for padding rows j >= k
  const float* sc;    // [kp] power-of-two row scale of the centroid codes
  const float4* cst;  // [kp] per-centroid error-bound terms (h_j, ||c~_j||, ||c_j||, ||c~_j - c_j||), rounded up;
                      // zeros for padding rows
  const int32_t* rows;  // row p of the code matrix holds point rows[p] (null: point p)
  const float4* xs;   // [n] (sx_i, ||x~_i||, ||x~_i - x_i||, ||x_i||), norms rounded up
  const float4* xs_sorted;  // with rows: xs of row p's point, written by the reduce stage
  const int32_t* lab_sorted;  // with rows: previous label of row p's point
  const uint8_t* Cq;  // [kp][Kp] centroid codes (row stride Kp * element size)
  int32_t* assign;
  FlagRec* flags;
  Ctl* ctl;
  int64_t n;
  int k, Kp, nkb, bn, nchunks, stages, abufs, first;
  uint32_t idesc;
  const unsigned long long* n_dev;  // non-null: the rows are the first min(n, *n_dev) (re-check pass)
  int stats16;        // read the code statistics of the BF16 re-check codes (qcmax16, dcmax16)
  int split;          // two-part BF16 codes: a row holds nkb / 2 blocks of hi, then as many of lo;
                      // x.c = hi.hi + lo.hi + hi.lo (single launches only)
  float gam_tc;       // coefficient of ||x~|| max ||c~|| in the contraction's error bound
  float hcoef;        // coefficient of max_j h_j in the score's error bound
  int fold;           // the accumulators hold (x.c_j - h_j) / (s_x s_c) (a K = 16 BF16 slice of -h_j parts);
                      // score = -(s_x s_c) acc
  uint32_t idesc16;   // instruction descriptor of that BF16 slice (E4M3 launches: a BF16 MMA on the same accumulator)
  uint64_t wait_ns;   // bound of every mbarrier wait
  int debug_stall;    // test knob: the epilogue also waits on a barrier nothing arrives on
  unsigned long long* flag_slots;  // slot counter of the flag list
  int64_t flag_cap;                // entries the flag list holds
  // batched mode (binst != null): per-instance descriptors; the fields above
  // then give only the launch shape (nkb, kp maxima), first, wait_ns and idesc
  const struct BInst* binst;
  const int64_t* btile_off;
  const int64_t* bcta;  // [grid + 1] first flattened tile of each CTA
  int nb, sorted;
  int64_t ntiles;
  Ctl* bctls;
  const CUtensorMap* bmaps;
  const CUtensorMap* bmaps_s;  // [nb] maps of the cluster-sorted code copies (gsort instances)
  float* bh;
  float* bsc;
  const float4* bcst;
  const uint8_t* bCq;
  const float4* bxs;
  const float4* bxs_sorted;
  const int32_t* blab_sorted;
  const int32_t* bperm;
};

struct TcLaunch {
  CUtensorMap mapX;   // codes of X: rows n, Kp elements, box (128 B, 128 rows), 128B swizzle
  CUtensorMap mapC;   // codes of C: rows kp, Kp elements, box (128 B, bn rows), 128B swizzle
  CUtensorMap mapH;   // folded: -h_j slices, rows kp, 16 elements, box (32 B, bn rows), 32B swizzle
  CUtensorMap mapXh;  // folded E4M3: 1/s_i slices of the point rows, box (32 B, 128 rows), 32B swizzle
  int fp8;
};

// ---------------------------------------------------------------- batched runs
// One device descriptor per independent instance; every per-instance array of
// the batch lives at an offset in one flattened array of the batch workspace.
struct BInst {
  const float* X;
  float* C;
  int32_t* assign;
  float* sums;
  int32_t* counts;
  int64_t n;
  int d, k;
  int64_t row_off;   // rows: xs, xs_sorted, lab_sorted, perm
  int64_t kc_off;    // centroids (unpadded): divide
  int64_t kp_off;    // centroids padded to whole chunks: h, sc, cursors
  int64_t offs_off;  // segment offsets (kp_off + instance index)
  int64_t sum_off;   // FP64 sums, k * d per instance
  int64_t tile_off;  // 128-row tiles
  int64_t xq_off;    // bytes: point codes [n][Kp]
  int64_t cq_off;    // bytes: centroid codes [kp][Kp]
  int Kp, nkb, kp, nchunks;
  float gam_tc;
  int rowb;  // bytes of one code row of a K block: 32 or 64 (one block, 32- or 64-byte swizzle), or 128
  int bn;    // centroid chunk width: a multiple of 32, at most the launch's (k rounded up to 32 when smaller)
  int gsort;        // from the second step on, the instance's tiles are its points in cluster-sorted order
                    // (k spans several chunks; the codes are copied in that order after each scatter)
  int64_t xqs_off;  // bytes: the cluster-sorted copy of the point codes (gsort instances)
};

// A contiguous range of one instance's flattened rows: the work item of the
// batched count and scatter stages (no instance search per row).
struct BChunk {
  int64_t r0;  // first flattened row
  int b;       // instance
  int n;       // rows (at most kBRowChunk)
};
constexpr int kBRowChunk = 4096;  // rows per chunk: 16 per thread of a 256-thread block
constexpr int kBHistMax = 8192;   // clusters of an instance counted in shared memory (more: global atomics)

struct BWork {
  const BInst* inst;
  int nb, iters;
  const BChunk* rchunks;    // [nrchunks] row chunks, in flattened order
  int nrchunks;
  int kmax;                 // largest k of the batch
  const int32_t* kc_inst;   // [KC] instance of each flattened centroid
  const int32_t* kp_inst;   // [KP] instance of each flattened padded centroid
  const int64_t* row_off;   // [nb + 1] prefix sums (binary searched)
  const int64_t* tile_off;  // [nb + 1]
  const BChunk* sitems;     // [nsitems] work items of the segmented sum (sorted positions of one instance)
  int64_t nsitems;
  const int64_t* cta_tile;  // [cta_grid + 1] tile range of each CTA of the assignment launch
  int cta_grid;
  int64_t R, KC, KP, T;     // totals: rows, centroids, padded centroids, tiles
  Ctl* ctls;                // [nb]
  unsigned long long* flag_slots;  // entries in the shared flag list
  const CUtensorMap* maps;  // [2 nb]: codes of X, codes of C
  const CUtensorMap* maps_s;  // [nb]: cluster-sorted code copies (gsort instances; zeros otherwise)
  float4* xs;
  float4* xs_sorted;
  int32_t* lab_sorted;
  int32_t* perm;
  FlagRec* flags;           // FlagRec.pad holds the instance
  int32_t* offs;
  int32_t* cursor;
  double* sums64;
  float* hq;
  float* scq;
  float4* cst;  // [KP] per-centroid error-bound terms
  uint8_t* Xq;
  uint8_t* Xqs;   // cluster-sorted copies of the gsort instances' point codes
  uint8_t* Cq;
  double* obj_hist;                  // [nb][iters]
  double* shift_hist;
  unsigned long long* changed_hist;
  unsigned long long* flagged_hist;
  unsigned long long* full_hist;
  int* empty_hist;
};

// RN(a / b) in FP64 from y = RN(1 / b), one division per divisor instead of
// one per quotient: q = RN(a y) is within an ulp of a / b, the remainder
// r = a - b q is then exact (one FMA), and RN(q + r y) is the correctly
// rounded quotient (Markstein's theorem on the final correction step of a
// division: P. Markstein, IBM J. Res. Dev. 34(1), 1990; J.-M. Muller et al.,
// Handbook of Floating-Point Arithmetic). Valid while no intermediate
// overflows or underflows: here a is a sum of FP32 values (|a| >= 2^-149 or
// 0, well inside the FP64 normal range) and b a count in [1, 2^31).
__device__ __forceinline__ double div_by_recip(double a, double b, double y) {
  const double q = a * y;
  const double r = fma(-q, b, a);
  return fma(r, y, q);
}

__device__ __forceinline__ int find_block(const int64_t* off, int nb, int64_t g) {
  int lo = 0, hi = nb;  // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

cudaError_t init_batched();
// keyed-reduce training (km_classes.cu)
cudaError_t launch_check_classes(const int32_t* y, int64_t n, int ncls, Ctl* ctl, cudaStream_t s);
cudaError_t launch_gda_means(const double* sums64, const int32_t* counts, int64_t n, int d, int ncls, float* phi,
                             float* mu, const Ctl* ctl, cudaStream_t s);
cudaError_t launch_nb_theta(const double* sums64, const int32_t* counts, int64_t n, int d, int ncls, float* prior,
                            float* theta, const Ctl* ctl, cudaStream_t s);
cudaError_t launch_gda_cov(const float* X, int64_t n, int d, const int32_t* y, const float* mu, int2* tiles_dev,
                           double* part, float* sigma, const Ctl* ctl, cudaStream_t s);
size_t gda_cov_scratch_bytes(int64_t n, int d);
cudaError_t launch_b_reset(const BWork& W, cudaStream_t s);
cudaError_t launch_b_copy_c(const BInst* inst, int nb, float* csave, int restore, cudaStream_t s);
cudaError_t launch_b_quant_x(const BWork& W, int fp8, cudaStream_t s);
cudaError_t launch_b_quant_c(const BWork& W, int fp8, cudaStream_t s);
cudaError_t launch_b_assign(const BWork& W, int fp8, int first, int sorted, int nkb_max, int kp_max, int bn,
                            int stages, int abufs, uint32_t idesc, cudaStream_t s);
cudaError_t launch_b_recheck(const BWork& W, cudaStream_t s);
cudaError_t launch_b_count(const BWork& W, cudaStream_t s);
cudaError_t launch_b_scan(const BWork& W, cudaStream_t s);
cudaError_t launch_b_scatter(const BWork& W, cudaStream_t s);
// Cluster-sorted code copies and row statistics of the gsort instances (after the scatter)
cudaError_t launch_b_permute(const BWork& W, cudaStream_t s);
cudaError_t launch_b_segsum(const BWork& W, cudaStream_t s);
cudaError_t launch_b_divide(const BWork& W, double tol, cudaStream_t s);

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
// FP32 assignment of the queued rows of the re-check stage (quantised paths); h = h_j of C.
cudaError_t launch_assign_simt_sub(const Problem& p, const Work& w, const float* h, cudaStream_t s);
cudaError_t launch_recheck(const Problem& p, const Work& w, const float* h, int first, cudaStream_t s,
                           const std::function<cudaError_t(cudaStream_t)>& tc16 = nullptr);
cudaError_t launch_count(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_scan(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_scatter(const Problem& p, const Work& w, cudaStream_t s);
// qmode 0: sums only; 1 / 2: also rewrite the BF16 / E4M3 point codes in the
// cluster-sorted order of this step (row p of w.Xq = point perm[p]).
cudaError_t init_segsum();
// det: exact fixed-point sums and objective into w.facc / w.oacc (grid of *w.xmax)
cudaError_t launch_segsum(const Problem& p, const Work& w, cudaStream_t s, int qmode = 0, int Kp = 0, int det = 0);
cudaError_t launch_divide(const Problem& p, const Work& w, int iter, double tol, cudaStream_t s, int det = 0);
// Small FP32 problems: every step of a call in one cooperative launch (km_small.cu)
bool small_path_fits(int64_t n, int d, int k);
size_t small_scratch_bytes(int64_t n, int d, int k);  // bytes of Work::small
// The quantised paths' centring vector (mean of the call's initial centroids) into w.mu
cudaError_t launch_centre(const Problem& p, const Work& w, cudaStream_t s);
cudaError_t launch_small_run(const Problem& p, const Work& w, int iters, double tol, int first, int recheck,
                             cudaStream_t s);
// max_i ||x_i|| bound into *w.xmax from per-point bounds (FP32 norms, or the .w of quantised row stats)
cudaError_t launch_xmax(const float* xnorm, const float4* xs, int64_t n, const Work& w, cudaStream_t s);
// Sharded step: the shard's partials (sums64 / facc, counts, objective, n_changed) into part
cudaError_t launch_finish_partial(const Problem& p, const Work& w, double* part, int det, cudaStream_t s);
// The divide from a reduced partials buffer; actl: 4 words of device scratch (status, shift, empties, ticket)
cudaError_t launch_apply_partials(const double* part, int k, int d, float* C, float* sums, int32_t* counts,
                                  unsigned long long* actl, cudaStream_t s);
cudaError_t launch_quant_x(const Problem& p, const Work& w, int mode, int Kp, uint8_t* Xq, float4* xs,
                           cudaStream_t s);
cudaError_t launch_quant_x_dual(const Problem& p, const Work& w, int Kp16, uint8_t* Xq, float4* xs16, float4* xs8,
                                cudaStream_t s);
// stats16: the code statistics go to qcmax16 / dcmax16 (BF16 re-check codes of an E4M3 run)
// Hc: BF16 [kp][16] slices of -h_j for the folded BF16 contraction (null: not folded)
cudaError_t launch_quant_c(const Problem& p, const Work& w, int mode, int kp, int Kp, uint8_t* Cq, void* Hc, float* h,
                           float* sc, float4* cst, cudaStream_t s, bool stats16 = false);
cudaError_t launch_assign_tc(const Problem& p, const TcLaunch& L, const TcParams& P, cudaStream_t s);
cudaError_t init_assign_tc();
// fold: -h_j folded into the contraction (a 32-byte slice per B stage row; A: a constant slice (BF16) or a
// 32-byte slice per A slot row (E4M3))
size_t tc_smem_bytes(int nkb, int bn, int stages, int kp, int fp8, int abufs, int fold = 0);
int tc_pick_buffers(int nkb, int bn, int kp, int fp8, int* abufs, int fold = 0);

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

// ---------------------------------------------------------------- exact fixed-point sums
// A value |v| <= 2^E is split into three integers q1, q2, q3 with |q_l| <= 2^20:
//   v = q1 2^(E-20) + q2 2^(E-41) + q3 2^(E-62) + r,  |r| <= 2^(E-63),
// each q_l taken by rounding to the nearest integer (ties to even) and every
// remainder exact in FP32 (it is the difference of v and a multiple of a power
// of two at least as fine as v's own spacing, or v itself). Integer sums of the
// q_l do not depend on the order of the additions. E is clamped to [-60, 128]
// so that every scale is a normal FP32 number.
struct FxScale {
  float inv[3];   // 2^(20 - E), 2^(41 - E), 2^(62 - E)
  float step[3];  // 2^(E - 20), 2^(E - 41), 2^(E - 62)
};

__device__ __forceinline__ FxScale fx_scale(float bound) {
  int e = 0;
  if (bound > 0.f && isfinite(bound)) frexpf(bound, &e);  // bound < 2^e
  e = e < -60 ? -60 : (e > 128 ? 128 : e);
  FxScale f;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    f.inv[l] = ldexpf(1.f, 20 + 21 * l - e);
    f.step[l] = ldexpf(1.f, e - 20 - 21 * l);
  }
  return f;
}

// Adds the three integer parts of v to q (|v| <= 2^E of the scale).
__device__ __forceinline__ void fx_add(float v, const FxScale& f, int (&q)[3]) {
  constexpr float kMagic = 12582912.f;  // 1.5 2^23: y = kMagic + RN(v s) exactly while |v s| < 2^22
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const float y = fmaf(v, f.inv[l], kMagic);
    q[l] += __float_as_int(y) - __float_as_int(kMagic);
    v = fmaf(-(y - kMagic), f.step[l], v);  // exact remainder
  }
}

// The FP64 value of integer sums a[0..2] on the scale's grid (fixed order; each
// product exact, |a_l| < 2^53).
__device__ __forceinline__ double fx_value(long long a0, long long a1, long long a2, const FxScale& f) {
  return ((double)a0 * (double)f.step[0] + (double)a1 * (double)f.step[1]) + (double)a2 * (double)f.step[2];
}

// Lexicographic (value, index) order used by every argmin: lower value first,
// then lower index.
// A stage skips its work once the stop rule fired or an earlier stage of the
// same step recorded an error (its outputs, e.g. labels, are then not valid).
__device__ __forceinline__ bool halted(const Ctl* c) { return (c->done | c->error) != 0; }

__device__ __forceinline__ bool lex_less(float a, int ia, float b, int ib) {
  return a < b || (a == b && ia < ib);
}

// ---------------------------------------------------------------- SPADE downsampling (km_spade.cu)

constexpr int kSB = 1024;  // candidate rows per batch

// Device control block of one downsampling call.
struct SpadeCtl {
  int64_t cursor;                   // rows below it are settled
  int32_t nb;                       // candidates of the current batch
  int32_t overflow;                 // the batch's found-row list overflowed
  int32_t done;                     // a batch found no candidate
  int32_t nonfinite;                // X holds a NaN / Inf
  int32_t batches, overflow_batches;
  unsigned long long n_pairs;       // found-row pairs listed in the current batch (may exceed the capacity)
  unsigned long long n_exact;       // distances re-evaluated in FP64
  unsigned long long n_computed;    // candidate rows whose distances were computed
  unsigned long long n_evaluated;   // rows the loop evaluates
  unsigned long long n_apprx;       // (candidate, row) pairs within apprx_width, all batches
};

struct SpadeArgs {
  const float* X;
  int64_t n;
  int d;
  int vec;                      // rows start on 16-byte boundaries (d % 4 == 0, aligned X)
  float a_lo, a_hi, w_lo, w_hi;  // FP32 decision bands of D < apprx and D < cw
  float w_mid, w_half;          // [w_lo, w_hi] inside [w_mid - w_half, w_mid + w_half]
  double apprx, cw;             // the widths (cw: the counting width of the policy)
  int policy;                   // 0: last writer (overwrite), 1: first writer (fill if zero)
  int32_t none;                 // writer value of a row no evaluated row has found
  int32_t* q;                   // [n] writer of each row
  int32_t* slot;                // [n] position in the current batch, -1 otherwise
  int32_t* cand;                // [kSB] candidate rows
  int32_t* ccount;              // [kSB] their counts
  uint32_t* nbr;                // [kSB][kSB / 32] bit k' of row k: earlier candidate k' found by k
  uint8_t* inP;                 // [kSB] evaluated by the loop
  int2* pairs;                  // (candidate, row) pairs within apprx_width
  int64_t pair_cap;
  int32_t* counts;              // [n] count of each evaluated row, -1 otherwise
  uint8_t* processed;           // [n] 1 for evaluated rows
  SpadeCtl* ctl;
};

cudaError_t init_spade();
size_t spade_pairs_smem();
cudaError_t launch_spade_init(const SpadeArgs& A, cudaStream_t s);
// One batch: select, tile pass (between events e0 and e1 when given), resolve, apply, finish.
cudaError_t launch_spade_batch(const SpadeArgs& A, cudaStream_t s, cudaEvent_t e0 = nullptr,
                               cudaEvent_t e1 = nullptr);
cudaError_t launch_spade_density(const SpadeArgs& A, int32_t* dens, cudaStream_t s);

}  // namespace km
