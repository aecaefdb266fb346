/*
 * kmeans.h -- C ABI of the B300 fused Lloyd k-means library (libkmeans.so).
 *
 * One Lloyd iteration is the loop nest that the paper's fusion (Sec. 3.5)
 * collapses into a single pass over the points: for every point the distance
 * to every centroid (dist = norm(v1 - v2), Sec. 3.4), the argmin (a
 * DeliteCollectElem over the point range, Sec. 2.4), and a keyed reduce of
 * per-cluster sums and counts (DeliteReduceElem, Sec. 2.4), followed by the
 * per-cluster divide avg = sum / length (the VectorOpsExp listing, Sec. 2.1).
 *
 * Definitions shared by every entry point (X is n x d, C is k x d, both FP32
 * row-major; a is the assignment):
 *   a_i      = min { j : ||x_i - c_j||^2 <= ||x_i - c_j'||^2 for all j' }
 *              (squared Euclidean distance; the lowest index wins ties)
 *   counts_j = |{ i : a_i = j }|,   sums_j = sum_{a_i = j} x_i
 *   c_j'     = sums_j / counts_j, computed in FP64 and rounded to FP32;
 *              an empty cluster (counts_j = 0) keeps c_j
 *   J        = sum_i ||x_i - c_{a_i}||^2 with the centroids used for the
 *              assignment (reported in FP64)
 *
 * Accuracy contract (all precisions): a_i equals the exact argmin for every
 * point whose relative top-2 distance gap (D_(2) - D_(1)) / D_(2) is at least
 * 1e-6. Points whose low-precision top-2 margin falls under a bound derived
 * from the rounding errors are re-checked with compensated FP32 distances.
 * Every centroid coordinate is within 1e-5 of the exact member mean, relative
 * to the mean of |x_it| over the cluster's members.
 *
 * Memory and ownership: unless a function says otherwise, every array pointer
 * is a DEVICE pointer (cudaMalloc'd or managed) owned by the caller; the
 * library never frees it. The library owns only its workspace (cached per
 * device, grown on demand, released at process exit). X must not overlap any
 * output array. Arrays need only the alignment of their element type (4
 * bytes for float and int32): kernels that read X or C in 16-byte pieces
 * check the base address and fall back to 4-byte accesses.
 *
 * Streams: work is issued on opts->stream (NULL = the legacy default stream)
 * and the call synchronises that stream before it returns, so outputs and
 * statistics are complete on return. Calls on one device are serialised by
 * a library lock.
 *
 * Errors: every function returns a km_status. On KM_EINVAL / KM_EUNSUPPORTED
 * nothing was launched. On any other error the outputs are unspecified but C
 * holds its value on entry. kmeans_last_error() returns a thread-local
 * message for the last failing call of the calling thread.
 *
 * Preconditions: 1 <= k <= n < 2^31, 1 <= d <= 256, X and C finite with
 * ||x_i||^2 and ||c_j||^2 finite in FP32 (else KM_ENONFINITE).
 */
#ifndef KMEANS_H
#define KMEANS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KM_OK = 0,
  KM_EINVAL = -1,        /* bad argument: sizes, null or host pointer, overlap */
  KM_ECUDA = -2,         /* a CUDA runtime call failed */
  KM_ENOMEM = -3,        /* workspace allocation failed */
  KM_EUNSUPPORTED = -4,  /* valid but not supported (precision, shape) */
  KM_ETIMEOUT = -5,      /* a bounded device-side wait expired */
  KM_ENONFINITE = -6     /* X or C holds a NaN / Inf (or a norm overflows FP32) */
} km_status;

/* Arithmetic of the distance contraction. FP32 is exact up to FP32 rounding
 * (SIMT FFMA); BF16 and FP8 run on the tensor cores with FP32 accumulation
 * and per-row scales; all of them re-check near-ties in FP32.
 * KM_BF16X3 splits every FP32 value v into two BF16 parts, v ~ hi + lo with
 * hi = RN(v), lo = RN(v - hi), and forms x.c from the three products
 * hi.hi + lo.hi + hi.lo on the tensor cores (the dropped lo.lo term and the
 * residuals v - hi - lo enter the error bound), so that its near-tie margin is
 * about 2^-8 of the BF16 one at three times the tensor work. Single-instance
 * calls only; K blocks are 64 elements wide as for BF16. */
typedef enum { KM_FP32 = 0, KM_BF16 = 1, KM_FP8E4M3 = 2, KM_BF16X3 = 3 } km_precision;

typedef struct {
  int32_t precision;  /* km_precision; default KM_FP32 */
  int32_t recheck;    /* 1 (default): re-check flagged near-ties in FP32.
                         0: keep the low-precision argmin (no accuracy contract) */
  int32_t profile;    /* 1: time every stage with CUDA events recorded between
                         the stages (captured into the run's graph) and report
                         the per-stage totals in km_stats.stage_ms */
  int32_t warm_start; /* 1: assign holds a valid assignment on entry (e.g. the
                         previous step's). It seeds the tensor-core epilogue
                         threshold and n_changed counts against it. Labels
                         outside [0, k) are ignored. 0 (default): assign is
                         output only and every point counts as changed */
  int32_t deterministic; /* 1: bit-reproducible results. The keyed reduce adds the
                         points in exact fixed point (every coordinate split into
                         three 21-bit integer parts on a grid set by max_i ||x_i||,
                         summed in 64-bit integers, so the order of the additions
                         does not matter) and forms sums, centroids and the
                         objective from those integers in a fixed order; two calls
                         on the same inputs return identical bits. The dropped
                         remainder is below 2^-62 of max_i ||x_i|| per point.
                         Single-instance calls only (KM_EUNSUPPORTED for batches).
                         0 (default): Kahan-compensated FP32 runs combined with
                         FP64 atomics (within the accuracy contract, but the last
                         bit of a sum can depend on the order of the atomics) */
  int32_t reuse_x;    /* 1: X is the same array, with the same contents, n, d, k and
                         precision, as in this device's previous successful call
                         of kmeans_step_ex / kmeans_run_ex / kmeans_step_partial,
                         and no other call of the library used the device in
                         between: the point codes, norms and cluster-sorted order
                         that call left in the workspace are reused and the first
                         step continues from its last assignment (as a warm start
                         would), so that a sequence of one-step calls runs like
                         one kmeans_run. When the cache does not match, the flag
                         is ignored. 0 (default): everything is recomputed */
  void* stream;       /* cudaStream_t to issue work on; NULL = legacy stream */
} km_opts;

/* Stages of one Lloyd step, in launch order (indexes of km_stats.stage_ms).
 * KM_STAGE_XNORM runs once per call (point norms, hoisted out of the loop). */
enum {
  KM_STAGE_XNORM = 0,   /* ||x_i|| bounds and the finiteness check of X */
  KM_STAGE_PREP = 1,    /* centroid half-norms h_j and the error-bound maxima */
  KM_STAGE_ASSIGN = 2,  /* fused distance + argmin + near-tie flagging */
  KM_STAGE_RECHECK = 3, /* compensated FP32 re-check of flagged points */
  KM_STAGE_COUNT = 4,   /* cluster histogram */
  KM_STAGE_SCAN = 5,    /* segment offsets */
  KM_STAGE_SCATTER = 6, /* point indices sorted by cluster */
  KM_STAGE_SEGSUM = 7,  /* segmented sums and the objective */
  KM_STAGE_DIVIDE = 8,  /* FP64 divide, shift, stop rule */
  KM_NSTAGES = 9
};

/* Statistics of a call (the last step for the run variants). */
typedef struct {
  double objective;     /* J(a^t, C^t) of the last step, FP64 */
  double shift;         /* max_j ||c_j^{t+1} - c_j^t||_2 of the last step */
  int64_t n_changed;    /* points whose assignment changed in the last step
                           (all n in the first step of a call without
                           warm_start) */
  int64_t n_flagged;    /* points re-checked in FP32 in the last step */
  int64_t n_full;       /* of those, points re-checked against all k centroids */
  int32_t n_empty;      /* empty clusters after the last step */
  int32_t iters_done;   /* Lloyd steps executed */
  float ms;             /* device time of the call (CUDA events) */
  int32_t launches;     /* kernel launches of the call when its steps run as one
                           captured graph (iters > 1), else 0 */
  float stage_ms[12];   /* with opts->profile: device time per stage summed
                           over the call's steps (KM_STAGE_*), else zeros */
  int64_t n_queued;     /* of the n_full points of the last step, those gathered
                           and re-scored by the second pass before the compensated
                           distances (BF16 tensor-core codes for KM_FP8E4M3, the
                           FP32 SIMT kernel otherwise); 0 for batched calls */
  int32_t iters_bf16;   /* steps of the call whose distance contraction ran with
                           BF16 codes instead of the requested precision (1 for a
                           KM_FP8E4M3 call without warm_start: its first step) */
  int32_t batch_shape;  /* kmeans_run_batched: the autotuned launch shape, chunk
                           width + 1000 x instance order (0: as given, 1: by work
                           per tile) + 10000 x row order (0: every instance in
                           the order of X, 1: instances whose k spans several
                           chunks in the previous step's cluster-sorted order,
                           from a sorted copy of their codes); 0 for other
                           calls */
} km_stats;

/* Fills *opts with the defaults (FP32, recheck on, legacy stream). */
void kmeans_default_opts(km_opts* opts);

/*
 * One Lloyd step. X: const float[n*d]. C: float[k*d], in: the centroids used
 * for the assignment, out: the updated centroids. assign: int32[n] out.
 * sums: float[k*d] out (per-cluster sums of X, rounded from FP64 partials).
 * counts: int32[k] out.
 */
int kmeans_step(const float* X, int64_t n, int32_t d, float* C, int32_t k,
                int32_t* assign, float* sums, int32_t* counts);

/*
 * Up to `iters` Lloyd steps from C (iters >= 1). tol <= 0: exactly `iters`
 * steps. tol > 0: stop after the first step whose assignment equals the
 * previous step's, or whose largest centroid shift is <= tol. Outputs are
 * those of the last step executed. The iterations run as one captured CUDA
 * graph with the stop test evaluated on the device.
 */
int kmeans_run(const float* X, int64_t n, int32_t d, float* C, int32_t k,
               int32_t* assign, float* sums, int32_t* counts, int32_t iters,
               double tol);

/* As kmeans_step / kmeans_run with options (NULL = defaults) and statistics
 * (NULL = not wanted). */
int kmeans_step_ex(const km_opts* opts, const float* X, int64_t n, int32_t d,
                   float* C, int32_t k, int32_t* assign, float* sums,
                   int32_t* counts, km_stats* stats);
int kmeans_run_ex(const km_opts* opts, const float* X, int64_t n, int32_t d,
                  float* C, int32_t k, int32_t* assign, float* sums,
                  int32_t* counts, int32_t iters, double tol, km_stats* stats);

/*
 * As kmeans_run_ex, but every array is a HOST pointer (pageable or pinned).
 * The library copies X and C to device memory it owns, runs, and copies
 * C, assign, sums and counts back before returning.
 */
int kmeans_run_host(const km_opts* opts, const float* X, int64_t n, int32_t d,
                    float* C, int32_t k, int32_t* assign, float* sums,
                    int32_t* counts, int32_t iters, double tol, km_stats* stats);

/* One independent problem of a batch (device pointers, as for kmeans_run). */
typedef struct {
  const float* X;     /* float[n*d] */
  int64_t n;
  int32_t d;          /* 1 <= d <= 128 */
  int32_t k;          /* 1 <= k <= n */
  float* C;           /* float[k*d] in/out */
  int32_t* assign;    /* int32[n] out */
  float* sums;        /* float[k*d] out */
  int32_t* counts;    /* int32[k] out */
} km_instance;

/*
 * Up to `iters` Lloyd steps of every instance of a batch, each with its own
 * n, d and k, as one captured CUDA graph whose every stage is a single launch
 * over all instances (a persistent tensor-core launch over the row tiles of
 * every instance for the assignment). The stop rule (tol, as for kmeans_run)
 * applies per instance; a finished instance is skipped by later steps.
 * inst: HOST array of `count` descriptors. opts->precision must be KM_BF16 or
 * KM_FP8E4M3 (KM_EUNSUPPORTED otherwise). per_inst: NULL or a host array of
 * `count` statistics. The first call for a given batch shape tunes the launch
 * shape (tile-chunk width, tile order) by timing the candidates, and caches
 * the choice per shape for the life of the process. Instances must not share
 * output arrays.
 */
int kmeans_run_batched(const km_opts* opts, const km_instance* inst,
                       int32_t count, int32_t iters, double tol,
                       km_stats* per_inst);

/* ------------------------------------------------------------------------
 * Sharded Lloyd step (data-parallel over devices). The n points are split into
 * contiguous shards, one per device; every device holds all k centroids. One
 * step is: kmeans_step_partial on every shard, one sum all-reduce of the
 * partials buffer across the devices (the caller's collective, e.g. NCCL),
 * then kmeans_apply_partials with the reduced buffer on every device, which
 * gives every device the same new centroids. This is the keyed reduce split
 * into chunks whose per-chunk results are merged by a combine (Sec. 2.4,
 * DeliteReduceElem's alloc / combine), with the runtime spreading the loop
 * over several devices (Sec. 2.4, the Delite runtime).
 *
 * Partials buffer: double[KM_PARTIALS_LEN(k, d)] on the device,
 *   [0, k d)         sum of x_i over the shard's members of each cluster
 *                    (row-major k x d, FP64 from the reduce's partials),
 *   [k d, k d + k)   member counts (exact integers stored as FP64),
 *   [k d + k]        the shard's objective sum ||x_i - c_{a_i}||^2 (FP64),
 *   [k d + k + 1]    the shard's count of points whose assignment changed.
 * Every entry is a sum over points, so the element-wise sum of the shards'
 * buffers is the buffer of the whole data set.
 */
#define KM_PARTIALS_LEN(k, d) ((int64_t)(k) * (int64_t)(d) + (int64_t)(k) + 2)

/*
 * The shard's part of one Lloyd step: assignment (with the near-tie re-check
 * of opts->precision) and the partials buffer. X: const float[n*d] (the
 * shard's points), C: const float[k*d] (the centroids, unchanged), assign:
 * int32[n] out (with opts->warm_start: the previous labels on entry),
 * part: double[KM_PARTIALS_LEN(k, d)] out. All DEVICE pointers. stats: as for
 * kmeans_step_ex except shift and n_empty (0 here; see kmeans_apply_partials).
 * Use opts->reuse_x on the second and later steps of a sequence on the same
 * shard to keep the cached codes and cluster-sorted order.
 */
int kmeans_step_partial(const km_opts* opts, const float* X, int64_t n, int32_t d, const float* C,
                        int32_t k, int32_t* assign, double* part, km_stats* stats);

/*
 * The divide of a sharded step from a reduced partials buffer: for every
 * cluster with a nonzero count, c_j = RN32(sum_j / count_j) in FP64; an empty
 * cluster keeps c_j. part: const double[KM_PARTIALS_LEN(k, d)], C: float[k*d]
 * in/out, sums: float[k*d] out (the sums rounded to FP32) or NULL, counts:
 * int32[k] out or NULL; all DEVICE pointers. stats (NULL = not wanted):
 * objective and n_changed from the buffer, shift = max_j ||c_j' - c_j||_2,
 * n_empty; the other fields 0. Given the same buffer every device computes
 * the same bits. opts: only `stream` is used. Counts in the buffer must be
 * non-negative integers below 2^31 (KM_EINVAL otherwise, C unchanged).
 */
int kmeans_apply_partials(const km_opts* opts, const double* part, int32_t k, int32_t d, float* C,
                          float* sums, int32_t* counts, km_stats* stats);

/*
 * Keyed reduce of a Lloyd step for a given assignment, without allocating:
 * counts_j = |{i : a_i = j}|, sums_j = sum_{a_i = j} x_i (FP64 partials rounded
 * to FP32), *objective = sum_i ||x_i - c_{a_i}||^2 (FP64; objective may be NULL).
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory (a host framework that owns all device memory,
 * code that must not trigger cudaFree's device-wide synchronisation). It calls
 * no cudaMalloc / cudaFree; its scratch is a fixed ~10.5 MB static device array
 * that every GPU loading the library holds until exit. Limits: n <= 1048576,
 * k <= 8192, k * d <= 262144, 1 <= d <= 256; larger sizes return KM_EINVAL.
 * X: const float[n*d], C: const float[k*d], assign: const int32[n] with labels
 * in [0, k) (else KM_EINVAL), sums: float[k*d] out, counts: int32[k] out; all
 * device pointers. Work is issued on `stream` (NULL = legacy stream); every
 * call synchronises `stream` and reads a status word back before it returns,
 * so the call is synchronous and can never be recorded into a stream capture
 * or a CUDA graph. The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress, with that device current) and caches
 * it for the lifetime of the device's primary context (a cudaDeviceReset ends
 * both). Every call shares the one scratch array (it
 * clears what must start at zero, so a call rejected for a bad label leaves
 * nothing behind for the next one), and calls that overlap on the GPU race
 * with each other.
 */
int kmeans_reduce_noalloc(const float* X, int64_t n, int32_t d, const float* C,
                          int32_t k, const int32_t* assign, float* sums,
                          int32_t* counts, double* objective, void* stream);

/*
 * Keyed-reduce training of the paper's GPU classifiers (Sec. 5: naive Bayes and
 * Gaussian discriminant analysis): the keyed reduce of a Lloyd step (Sec. 2.4)
 * keyed by a class label y_i in [0, ncls) instead of the assignment. With
 * n_c = |{i : y_i = c}| and S_c = sum_{y_i = c} x_i (FP32 Kahan runs combined in
 * FP64, as the k-means sums):
 *
 * kmeans_gda_train -- shared-covariance GDA:
 *   phi[c] = n_c / n; mu[c] = S_c / n_c (0 for an empty class), rounded to FP32;
 *   sigma = (1/n) sum_i (x_i - mu_{y_i})(x_i - mu_{y_i})^T, d x d row-major,
 *   symmetric (FP32 partials over 64 rows, Kahan-added, combined in FP64, rounded
 *   to FP32; the same on every run).
 * kmeans_nb_train -- multinomial naive Bayes with add-one smoothing (X holds
 *   non-negative feature counts):
 *   prior[c] = n_c / n; theta[c][j] = (S_cj + 1) / (sum_j S_cj + d).
 *
 * X: const float[n*d] row-major, y: const int32[n]; outputs phi/prior float[ncls],
 * mu/theta float[ncls*d], sigma float[d*d]; all device pointers owned by the
 * caller. 1 <= n < 2^31, 1 <= d <= 256, 1 <= ncls <= 2^20; a label outside
 * [0, ncls) gives KM_EINVAL (outputs unspecified). opts: only `stream` is used
 * (NULL opts = defaults); the stream is synchronised before returning. The
 * library's workspace is reused (grown with cudaMalloc when needed).
 */
int kmeans_gda_train(const km_opts* opts, const float* X, int64_t n, int32_t d,
                     const int32_t* y, int32_t ncls, float* phi, float* mu, float* sigma);
int kmeans_nb_train(const km_opts* opts, const float* X, int64_t n, int32_t d,
                    const int32_t* y, int32_t ncls, float* prior, float* theta);

/* ------------------------------------------------------------------------
 * SPADE density downsampling (Sec. 4.1, "Downsampling in Bioinformatics"),
 * the paper's second fused-loop workload, on the same library.
 *
 * With D(i, j) = sum_t |x_it - x_jt| evaluated in FP64 (columns in increasing
 * order) over the rows of X (n x d, FP32, row-major, DEVICE), the result is
 * that of the paper's loop run sequentially over i = 0..n-1:
 *   if the density of row i is still 0, row i is evaluated: its count
 *   c = #{j : D(i, j) < kernel_width} (policy KM_SPADE_FIRST also counts
 *   D < apprx_width, as the C++ snippet's else-if does), and every row j with
 *   D(i, j) < apprx_width gets density c: always (KM_SPADE_LAST, the
 *   generated code's bulk update) or only while its density is still 0
 *   (KM_SPADE_FIRST, the snippet's compare-and-swap).
 * Every threshold decision equals the FP64 loop's (pairs whose FP32 distance
 * lies within the rounding bound of a width are re-evaluated in FP64).
 *
 * Outputs (DEVICE, caller-owned): densities int32[n]; counts int32[n] or NULL
 * (c of every evaluated row, -1 for skipped rows); processed uint8[n] or NULL
 * (1 for evaluated rows). stats: HOST pointer or NULL.
 * Preconditions: 1 <= n < 2^31 - 1, 1 <= d <= 4096, apprx_width and
 * kernel_width finite and > 0, policy KM_SPADE_LAST or KM_SPADE_FIRST
 * (KM_EINVAL otherwise); X finite (KM_ENONFINITE otherwise). opts: only
 * opts->stream is used (NULL = defaults); the call synchronises that stream.
 * Workspace (about 13 n bytes + 64 MiB) is owned by the library and reused.
 */
typedef enum { KM_SPADE_LAST = 0, KM_SPADE_FIRST = 1 } km_spade_policy;

typedef struct {
  int64_t n_evaluated;   /* rows the loop evaluates (density still 0 when reached) */
  int64_t n_computed;    /* rows whose distances were computed: evaluated rows plus
                            candidates of a batch that an earlier evaluated
                            candidate of the same batch turned out to find */
  int64_t n_found_pairs; /* (computed row, row) pairs within apprx_width */
  int64_t n_exact;       /* distances re-evaluated in FP64 near a width */
  int32_t batches;       /* candidate batches */
  int32_t overflow_batches; /* batches whose found-row list overflowed (slower path) */
  float ms;              /* device time of the call */
  float ms_pairs;        /* device time of the tile passes (CUDA events around each) */
} km_spade_stats;

int kmeans_spade_densities(const km_opts* opts, const float* X, int64_t n, int32_t d, double apprx_width,
                           double kernel_width, int32_t policy, int32_t* densities, int32_t* counts,
                           uint8_t* processed, km_spade_stats* stats);

/* ------------------------------------------------------------------------
 * Diagnostics (not on the Lloyd path; used by the tests and the benchmark).
 *
 * kmeans_probe_mma: one 128 x 128 FP32 tile D = A B^T of the tensor-core
 * contraction formed exactly as the distance kernel forms it (operands staged
 * K-major with the 128-byte swizzle, the kernel's shared-memory and
 * instruction descriptors, one tcgen05.mma per 32 bytes of K accumulating in
 * K order into one TMEM accumulator, read back with tcgen05.ld). It exposes
 * the accumulator's rounding, on which the near-tie margin's gamma'_K term
 * rests. precision: KM_BF16 (A, B hold BF16 bit patterns, 2 bytes) or
 * KM_FP8E4M3 (E4M3 bytes). A: DEVICE [128][K] codes, B: DEVICE [128][K]
 * codes, both row-major, 16-byte aligned; K = 64, 128, 192 or 256 (BF16) or
 * 128, 256, 384 or 512 (E4M3). D: DEVICE float[128 * 128], D[m*128 + n] =
 * sum_k A[m][k] B[n][k] as accumulated by the tensor core. The call
 * synchronises `stream` (NULL = legacy stream). KM_EINVAL for bad sizes,
 * KM_ETIMEOUT if the completion wait (bounded at 1 s) expired.
 *
 * kmeans_probe_ffma: times one launch of independent FP32 FMA chains over
 * every SM (8 CTAs of 256 threads per SM, 16 FMAs per thread and iteration,
 * `iters` iterations; packed != 0 uses the two-lane FFMA2 instruction) with
 * CUDA events on `stream`. *flops = 2 x FMAs executed, *ms = device time: the
 * measured FP32 SIMT peak is *flops / *ms.
 */
int kmeans_probe_mma(int32_t precision, const void* A, const void* B, int32_t K, float* D, void* stream);
int kmeans_probe_ffma(int32_t packed, int32_t iters, double* flops, float* ms, void* stream);

/* Message of the calling thread's last failing call ("" if none). */
const char* kmeans_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int32_t kmeans_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KMEANS_H */
