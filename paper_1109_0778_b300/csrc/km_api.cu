// C ABI of the fused Lloyd k-means library: argument validation, the per-device
// context and workspace, the stage sequence of one Lloyd step, graph capture of
// multi-step runs, and statistics. Declarations and contracts: include/kmeans.h.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <functional>
#include <initializer_list>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "km_internal.cuh"
#include "km_tc.cuh"

#define KM_API extern "C" __attribute__((visibility("default")))

namespace km {

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

}  // namespace km

namespace {

using namespace km;

thread_local std::string g_err;

}  // namespace

void km::set_last_error(const char* msg) { g_err = msg; }

namespace {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define KM_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(KM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                 \
  } while (0)

struct GraphKey {
  const void *X, *C, *assign, *sums, *counts;
  int64_t n;
  int d, k, iters, prec, profile;
  double tol;
  uint64_t ws_gen;
  bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof o) == 0; }
};

struct DevCtx {
  std::mutex mu;
  int dev = -1;
  bool inited = false;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t ws_gen = 0;
  void* stage = nullptr;  // device copies for the host-pointer entry point
  void* cls = nullptr;    // class counts and covariance accumulators of the training entry points
  size_t cls_bytes = 0;
  void* spade = nullptr;  // downsampling state (km_spade.cu)
  size_t spade_bytes = 0;
  size_t stage_bytes = 0;
  void* host = nullptr;   // pinned read-back of Ctl and the per-step history
  size_t host_bytes = 0;
  bool graph_valid = false;
  // What the workspace holds after the last successful single-instance call
  // (opts->reuse_x): point codes, norms and cluster-sorted order of that X.
  struct XCache {
    bool valid = false;
    const void* X = nullptr;
    int64_t n = 0;
    int d = 0, k = 0, prec = -1, lay_warm = 0, det = 0;
    uint64_t ws_gen = 0;
  } xc;
  unsigned long long* actl = nullptr;  // status words of kmeans_apply_partials
  int graph_kernels = 0;  // kernel nodes of the cached graph
  GraphKey gkey{};
  cudaGraphExec_t gexec = nullptr;
  std::vector<cudaEvent_t> prof;  // stage-boundary events of profiled calls
};

constexpr int kEvPerStep = 9;  // boundaries of the 8 per-step stages

int ensure_events(DevCtx* c, size_t count) {
  while (c->prof.size() < count) {
    cudaEvent_t e;
    KM_CUDA(cudaEventCreate(&e));
    c->prof.push_back(e);
  }
  return KM_OK;
}

// Records a stage boundary; inside a stream capture the record becomes an
// event node of the graph so that graph replays time their stages too.
cudaError_t mark(cudaEvent_t e, cudaStream_t s) {
  if (!e) return cudaSuccess;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(s, &cs);
  if (r != cudaSuccess) return r;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

std::mutex g_ctx_mu;
DevCtx* g_ctx[64] = {nullptr};

DevCtx* get_ctx(int dev) {
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  if (!g_ctx[dev]) {
    g_ctx[dev] = new DevCtx();
    g_ctx[dev]->dev = dev;
  }
  return g_ctx[dev];
}

int init_ctx(DevCtx* c) {
  if (c->inited) return KM_OK;
  KM_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  KM_CUDA(cudaEventCreate(&c->ev0));
  KM_CUDA(cudaEventCreate(&c->ev1));
  KM_CUDA(init_assign_simt());
  KM_CUDA(init_assign_tc());
  KM_CUDA(init_segsum());
  KM_CUDA(init_batched());
  KM_CUDA(init_spade());
  c->inited = true;
  return KM_OK;
}

size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

// Shape of the tensor-core path for (d, k, precision).
// Kp: d padded to whole 128-byte K blocks; Kw: elements of one point code row
// (Kp, or 2 Kp for the two-part BF16 codes); nkb: K blocks of one point code
// row. fold (128-centroid chunks): every centroid also has a 16-element BF16
// slice holding -h_j (E4M3: -h_j / s_c; Hc, staged with the 32-byte swizzle),
// contracted with a slice of ones (E4M3: each point row's [1/s_x, ...] slice,
// Xh) by one BF16 MMA step on the same accumulator, so the accumulators hold
// (x.c_j - h_j) / (s_x s_c) and the epilogue takes no h_j and no multiply-add.
// Kc: elements of one centroid code row.
struct TcShape {
  int fp8, split, esz, Kp, Kw, nkb, bn, kp, nchunks, stages, abufs, fold, Kc;
  int qmode() const { return split ? 2 : fp8 ? 1 : 0; }  // quantisation stage mode
};

TcShape tc_shape(int precision, int d, int k) {
  TcShape t{};
  t.fp8 = precision == KM_FP8E4M3;
  t.split = precision == KM_BF16X3;
  t.esz = t.fp8 ? 1 : 2;
  const int kbe = 128 / t.esz;
  t.Kp = (d + kbe - 1) / kbe * kbe;
  t.Kw = t.split ? 2 * t.Kp : t.Kp;
  t.nkb = t.Kw / kbe;
  t.kp = (k + 127) / 128 * 128;  // padded to whole chunks of any width
  t.Kc = t.Kw;
  t.fold = 0;
  if (!t.split && t.nkb <= 2) {  // BF16 / E4M3, 128-centroid chunks, -h_j folded in when it fits
    t.bn = 128;
    t.nchunks = t.kp / 128;
    t.stages = tc_pick_buffers(t.nkb, 128, t.kp, t.fp8, &t.abufs, 1);
    if (t.stages >= 2) {
      t.fold = 1;
      return t;
    }
  }
  // chunk width: 128 centroids for short rows, else 64; 32 when only that
  // leaves room for two B stages (the widest two-part codes)
  for (int bn = t.nkb <= 2 ? 128 : 64; bn >= 32; bn /= 2) {
    t.bn = bn;
    t.nchunks = t.kp / t.bn;
    // dynamic shared memory: A slots, B stages, h_j (and scales)
    t.stages = tc_pick_buffers(t.nkb, t.bn, t.kp, t.fp8, &t.abufs);
    if (t.stages >= 2 || (!t.split && bn == 64)) break;
  }
  return t;
}

// A cold E4M3 run does its first step with BF16 codes (far fewer near
// candidates without a previous assignment); later steps use E4M3 codes that the
// first step's reduce stage writes in sorted order.
bool cold_bf16_first(int precision, int warm, int d, int k) {
  return precision == KM_FP8E4M3 && !warm && tc_shape(KM_BF16, d, k).stages >= 2;
}

struct Layout {
  size_t ctl, xnorm, flags, perm, offs, cursor, sums64, chalf, cnorm, Csave, obj, shift, changed,
      flagged, full, empty, queued, Xq, xs, xs16, Cq, hq, scq, state, state3, xss, labs, fq_rows, fq_old, X_sub, xn_sub,
      flags2, xq16, xs16q, cq16, hq16, scq16, hc, hc16, xh, pcounts, xmax, facc, oacc, small, cst, cst16, mu, total;
  int64_t fq_cap;
  int Kp16;  // BF16 code width of an E4M3 run's re-check codes (0: none)
};

// E4M3 runs re-score queued points with BF16 codes on the tensor cores when that shape fits.
bool rescore16(int precision, int d, int k) { return precision == KM_FP8E4M3 && tc_shape(KM_BF16, d, k).stages >= 2; }

// Rows the re-check queue of the quantised paths holds: an eighth of the points
// (at least 4096, at most n); further unresolved points are settled one by one.
int64_t requeue_cap(int64_t n) { return std::min<int64_t>(n, std::max<int64_t>(4096, n / 8)); }

// Regions whose contents a later call may reuse (opts->reuse_x: codes, norms,
// sorted order) come first and depend only on (n, k, d, precision, warm); the
// per-step histories (sized by iters) and the deterministic accumulators follow.
Layout layout_for(int64_t n, int k, int d, int iters, int precision, int warm, int det) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
  const size_t kd = (size_t)k * d;
  L.ctl = take(sizeof(Ctl));
  L.xnorm = take(4 * (size_t)n);
  L.flags = take(sizeof(FlagRec) * (size_t)n);
  L.perm = take(4 * (size_t)n);
  L.offs = take(4 * ((size_t)k + 1));
  L.cursor = take(4 * (size_t)k);
  L.sums64 = take(8 * kd);
  L.chalf = take(4 * (size_t)k);
  L.cnorm = take(4 * (size_t)k);
  L.Csave = take(4 * kd);
  L.pcounts = take(4 * (size_t)k);
  L.xmax = take(4);
  L.labs = take(4 * (size_t)n);  // labels in cluster-sorted order (scatter stage)
  if (precision != KM_FP32) {
    const TcShape t = tc_shape(precision, d, k);
    size_t xq = (size_t)n * t.Kw * t.esz, cq = (size_t)t.kp * t.Kc * t.esz;
    const bool cold = cold_bf16_first(precision, warm, d, k);
    if (cold) {
      const TcShape t16 = tc_shape(KM_BF16, d, k);
      xq = std::max(xq, (size_t)n * t16.Kp * 2);
      cq = std::max(cq, (size_t)t16.kp * t16.Kc * 2);
    }
    L.Xq = take(xq);
    L.xs = take(16 * (size_t)n);
    L.mu = take(4 * (size_t)d);  // the codes' centring vector (reused with them)
    L.xs16 = cold ? take(16 * (size_t)n) : 0;
    L.Cq = take(cq);
    // -h_j slices of the folded BF16 contraction (the main shape, or the BF16 first step of a cold call)
    const bool hfold = t.fold || (cold && tc_shape(KM_BF16, d, k).fold);
    L.hc = hfold ? take(32 * (size_t)std::max(t.kp, tc_shape(KM_BF16, d, k).kp)) : 0;
    L.xh = (t.fp8 && t.fold) ? take(32 * (size_t)n) : 0;  // the points' 1/s_x slices (folded E4M3)
    L.hq = take(4 * (size_t)t.kp);
    L.scq = take(4 * (size_t)t.kp);
    // per-centroid error terms of the main codes (or of a cold call's BF16 first step)
    L.cst = take(16 * (size_t)std::max(t.kp, tc_shape(KM_BF16, d, k).kp));
    L.xss = take(16 * (size_t)n);
    L.fq_cap = requeue_cap(n);
    L.fq_rows = take(4 * (size_t)L.fq_cap);
    L.fq_old = take(4 * (size_t)L.fq_cap);
    L.X_sub = take(4 * (size_t)L.fq_cap * d);
    L.xn_sub = take(4 * (size_t)L.fq_cap);
    L.flags2 = take(sizeof(FlagRec) * (size_t)L.fq_cap);
    const int width = simt_slab_width(d);  // the queued rows' FP32 pass may carry state across slabs
    L.state = (width > 0 && width < k) ? take(16 * (size_t)L.fq_cap) : 0;
    L.state3 = (width > 0 && width < k) ? take(4 * (size_t)L.fq_cap) : 0;
    if (rescore16(precision, d, k)) {
      const TcShape t16 = tc_shape(KM_BF16, d, k);
      L.Kp16 = t16.Kp;
      L.xq16 = take((size_t)L.fq_cap * t16.Kp * 2);
      L.xs16q = take(16 * (size_t)L.fq_cap);
      L.cq16 = take((size_t)t16.kp * t16.Kc * 2);
      L.hc16 = t16.fold ? take(32 * (size_t)t16.kp) : 0;
      L.hq16 = take(4 * (size_t)t16.kp);
      L.scq16 = take(4 * (size_t)t16.kp);
      L.cst16 = take(16 * (size_t)t16.kp);
    } else {
      L.Kp16 = 0;
      L.xq16 = L.xs16q = L.cq16 = L.hq16 = L.scq16 = L.hc16 = L.cst16 = 0;
    }
  } else {
    L.hc = L.hc16 = L.xh = 0;
    L.Kp16 = 0;
    L.xq16 = L.xs16q = L.cq16 = L.hq16 = L.scq16 = L.cst = L.cst16 = 0;
    L.Xq = L.xs = L.xs16 = L.Cq = L.hq = L.scq = L.xss = L.mu = 0;
    const int width = simt_slab_width(d);
    L.state = (width > 0 && width < k) ? take(16 * (size_t)n) : 0;  // also serves the re-check pass
    if (width > 0) {
      // flagged points are gathered and re-scored by the slab kernel keeping two candidates and a third score
      L.fq_cap = requeue_cap(n);
      L.fq_rows = take(4 * (size_t)L.fq_cap);
      L.fq_old = take(4 * (size_t)L.fq_cap);
      L.X_sub = take(4 * (size_t)L.fq_cap * d);
      L.xn_sub = take(4 * (size_t)L.fq_cap);
      L.flags2 = take(sizeof(FlagRec) * (size_t)L.fq_cap);
      L.state3 = width < k ? take(4 * (size_t)L.fq_cap) : 0;
    } else {
      L.fq_rows = L.fq_old = L.X_sub = L.xn_sub = L.flags2 = L.state3 = 0;
      L.fq_cap = 0;
    }
  }
  L.obj = take(8 * (size_t)iters);
  L.shift = take(8 * (size_t)iters);
  L.changed = take(8 * (size_t)iters);
  L.flagged = take(8 * (size_t)iters);
  L.full = take(8 * (size_t)iters);
  L.empty = take(4 * (size_t)iters);
  L.queued = take(8 * (size_t)iters);
  L.facc = det ? take(3 * 8 * kd) : 0;
  L.oacc = det ? take(3 * 8) : 0;
  L.small = (precision == KM_FP32 && small_path_fits(n, d, k)) ? take(small_scratch_bytes(n, d, k)) : 0;
  L.total = o;
  return L;
}

// Grows the workspace (never shrinks); sums64 must start at zero.
int ensure_ws(DevCtx* c, const Layout& L, cudaStream_t s) {
  if (L.total > c->ws_bytes) {
    if (c->ws) {
      KM_CUDA(cudaDeviceSynchronize());
      cudaFree(c->ws);
      c->ws = nullptr;
      c->ws_bytes = 0;
    }
    size_t want = align_up(L.total + L.total / 4, 1 << 20);
    if (cudaMalloc(&c->ws, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "workspace allocation of %zu bytes failed", want);
    }
    c->ws_bytes = want;
    c->ws_gen++;
    c->graph_valid = false;
    KM_CUDA(cudaMemsetAsync(c->ws, 0, want, s));
  }
  return KM_OK;
}

Work make_work(DevCtx* c, const Layout& L) {
  char* b = (char*)c->ws;
  Work w;
  w.ctl = (Ctl*)(b + L.ctl);
  w.xnorm = (float*)(b + L.xnorm);
  w.flags = (FlagRec*)(b + L.flags);
  w.perm = (int32_t*)(b + L.perm);
  w.offs = (int32_t*)(b + L.offs);
  w.cursor = (int32_t*)(b + L.cursor);
  w.sums64 = (double*)(b + L.sums64);
  w.chalf = (float*)(b + L.chalf);
  w.cnorm = (float*)(b + L.cnorm);
  w.Csave = (float*)(b + L.Csave);
  w.obj_hist = (double*)(b + L.obj);
  w.shift_hist = (double*)(b + L.shift);
  w.changed_hist = (unsigned long long*)(b + L.changed);
  w.flagged_hist = (unsigned long long*)(b + L.flagged);
  w.full_hist = (unsigned long long*)(b + L.full);
  w.empty_hist = (int*)(b + L.empty);
  w.queued_hist = (unsigned long long*)(b + L.queued);
  w.pcounts = (int32_t*)(b + L.pcounts);
  w.xmax = (unsigned int*)(b + L.xmax);
  w.facc = L.facc ? (unsigned long long*)(b + L.facc) : nullptr;
  w.oacc = L.oacc ? (unsigned long long*)(b + L.oacc) : nullptr;
  w.small = L.small ? (void*)(b + L.small) : nullptr;
  w.Xq = L.Xq ? (uint8_t*)(b + L.Xq) : nullptr;
  w.xs = L.xs ? (float4*)(b + L.xs) : nullptr;
  w.Cq = L.Cq ? (uint8_t*)(b + L.Cq) : nullptr;
  w.hq = L.hq ? (float*)(b + L.hq) : nullptr;
  w.scq = L.scq ? (float*)(b + L.scq) : nullptr;
  w.cst = L.cst ? (float4*)(b + L.cst) : nullptr;
  w.mu = L.mu ? (float*)(b + L.mu) : nullptr;
  w.Hc = L.hc ? (void*)(b + L.hc) : nullptr;
  w.Xh = L.xh ? (void*)(b + L.xh) : nullptr;
  w.state = L.state ? (float4*)(b + L.state) : nullptr;
  w.state3 = L.state3 ? (float*)(b + L.state3) : nullptr;
  w.xs16 = L.xs16 ? (float4*)(b + L.xs16) : nullptr;
  w.xs_sorted = L.xss ? (float4*)(b + L.xss) : nullptr;
  w.lab_sorted = L.labs ? (int32_t*)(b + L.labs) : nullptr;
  w.fq_cap = L.fq_cap;
  w.fq_rows = L.fq_rows ? (int32_t*)(b + L.fq_rows) : nullptr;
  w.fq_old = L.fq_old ? (int32_t*)(b + L.fq_old) : nullptr;
  w.X_sub = L.X_sub ? (float*)(b + L.X_sub) : nullptr;
  w.xn_sub = L.xn_sub ? (float*)(b + L.xn_sub) : nullptr;
  w.flags2 = L.flags2 ? (FlagRec*)(b + L.flags2) : nullptr;
  w.Xq16 = L.xq16 ? (uint8_t*)(b + L.xq16) : nullptr;
  w.xs16q = L.xs16q ? (float4*)(b + L.xs16q) : nullptr;
  w.Kp16 = L.Kp16;
  return w;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D K-major code matrix [rows][Kp] -> boxes of (128 bytes of K) x box_rows, 128-byte swizzle.
// Codes [rows][Kp] -> boxes of rowb bytes (128: the 128-byte swizzle; 64 / 32: a
// single block of the 64- / 32-byte swizzle, Kp * esz == rowb) x box_rows.
int encode_codes_map(CUtensorMap* m, void* base, int64_t rows, int Kp, int esz, int box_rows, int rowb = 128) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(KM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (rowb != 128 && Kp * esz != rowb) return fail(KM_EINVAL, "code rows of %d bytes in %d-byte boxes", Kp * esz, rowb);
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
  cuuint32_t box[2] = {(cuuint32_t)(rowb / esz), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapSwizzle sw =
      rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : rowb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r = enc(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                   rowb == 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(KM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KM_OK;
}

// [rows][16] BF16 -h_j slices -> boxes of 16 elements (32 B) x box_rows, 32-byte swizzle.
int encode_h_map(CUtensorMap* m, void* base, int64_t rows, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(KM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {16, (cuuint64_t)rows};
  cuuint64_t strides[1] = {32};
  cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(KM_ECUDA, "cuTensorMapEncodeTiled (h slices) failed (%d)", (int)r);
  return KM_OK;
}

// Per-call state of a step sequence: precision, recheck switch, tensor-core launch data.
struct StepCfg {
  int precision;
  int recheck;
  int warm;  // assign holds a valid assignment on entry
  int det;   // exact fixed-point reduce (opts->deterministic)
  int reuse; // the first step continues from the cached sorted codes and labels of the previous call
  double* part;  // non-null: a shard's partial step (no divide; partials into part)
  TcShape t;
  TcLaunch L;
  TcParams P;
  bool cold;  // first step with BF16 codes (E4M3 runs without a warm start)
  TcShape t0;
  TcLaunch L0;
  TcParams P0;
  // E4M3 runs: BF16 re-score of the queued points (centroid codes Cq16 / hq16 / scq16)
  bool rs16;
  TcShape t16;
  TcLaunch L16;
  TcParams P16;
  uint8_t* Cq16;
  void* Hc16;  // -h_j slices of the re-score codes (folded BF16), null otherwise
  float *hq16, *scq16;
  float4* cst16;
};

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char *pa = (const char*)a, *pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

int check_device_ptr(const void* p, const char* name, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(KM_EINVAL, "%s is not a CUDA-accessible pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(KM_EINVAL, "%s is not device memory (use kmeans_run_host for host arrays)", name);
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    return fail(KM_EINVAL, "%s lives on device %d, the current device is %d", name, at.device, dev);
  return KM_OK;
}

// Argument checks that need no CUDA call: sizes, iterations, precision and shape.
int validate_shape(const km_opts& o, const Problem& p, int iters) {
  if (p.n < 1 || p.n > INT32_MAX) return fail(KM_EINVAL, "n = %lld outside [1, 2^31)", (long long)p.n);
  if (p.k < 1 || (int64_t)p.k > p.n) return fail(KM_EINVAL, "k = %d outside [1, n]", p.k);
  if (p.d < 1 || p.d > kMaxD) return fail(KM_EINVAL, "d = %d outside [1, %d]", p.d, kMaxD);
  if (iters < 1) return fail(KM_EINVAL, "iters = %d < 1", iters);
  if (o.precision != KM_FP32 && o.precision != KM_BF16 && o.precision != KM_FP8E4M3 && o.precision != KM_BF16X3)
    return fail(KM_EINVAL, "unknown precision %d", o.precision);
  if (o.precision != KM_FP32 && tc_shape(o.precision, p.d, p.k).stages < 2)
    return fail(KM_EUNSUPPORTED, "d = %d, k = %d do not fit the tensor-core tile pipeline (k is staged in shared memory)",
                p.d, p.k);
  return KM_OK;
}

// Argument checks that need no CUDA call.
int validate_args(const km_opts& o, const Problem& p, int iters) {
  if (!p.X || !p.C || !p.assign || !p.sums || !p.counts) return fail(KM_EINVAL, "null array pointer");
  int rc = validate_shape(o, p, iters);
  if (rc) return rc;
  const size_t nd = (size_t)p.n * p.d * 4, kd = (size_t)p.k * p.d * 4;
  const size_t na = (size_t)p.n * 4, nk = (size_t)p.k * 4;
  if (overlaps(p.X, nd, p.C, kd) || overlaps(p.X, nd, p.assign, na) || overlaps(p.X, nd, p.sums, kd) ||
      overlaps(p.X, nd, p.counts, nk) || overlaps(p.C, kd, p.assign, na) || overlaps(p.C, kd, p.sums, kd) ||
      overlaps(p.C, kd, p.counts, nk) || overlaps(p.assign, na, p.sums, kd) ||
      overlaps(p.assign, na, p.counts, nk) || overlaps(p.sums, kd, p.counts, nk))
    return fail(KM_EINVAL, "arrays overlap");
  return KM_OK;
}

int validate_device_ptrs(const Problem& p, int dev) {
  int rc;
  if ((rc = check_device_ptr(p.X, "X", dev))) return rc;
  if ((rc = check_device_ptr(p.C, "C", dev))) return rc;
  if ((rc = check_device_ptr(p.assign, "assign", dev))) return rc;
  if ((rc = check_device_ptr(p.sums, "sums", dev))) return rc;
  if ((rc = check_device_ptr(p.counts, "counts", dev))) return rc;
  return KM_OK;
}

// The stage sequence of one Lloyd step (all on stream s). With `ev`
// (kEvPerStep events) every stage boundary is recorded.
// `sorted`: the point codes are in the previous step's cluster-sorted order
// (row p = point perm[p]), written by that step's reduce stage.
// KM_DEBUG_SYNC: launch stage by stage, synchronising after each one and
// naming the first stage whose launch or execution fails (diagnosis only).
bool debug_sync() {
  static const bool on = getenv("KM_DEBUG_SYNC") != nullptr;
  return on;
}

cudaError_t enqueue_step(const Problem& p, const Work& w, const StepCfg& cfg, int first, int sorted, double tol,
                         cudaStream_t s, const cudaEvent_t* ev) {
  cudaError_t e;
  static const char* names[] = {"prep", "assign", "recheck", "count", "scan", "scatter", "segsum", "divide"};
  auto at = [&](int i) -> cudaError_t {
    if (debug_sync() && i > 0) {
      cudaError_t r = cudaStreamSynchronize(s);
      if (r == cudaSuccess) r = cudaGetLastError();
      fprintf(stderr, "[kmeans] stage %s (step first=%d sorted=%d): %s\n", names[i - 1], first, sorted,
              cudaGetErrorString(r));
      if (r != cudaSuccess) return r;
    }
    return ev ? mark(ev[i], s) : cudaSuccess;
  };
  const bool tcp = cfg.precision != KM_FP32;
  const bool cold = tcp && cfg.cold && !sorted;  // this step runs on the cold-start BF16 codes
  const TcShape& t = cold ? cfg.t0 : cfg.t;
  if ((e = cudaMemsetAsync(w.ctl, 0, kCtlIterBytes, s))) return e;
  if ((e = at(0))) return e;
  if (tcp) e = launch_quant_c(p, w, t.qmode(), t.kp, t.Kp, w.Cq, t.fold ? w.Hc : nullptr, w.hq, w.scq, w.cst, s);
  else e = launch_prep(p, w, s);
  if (e) return e;
  if ((e = at(1))) return e;
  if (tcp) {
    TcParams P = cold ? cfg.P0 : cfg.P;
    P.first = first;
    P.rows = sorted ? w.perm : nullptr;
    P.xs_sorted = w.xs_sorted;
    P.lab_sorted = w.lab_sorted;
    e = launch_assign_tc(p, cold ? cfg.L0 : cfg.L, P, s);
  } else {
    e = launch_assign_simt(p, w, first, s);
  }
  if (e) return e;
  if ((e = at(2))) return e;
  if (cfg.recheck) {
    std::function<cudaError_t(cudaStream_t)> tc16;
    if (cfg.rs16 && !cold)
      tc16 = [&](cudaStream_t st) {
        const TcShape& t16 = cfg.t16;
        cudaError_t r = launch_quant_c(p, w, 0, t16.kp, t16.Kp, cfg.Cq16, t16.fold ? cfg.Hc16 : nullptr, cfg.hq16,
                                       cfg.scq16, cfg.cst16, st, true);
        if (r != cudaSuccess) return r;
        Problem q = p;
        q.n = w.fq_cap;
        TcParams P = cfg.P16;
        P.first = first;
        return launch_assign_tc(q, cfg.L16, P, st);
      };
    if ((e = launch_recheck(p, w, w.chalf, first, s, tc16))) return e;  // (uncentred h_j: it scores x itself)
  }
  if ((e = at(3))) return e;
  if ((e = launch_count(p, w, s))) return e;
  if ((e = at(4))) return e;
  if ((e = launch_scan(p, w, s))) return e;
  if ((e = at(5))) return e;
  if ((e = launch_scatter(p, w, s))) return e;
  if ((e = at(6))) return e;
  if ((e = launch_segsum(p, w, s, tcp ? cfg.t.qmode() + 1 : 0, tcp ? cfg.t.Kp : 0, cfg.det))) return e;
  if ((e = at(7))) return e;
  if (cfg.part) e = launch_finish_partial(p, w, cfg.part, cfg.det, s);
  else e = launch_divide(p, w, first ? 0 : 1, tol, s, cfg.det);
  if (e) return e;
  if ((e = at(8))) return e;
  return cudaSuccess;
}

// Whether a step of the call starts from the unsorted point codes and no
// previous labels (`first`), and whether its rows are in the previous step's
// cluster-sorted order (`sorted`: the quantised paths after their first step,
// and from the first step on when the call reuses the previous call's codes).
int step_first(const StepCfg& cfg, int it) {
  return it == 0 && !cfg.warm && !(cfg.reuse && cfg.precision != KM_FP32);
}
int step_sorted(const StepCfg& cfg, int it) { return it > 0 || (cfg.reuse && cfg.precision != KM_FP32); }

const cudaEvent_t* step_events(DevCtx* c, bool profile, int it) {
  return profile ? c->prof.data() + 2 + (size_t)it * kEvPerStep : nullptr;
}

// Kernel nodes of a captured graph (the launches one replay makes).
int kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  int k = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
      }
  }
  cudaGetLastError();
  return k;
}

int get_graph(DevCtx* c, const GraphKey& key, const Problem& p, const Work& w, const StepCfg& cfg, int iters,
              double tol, bool profile, cudaGraphExec_t* out) {
  if (c->graph_valid && c->gkey == key) {
    *out = c->gexec;
    return KM_OK;
  }
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->graph_valid = false;
  cudaGraph_t g = nullptr;
  KM_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < iters && e == cudaSuccess; ++it)
    e = enqueue_step(p, w, cfg, step_first(cfg, it), step_sorted(cfg, it), tol, c->cap_stream,
                     step_events(c, profile, it));
  cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(KM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e ? e : e2));
  }
  c->graph_kernels = kernel_nodes(g);
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec = nullptr;
    return fail(KM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  c->gkey = key;
  c->graph_valid = true;
  *out = c->gexec;
  return KM_OK;
}

struct HostReadback {
  Ctl ctl;
};

#define KM_TRACE(...)                         \
  do {                                        \
    if (debug_sync()) {                       \
      fprintf(stderr, "[kmeans] " __VA_ARGS__); \
      fflush(stderr);                         \
    }                                         \
  } while (0)

// Runs `iters` steps on device arrays. The caller holds c->mu. part != null:
// one partial step of a shard (kmeans_step_partial; iters = 1, C unchanged).
int run_locked(DevCtx* c, const km_opts& o, const Problem& p_in, int iters, double tol, bool graph,
               km_stats* st, double* part = nullptr) {
  Problem p = p_in;
  int rc = init_ctx(c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  const int det = o.deterministic ? 1 : 0;
  // the previous call's codes and sorted order are reused only when everything they depend on matches
  const DevCtx::XCache xc = c->xc;
  bool reuse = o.reuse_x && xc.valid && xc.X == (const void*)p.X && xc.n == p.n && xc.d == p.d && xc.k == p.k &&
               xc.prec == o.precision && xc.det == det;
  c->xc.valid = false;  // until this call succeeds
  const int lay_warm = reuse ? xc.lay_warm : o.warm_start;
  const Layout L = layout_for(p.n, p.k, p.d, iters, o.precision, lay_warm, det);
  KM_TRACE("layout: %zu bytes (n=%lld d=%d k=%d prec=%d)\n", L.total, (long long)p.n, p.d, p.k, o.precision);
  if ((rc = ensure_ws(c, L, s))) return rc;
  if (reuse && c->ws_gen != xc.ws_gen) reuse = false;  // the workspace was reallocated
  KM_TRACE("workspace ready at %p (%zu bytes)\n", c->ws, c->ws_bytes);
  // the per-step histories are consecutive regions of the workspace: read back with the control block in
  // two copies (host layout: the control block, then the histories at their workspace offsets from L.obj)
  const size_t hist_bytes = L.queued + 8 * (size_t)iters - L.obj;
  const size_t host_need = align_up(sizeof(Ctl), 64) + hist_bytes + 64;
  if (host_need > c->host_bytes) {
    if (c->host) cudaFreeHost(c->host);
    c->host = nullptr;
    c->host_bytes = 0;
    if (cudaMallocHost(&c->host, host_need * 2) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "pinned host allocation failed");
    }
    c->host_bytes = host_need * 2;
  }
  Work w = make_work(c, L);
  if (part) {  // a partial step sums straight into the caller's buffer; its counts stay in the workspace
    w.sums64 = part;
    p.counts = w.pcounts;
  }
  const bool profile = o.profile != 0;
  if (profile && (rc = ensure_events(c, 2 + (size_t)iters * kEvPerStep))) return rc;
  StepCfg cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.precision = o.precision;
  cfg.recheck = o.recheck;
  cfg.warm = o.warm_start;
  cfg.det = det;
  cfg.reuse = reuse ? 1 : 0;
  cfg.part = part;
  auto fill_tc = [&](int precision, const float4* xs, TcShape& t, TcLaunch& Lc, TcParams& P) -> int {
    t = tc_shape(precision, p.d, p.k);
    Lc.fp8 = t.fp8;
    int r2;
    if ((r2 = encode_codes_map(&Lc.mapX, w.Xq, p.n, t.Kw, t.esz, 128))) return r2;
    if ((r2 = encode_codes_map(&Lc.mapC, w.Cq, t.kp, t.Kc, t.esz, t.bn))) return r2;
    memset(&Lc.mapH, 0, sizeof Lc.mapH);  // the re-score codes' map is encoded by the caller (own slices)
    memset(&Lc.mapXh, 0, sizeof Lc.mapXh);
    if (t.fold && w.Hc && (r2 = encode_h_map(&Lc.mapH, w.Hc, t.kp, t.bn))) return r2;
    if (t.fold && t.fp8 && (r2 = encode_h_map(&Lc.mapXh, w.Xh, p.n, 128))) return r2;
    memset(&P, 0, sizeof P);
    P.h = w.hq;
    P.sc = w.scq;
    P.cst = w.cst;
    P.rows = nullptr;
    P.xs = xs;
    P.xs_sorted = w.xs_sorted;
    P.lab_sorted = w.lab_sorted;
    P.Cq = w.Cq;
    P.assign = p.assign;
    P.flags = w.flags;
    P.ctl = w.ctl;
    P.flag_slots = &w.ctl->n_flagged;
    P.flag_cap = p.n;
    P.n = p.n;
    P.k = p.k;
    P.Kp = t.Kp;
    P.nkb = t.nkb;
    P.bn = t.bn;
    P.nchunks = t.nchunks;
    P.stages = t.stages;
    P.abufs = t.abufs;
    P.idesc = tc::idesc_f32acc(t.fp8 ? 0u : 1u, 128, (uint32_t)t.bn);
    P.split = t.split;
    // truncating FP32 accumulation of K products; the two-part codes sum 3 Kp
    // products and drop lo.lo, |x_lo . c_lo| <= u^2 (1 + u)^2 ||x_hi|| ||c_hi||
    // (u = 2^-8, split_bf16 keeps |lo| <= u (1 + u) |hi| per element). Folded
    // BF16 adds the extra K = 16 slice: products 1 x (-h1, -h2, -h3) of total
    // magnitude <= (1 + 2^-7) h_j enter the accumulation, and -(h1 + h2 + h3)
    // differs from the FP32 h_j by <= 2^-27 h_j.
    const double K = t.split ? 3.0 * t.Kp : (t.fold ? t.Kp + 16.0 : t.Kp);
    const double gk = K * 0x1p-23 / (1.0 - K * 0x1p-23);
    double gam = gk;
    if (t.split) gam += 0x1p-16 * (1.0 + 0x1p-8) * (1.0 + 0x1p-8);
    P.gam_tc = (float)(gam * (1.0 + 1e-6));
    P.fold = t.fold;
    P.idesc16 = tc::idesc_f32acc(1u, 128, (uint32_t)t.bn);  // the folded -h_j slice is a BF16 step
    // score error from h_j: RN to FP32 of the FP64 h (u) and, without folding,
    // the epilogue's multiply-add (2u); folded: u, the three-part remainder and
    // the accumulation of the -h_j products
    P.hcoef = t.fold ? (float)((0x1p-24 + 0x1p-27 + gk * (1.0 + 0x1p-7)) * (1.0 + 1e-6)) : 3.f * 0x1p-24f;
    P.wait_ns = 2000000000ull;
    if (getenv("KM_DEBUG_STALL")) {  // test knob: make a bounded wait expire (50 ms)
      P.debug_stall = 1;
      P.wait_ns = 50000000ull;
    }
    return KM_OK;
  };
  if (o.precision != KM_FP32) {
    cfg.cold = !reuse && cold_bf16_first(o.precision, o.warm_start, p.d, p.k);
    if ((rc = fill_tc(o.precision, w.xs, cfg.t, cfg.L, cfg.P))) return rc;
    KM_TRACE("main shape Kp=%d nkb=%d bn=%d kp=%d stages=%d abufs=%d cold=%d\n", cfg.t.Kp, cfg.t.nkb, cfg.t.bn,
             cfg.t.kp, cfg.t.stages, cfg.t.abufs, (int)cfg.cold);
    if (cfg.cold && (rc = fill_tc(KM_BF16, w.xs16, cfg.t0, cfg.L0, cfg.P0))) return rc;
    cfg.rs16 = w.Xq16 != nullptr;
    if (cfg.rs16) {
      // BF16 re-score of the queued points: codes of the gathered rows (Xq16, row r = point
      // fq_rows[r]), this step's BF16 centroid codes, its own flag list and statistics
      if ((rc = fill_tc(KM_BF16, w.xs16q, cfg.t16, cfg.L16, cfg.P16))) return rc;
      char* wb = (char*)c->ws;
      cfg.Cq16 = (uint8_t*)(wb + L.cq16);
      cfg.hq16 = (float*)(wb + L.hq16);
      cfg.scq16 = (float*)(wb + L.scq16);
      cfg.cst16 = (float4*)(wb + L.cst16);
      if ((rc = encode_codes_map(&cfg.L16.mapX, w.Xq16, w.fq_cap, cfg.t16.Kw, cfg.t16.esz, 128))) return rc;
      if ((rc = encode_codes_map(&cfg.L16.mapC, cfg.Cq16, cfg.t16.kp, cfg.t16.Kc, cfg.t16.esz, cfg.t16.bn)))
        return rc;
      cfg.Hc16 = L.hc16 ? (void*)(wb + L.hc16) : nullptr;
      if (cfg.t16.fold && (rc = encode_h_map(&cfg.L16.mapH, cfg.Hc16, cfg.t16.kp, cfg.t16.bn))) return rc;
      TcParams& Q = cfg.P16;
      Q.h = cfg.hq16;
      Q.sc = cfg.scq16;
      Q.cst = cfg.cst16;
      Q.Cq = cfg.Cq16;
      Q.rows = w.fq_rows;
      Q.xs_sorted = w.xs16q;
      Q.lab_sorted = w.fq_old;
      Q.flags = w.flags2;
      Q.flag_slots = &w.ctl->n_flagged2;
      Q.flag_cap = w.fq_cap;
      Q.n = w.fq_cap;
      Q.n_dev = &w.ctl->n_fullq;
      Q.stats16 = 1;
      Q.debug_stall = 0;
      Q.wait_ns = 2000000000ull;
    }
    if (cfg.cold)
      KM_TRACE("cold shape Kp=%d nkb=%d bn=%d kp=%d stages=%d abufs=%d\n", cfg.t0.Kp, cfg.t0.nkb, cfg.t0.bn,
               cfg.t0.kp, cfg.t0.stages, cfg.t0.abufs);
  }
  KM_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s));
  KM_CUDA(cudaMemsetAsync(w.sums64, 0, 8 * (size_t)p.k * p.d, s));
  if (det) {
    KM_CUDA(cudaMemsetAsync(w.facc, 0, 3 * 8 * (size_t)p.k * p.d, s));
    KM_CUDA(cudaMemsetAsync(w.oacc, 0, 3 * 8, s));
  }
  if (!part) KM_CUDA(cudaMemcpyAsync(w.Csave, p.C, (size_t)p.k * p.d * 4, cudaMemcpyDeviceToDevice, s));
  KM_CUDA(cudaEventRecord(c->ev0, s));
  if (profile) KM_CUDA(cudaEventRecord(c->prof[0], s));
  KM_TRACE("prologue copies queued (reuse=%d det=%d partial=%d)\n", (int)reuse, det, part ? 1 : 0);
  // small FP32 problems: the whole call is one cooperative kernel (km_small.cu); profiled, deterministic
  // and partial calls take the staged path, which records their stage events and partials
  const bool small = o.precision == KM_FP32 && !profile && !det && !part && !debug_sync() && w.small &&
                     small_path_fits(p.n, p.d, p.k);
  if (small) {
    // the kernel computes the point norms it needs itself
  } else if (reuse) {
    // codes, row statistics, norms, sorted order and max ||x|| are those the previous call left
  } else if (o.precision != KM_FP32 && cfg.cold) {
    KM_CUDA(launch_centre(p, w, s));
    KM_CUDA(launch_quant_x_dual(p, w, cfg.t0.Kp, w.Xq, w.xs16, w.xs, s));
  } else if (o.precision != KM_FP32) {
    KM_CUDA(launch_centre(p, w, s));
    KM_CUDA(launch_quant_x(p, w, cfg.t.qmode(), cfg.t.Kp, w.Xq, w.xs, s));
  } else {
    KM_CUDA(launch_xnorm(p, w, s));
  }
  if (!reuse && det) KM_CUDA(launch_xmax(w.xnorm, nullptr, p.n, w, s));  // (uncentred norms on every path)
  if (debug_sync()) {
    cudaError_t r = cudaStreamSynchronize(s);
    KM_TRACE("point quantisation / norms: %s\n", cudaGetErrorString(r));
    KM_CUDA(r);
  }
  if (profile) KM_CUDA(cudaEventRecord(c->prof[1], s));
  int launches = 0;
  if (small) {
    KM_CUDA(launch_small_run(p, w, iters, tol, step_first(cfg, 0), o.recheck, s));
    launches = 1;
  } else if (graph && iters > 1 && !debug_sync()) {
    GraphKey key;
    memset(&key, 0, sizeof key);
    key.X = p.X; key.C = p.C; key.assign = p.assign; key.sums = p.sums; key.counts = p.counts;
    key.n = p.n; key.d = p.d; key.k = p.k; key.iters = iters; key.prec = o.precision; key.tol = tol;
    key.profile = (profile ? 1 : 0) | (o.recheck ? 2 : 0) | (o.warm_start ? 4 : 0) |
                  (getenv("KM_DEBUG_STALL") ? 8 : 0) | (det ? 16 : 0) | (reuse ? 32 : 0);
    key.ws_gen = c->ws_gen;
    cudaGraphExec_t ge = nullptr;
    if ((rc = get_graph(c, key, p, w, cfg, iters, tol, profile, &ge))) return rc;
    KM_CUDA(cudaGraphLaunch(ge, s));
    launches = 1 + c->graph_kernels;  // the point-norm / quantisation kernel, then the graph
  } else {
    for (int it = 0; it < iters; ++it)
      KM_CUDA(enqueue_step(p, w, cfg, step_first(cfg, it), step_sorted(cfg, it), tol, s, step_events(c, profile, it)));
  }
  KM_CUDA(cudaEventRecord(c->ev1, s));
  char* h = (char*)c->host;
  Ctl* hc = (Ctl*)h;
  char* hh = h + align_up(sizeof(Ctl), 64);  // the histories, at their offsets from L.obj
  const double* hobj = (const double*)hh;
  const double* hshift = (const double*)(hh + (L.shift - L.obj));
  const unsigned long long* hchanged = (const unsigned long long*)(hh + (L.changed - L.obj));
  const unsigned long long* hflag = (const unsigned long long*)(hh + (L.flagged - L.obj));
  const unsigned long long* hfull = (const unsigned long long*)(hh + (L.full - L.obj));
  const unsigned long long* hqueued = (const unsigned long long*)(hh + (L.queued - L.obj));
  const int* hempty = (const int*)(hh + (L.empty - L.obj));
  KM_CUDA(cudaMemcpyAsync(hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hh, (const char*)c->ws + L.obj, hist_bytes, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (hc->iters_done < 0 || hc->iters_done > iters)
    return fail(KM_ECUDA, "device control block is inconsistent (%d steps recorded, %d run)", hc->iters_done, iters);
  if (hc->nonfinite || hc->error) {
    if (!part) {  // a partial step leaves C alone
      KM_CUDA(cudaMemcpyAsync(p.C, w.Csave, (size_t)p.k * p.d * 4, cudaMemcpyDeviceToDevice, s));
      KM_CUDA(cudaStreamSynchronize(s));
    }
    if (hc->nonfinite) return fail(KM_ENONFINITE, "X or C holds a non-finite value (or a norm overflows FP32)");
    return fail(hc->error, "device stage reported error %d", hc->error);
  }
  if (getenv("KM_LOG")) {  // per-step history on stderr, for diagnosis
    for (int it = 0; it < hc->iters_done; ++it)
      fprintf(stderr, "[kmeans] step %d: J=%.9g changed=%llu flagged=%llu full=%llu empty=%d shift=%.3g\n", it,
              hobj[it], hchanged[it], hflag[it], hfull[it], hempty[it], hshift[it]);
  }
  if (st) {
    memset(st, 0, sizeof *st);
    const int last = hc->iters_done - 1;
    st->iters_done = hc->iters_done;
    st->launches = launches;
    if (last >= 0) {
      st->objective = hobj[last];
      st->shift = hshift[last];
      st->n_changed = (int64_t)hchanged[last];
      st->n_flagged = (int64_t)hflag[last];
      st->n_full = (int64_t)hfull[last];
      st->n_empty = hempty[last];
      st->n_queued = (int64_t)hqueued[last];
      // a cold E4M3 call computes its first step's distances with BF16 codes
      st->iters_bf16 = (o.precision == KM_FP8E4M3 && cfg.cold) ? 1 : 0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    st->ms = ms;
    if (profile) {
      float t = 0.f;
      KM_CUDA(cudaEventElapsedTime(&t, c->prof[0], c->prof[1]));
      st->stage_ms[KM_STAGE_XNORM] = t;
      for (int it = 0; it < iters; ++it) {
        const cudaEvent_t* ev = step_events(c, true, it);
        for (int sg = 0; sg < kEvPerStep - 1; ++sg) {
          KM_CUDA(cudaEventElapsedTime(&t, ev[sg], ev[sg + 1]));
          st->stage_ms[KM_STAGE_PREP + sg] += t;
        }
      }
    }
  }
  // the workspace now holds this X's codes, norms and (quantised paths) sorted order
  c->xc.valid = true;
  c->xc.X = p.X;
  c->xc.n = p.n;
  c->xc.d = p.d;
  c->xc.k = p.k;
  c->xc.prec = o.precision;
  c->xc.lay_warm = lay_warm;
  c->xc.det = det;
  c->xc.ws_gen = c->ws_gen;
  return KM_OK;
}

km_opts resolve(const km_opts* o) {
  km_opts r;
  kmeans_default_opts(&r);
  if (o) r = *o;
  return r;
}

int device_entry(const km_opts* opts, const float* X, int64_t n, int32_t d, float* C, int32_t k,
                 int32_t* assign, float* sums, int32_t* counts, int32_t iters, double tol, bool graph,
                 km_stats* stats) {
  g_err.clear();
  const km_opts o = resolve(opts);
  Problem p{X, n, d, C, k, assign, sums, counts};
  int rc = validate_args(o, p, iters);
  if (rc) return rc;
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  if ((rc = validate_device_ptrs(p, dev))) return rc;
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  return run_locked(c, o, p, iters, tol, graph, stats);
}

}  // namespace

KM_API void kmeans_default_opts(km_opts* opts) {
  if (!opts) return;
  memset(opts, 0, sizeof *opts);
  opts->precision = KM_FP32;
  opts->recheck = 1;
}

KM_API int kmeans_step(const float* X, int64_t n, int32_t d, float* C, int32_t k, int32_t* assign,
                       float* sums, int32_t* counts) {
  return device_entry(nullptr, X, n, d, C, k, assign, sums, counts, 1, 0.0, false, nullptr);
}

KM_API int kmeans_run(const float* X, int64_t n, int32_t d, float* C, int32_t k, int32_t* assign,
                      float* sums, int32_t* counts, int32_t iters, double tol) {
  return device_entry(nullptr, X, n, d, C, k, assign, sums, counts, iters, tol, true, nullptr);
}

KM_API int kmeans_step_ex(const km_opts* opts, const float* X, int64_t n, int32_t d, float* C,
                          int32_t k, int32_t* assign, float* sums, int32_t* counts, km_stats* stats) {
  return device_entry(opts, X, n, d, C, k, assign, sums, counts, 1, 0.0, false, stats);
}

KM_API int kmeans_run_ex(const km_opts* opts, const float* X, int64_t n, int32_t d, float* C,
                         int32_t k, int32_t* assign, float* sums, int32_t* counts, int32_t iters,
                         double tol, km_stats* stats) {
  return device_entry(opts, X, n, d, C, k, assign, sums, counts, iters, tol, true, stats);
}

KM_API int kmeans_step_partial(const km_opts* opts, const float* X, int64_t n, int32_t d, const float* C,
                               int32_t k, int32_t* assign, double* part, km_stats* stats) {
  g_err.clear();
  const km_opts o = resolve(opts);
  if (!X || !C || !assign || !part) return fail(KM_EINVAL, "null array pointer");
  Problem p{X, n, d, const_cast<float*>(C), k, assign, nullptr, nullptr};
  int rc = validate_shape(o, p, 1);
  if (rc) return rc;
  const size_t nd = (size_t)n * d * 4, kd = (size_t)k * d * 4, na = (size_t)n * 4;
  const size_t np = 8 * (size_t)KM_PARTIALS_LEN(k, d);
  if (overlaps(X, nd, C, kd) || overlaps(X, nd, assign, na) || overlaps(X, nd, part, np) || overlaps(C, kd, assign, na) ||
      overlaps(C, kd, part, np) || overlaps(assign, na, part, np))
    return fail(KM_EINVAL, "arrays overlap");
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  if ((rc = check_device_ptr(X, "X", dev)) || (rc = check_device_ptr(C, "C", dev)) ||
      (rc = check_device_ptr(assign, "assign", dev)) || (rc = check_device_ptr(part, "part", dev)))
    return rc;
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  return run_locked(c, o, p, 1, 0.0, false, stats, part);
}

KM_API int kmeans_apply_partials(const km_opts* opts, const double* part, int32_t k, int32_t d, float* C,
                                 float* sums, int32_t* counts, km_stats* stats) {
  g_err.clear();
  const km_opts o = resolve(opts);
  if (!part || !C) return fail(KM_EINVAL, "null array pointer");
  if (k < 1 || d < 1 || d > kMaxD) return fail(KM_EINVAL, "k = %d, d = %d: need k >= 1, 1 <= d <= %d", k, d, kMaxD);
  const size_t kd = (size_t)k * d * 4, nk = (size_t)k * 4, np = 8 * (size_t)KM_PARTIALS_LEN(k, d);
  if (overlaps(part, np, C, kd) || (sums && (overlaps(part, np, sums, kd) || overlaps(C, kd, sums, kd))) ||
      (counts && (overlaps(part, np, counts, nk) || overlaps(C, kd, counts, nk))) ||
      (sums && counts && overlaps(sums, kd, counts, nk)))
    return fail(KM_EINVAL, "arrays overlap");
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  int rc;
  if ((rc = check_device_ptr(part, "part", dev)) || (rc = check_device_ptr(C, "C", dev)) ||
      (sums && (rc = check_device_ptr(sums, "sums", dev))) || (counts && (rc = check_device_ptr(counts, "counts", dev))))
    return rc;
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  if ((rc = init_ctx(c))) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  if (!c->actl) {
    if (cudaMalloc(&c->actl, 4 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "status allocation failed");
    }
  }
  KM_CUDA(cudaEventRecord(c->ev0, s));
  KM_CUDA(launch_apply_partials(part, k, d, C, sums, counts, c->actl, s));
  KM_CUDA(cudaEventRecord(c->ev1, s));
  unsigned long long h[4] = {0, 0, 0, 0};
  double tail[2] = {0.0, 0.0};
  KM_CUDA(cudaMemcpyAsync(h, c->actl, sizeof h, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(tail, part + (int64_t)k * d + k, sizeof tail, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (h[0]) return fail(KM_EINVAL, "the partials buffer holds a count that is not an integer in [0, 2^31)");
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->objective = tail[0];
    stats->n_changed = (int64_t)tail[1];
    double s2;
    memcpy(&s2, &h[1], sizeof s2);
    stats->shift = sqrt(s2);
    stats->n_empty = (int32_t)h[2];
    stats->iters_done = 1;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    stats->ms = ms;
  }
  return KM_OK;
}

KM_API int kmeans_run_host(const km_opts* opts, const float* X, int64_t n, int32_t d, float* C,
                           int32_t k, int32_t* assign, float* sums, int32_t* counts, int32_t iters,
                           double tol, km_stats* stats) {
  g_err.clear();
  km_opts o = resolve(opts);
  o.reuse_x = 0;  // the device copy of X is refreshed by every call
  Problem hp{X, n, d, C, k, assign, sums, counts};
  int rc = validate_args(o, hp, iters);
  if (rc) return rc;
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  if ((rc = init_ctx(c))) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  const size_t nd = align_up((size_t)n * d * 4), kd = align_up((size_t)k * d * 4);
  const size_t na = align_up((size_t)n * 4), nk = align_up((size_t)k * 4);
  const size_t need = nd + 2 * kd + na + nk;
  if (need > c->stage_bytes) {
    if (c->stage) {
      KM_CUDA(cudaDeviceSynchronize());
      cudaFree(c->stage);
      c->stage = nullptr;
      c->stage_bytes = 0;
      c->graph_valid = false;
    }
    if (cudaMalloc(&c->stage, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "staging allocation of %zu bytes failed", need);
    }
    c->stage_bytes = need;
  }
  char* b = (char*)c->stage;
  Problem p{(const float*)b, n, d, (float*)(b + nd), k, (int32_t*)(b + nd + kd), (float*)(b + nd + kd + na),
            (int32_t*)(b + nd + 2 * kd + na)};
  KM_CUDA(cudaMemcpyAsync((void*)p.X, X, (size_t)n * d * 4, cudaMemcpyHostToDevice, s));
  KM_CUDA(cudaMemcpyAsync(p.C, C, (size_t)k * d * 4, cudaMemcpyHostToDevice, s));
  if ((rc = run_locked(c, o, p, iters, tol, true, stats))) return rc;
  KM_CUDA(cudaMemcpyAsync(C, p.C, (size_t)k * d * 4, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(assign, p.assign, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(sums, p.sums, (size_t)k * d * 4, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(counts, p.counts, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  return KM_OK;
}

// ============================================================================ keyed-reduce training

namespace {

// The class keyed reduce shared by GDA and NB: n_c into counts, S_c into
// w.sums64 (FP64), then `finish` enqueues the method's own kernels. Runs
// synchronously on opts->stream; bad labels give KM_EINVAL.
template <typename Finish>
int class_train(const km_opts* opts, const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls,
                std::initializer_list<std::pair<const void*, const char*>> outs, size_t cov_bytes,
                Finish&& finish) {
  g_err.clear();
  const km_opts o = resolve(opts);
  if (!X || !y) return fail(KM_EINVAL, "X and y must be non-null");
  if (n < 1 || n > INT32_MAX) return fail(KM_EINVAL, "n = %lld outside [1, 2^31)", (long long)n);
  if (d < 1 || d > kMaxD) return fail(KM_EINVAL, "d = %d outside [1, %d]", d, kMaxD);
  if (ncls < 1 || ncls > (1 << 20)) return fail(KM_EINVAL, "ncls = %d outside [1, 2^20]", ncls);
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  int rc;
  if ((rc = check_device_ptr(X, "X", dev)) || (rc = check_device_ptr(y, "y", dev))) return rc;
  for (const auto& op : outs) {
    if (!op.first) return fail(KM_EINVAL, "%s must be non-null", op.second);
    if ((rc = check_device_ptr(op.first, op.second, dev))) return rc;
  }
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  c->xc.valid = false;  // this call overwrites the workspace
  if ((rc = init_ctx(c))) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  const Layout L = layout_for(n, ncls, d, 1, KM_FP32, 0, 0);
  if ((rc = ensure_ws(c, L, s))) return rc;
  const Work w = make_work(c, L);
  const size_t cnt_bytes = align_up(4 * (size_t)ncls), need = cnt_bytes + align_up(cov_bytes) + 1024;
  if (need > c->cls_bytes) {
    if (c->cls) {
      KM_CUDA(cudaDeviceSynchronize());
      cudaFree(c->cls);
      c->cls = nullptr;
      c->cls_bytes = 0;
    }
    if (cudaMalloc(&c->cls, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "class buffer allocation of %zu bytes failed", need);
    }
    c->cls_bytes = need;
  }
  char* cb = (char*)c->cls;
  int32_t* counts = (int32_t*)cb;
  double* cov64 = (double*)(cb + cnt_bytes);
  int2* tiles = (int2*)(cb + cnt_bytes + align_up(cov_bytes));
  KM_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s));
  KM_CUDA(cudaMemsetAsync(w.sums64, 0, 8 * (size_t)ncls * d, s));
  KM_CUDA(cudaMemsetAsync(counts, 0, 4 * (size_t)ncls, s));
  KM_CUDA(cudaMemsetAsync(w.Csave, 0, 4 * (size_t)ncls * d, s));  // zero centres: the reduce's objective is unused
  // the keyed reduce of a Lloyd step with the labels as keys
  Problem p{X, n, d, w.Csave, ncls, const_cast<int32_t*>(y), nullptr, counts};
  KM_CUDA(launch_check_classes(y, n, ncls, w.ctl, s));
  KM_CUDA(launch_count(p, w, s));
  KM_CUDA(launch_scan(p, w, s));
  KM_CUDA(launch_scatter(p, w, s));
  KM_CUDA(launch_segsum(p, w, s));
  KM_CUDA(finish(w, counts, cov64, tiles, s));
  if (sizeof(Ctl) > c->host_bytes) {  // pinned read-back of the control block
    if (c->host) cudaFreeHost(c->host);
    c->host = nullptr;
    c->host_bytes = 0;
    if (cudaMallocHost(&c->host, 4096) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "pinned host allocation failed");
    }
    c->host_bytes = 4096;
  }
  Ctl* hc = (Ctl*)c->host;
  KM_CUDA(cudaMemcpyAsync(hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (hc->error) return fail(hc->error, "a label lies outside [0, %d)", ncls);
  return KM_OK;
}

}  // namespace

KM_API int kmeans_gda_train(const km_opts* opts, const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls,
                        float* phi, float* mu, float* sigma) {
  return class_train(opts, X, n, d, y, ncls, {{phi, "phi"}, {mu, "mu"}, {sigma, "sigma"}},
                     gda_cov_scratch_bytes(n, d),
                     [&](const Work& w, const int32_t* counts, double* cov64, int2* tiles, cudaStream_t s) {
                       cudaError_t e = launch_gda_means(w.sums64, counts, n, d, ncls, phi, mu, w.ctl, s);
                       if (e == cudaSuccess) e = launch_gda_cov(X, n, d, y, mu, tiles, cov64, sigma, w.ctl, s);
                       return e;
                     });
}

KM_API int kmeans_nb_train(const km_opts* opts, const float* X, int64_t n, int32_t d, const int32_t* y, int32_t ncls,
                       float* prior, float* theta) {
  return class_train(opts, X, n, d, y, ncls, {{prior, "prior"}, {theta, "theta"}}, 0,
                     [&](const Work& w, const int32_t* counts, double*, int2*, cudaStream_t s) {
                       return launch_nb_theta(w.sums64, counts, n, d, ncls, prior, theta, w.ctl, s);
                     });
}

// ============================================================================ SPADE downsampling

namespace {

// Largest float <= v (lo) or smallest float >= v (hi).
float float_below(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
float float_above(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

}  // namespace

KM_API int kmeans_spade_densities(const km_opts* opts, const float* X, int64_t n, int32_t d, double apprx_width,
                                  double kernel_width, int32_t policy, int32_t* densities, int32_t* counts,
                                  uint8_t* processed, km_spade_stats* stats) {
  g_err.clear();
  const km_opts o = resolve(opts);
  if (!X || !densities) return fail(KM_EINVAL, "X and densities must be non-null");
  if (n < 1 || n >= INT32_MAX) return fail(KM_EINVAL, "n = %lld outside [1, 2^31 - 1)", (long long)n);
  if (d < 1 || d > 4096) return fail(KM_EINVAL, "d = %d outside [1, 4096]", d);
  if (!(apprx_width > 0.0) || !std::isfinite(apprx_width) || !(kernel_width > 0.0) || !std::isfinite(kernel_width))
    return fail(KM_EINVAL, "widths must be finite and > 0 (apprx %g, kernel %g)", apprx_width, kernel_width);
  if (policy != KM_SPADE_LAST && policy != KM_SPADE_FIRST) return fail(KM_EINVAL, "unknown policy %d", policy);
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  int rc;
  if ((rc = check_device_ptr(X, "X", dev)) || (rc = check_device_ptr(densities, "densities", dev))) return rc;
  if (counts && (rc = check_device_ptr(counts, "counts", dev))) return rc;
  if (processed && (rc = check_device_ptr(processed, "processed", dev))) return rc;
  const size_t nd = (size_t)n * d * 4;
  if (overlaps(X, nd, densities, 4 * (size_t)n) || (counts && overlaps(X, nd, counts, 4 * (size_t)n)) ||
      (processed && overlaps(X, nd, processed, (size_t)n)))
    return fail(KM_EINVAL, "outputs overlap X");
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  c->xc.valid = false;  // this call overwrites the workspace
  if ((rc = init_ctx(c))) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;

  // workspace: control block, per-row state, batch state, found-row list
  const int64_t cap = std::min<int64_t>((int64_t)8 << 20, std::max<int64_t>((int64_t)1 << 16, (int64_t)kSB * n));
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t at = off; off = align_up(off + bytes); return at; };
  const size_t o_ctl = take(sizeof(SpadeCtl)), o_q = take(4 * (size_t)n), o_slot = take(4 * (size_t)n),
               o_cnt = take(4 * (size_t)n), o_proc = take((size_t)n), o_cand = take(4 * (size_t)kSB),
               o_cc = take(4 * (size_t)kSB), o_inp = take((size_t)kSB), o_nbr = take(4 * (size_t)kSB * (kSB / 32)),
               o_pairs = take(8 * (size_t)cap);
  if (off > c->spade_bytes) {
    if (c->spade) {
      KM_CUDA(cudaDeviceSynchronize());
      cudaFree(c->spade);
      c->spade = nullptr;
      c->spade_bytes = 0;
    }
    if (cudaMalloc(&c->spade, off) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "downsampling workspace of %zu bytes failed", off);
    }
    c->spade_bytes = off;
  }
  char* base = (char*)c->spade;
  SpadeArgs A;
  memset(&A, 0, sizeof A);
  A.X = X;
  A.n = n;
  A.d = d;
  A.vec = (d % 4 == 0) && ((uintptr_t)X % 16 == 0);
  // decision bands: |D^ - D| <= gamma D (FP32 sum of d rounded terms), |D64 - D| <= g64 D
  const double g32 = (double)(d + 2) * 0x1p-24 / (1.0 - (double)(d + 2) * 0x1p-24);
  const double g64 = (double)(d + 2) * 0x1p-53 / (1.0 - (double)(d + 2) * 0x1p-53);
  const double cw = policy == KM_SPADE_LAST ? kernel_width : std::max(apprx_width, kernel_width);
  auto band = [&](double w, float& lo, float& hi) {
    lo = float_below(w * (1.0 - g32) / (1.0 + g64) * (1.0 - 0x1p-40));
    hi = float_above(w * (1.0 + g32) / (1.0 - g64) * (1.0 + 0x1p-40));
  };
  band(apprx_width, A.a_lo, A.a_hi);
  band(cw, A.w_lo, A.w_hi);
  // |fl(D - w_mid)| <= w_half for every D in [w_lo, w_hi] (rounding is monotone)
  A.w_mid = (float)(0.5 * ((double)A.w_lo + (double)A.w_hi));
  A.w_half = float_above(std::max((double)A.w_mid - (double)A.w_lo, (double)A.w_hi - (double)A.w_mid));
  A.apprx = apprx_width;
  A.cw = cw;
  A.policy = policy;
  A.none = policy == KM_SPADE_LAST ? -1 : INT32_MAX;
  A.ctl = (SpadeCtl*)(base + o_ctl);
  A.q = (int32_t*)(base + o_q);
  A.slot = (int32_t*)(base + o_slot);
  A.counts = (int32_t*)(base + o_cnt);
  A.processed = (uint8_t*)(base + o_proc);
  A.cand = (int32_t*)(base + o_cand);
  A.ccount = (int32_t*)(base + o_cc);
  A.inP = (uint8_t*)(base + o_inp);
  A.nbr = (uint32_t*)(base + o_nbr);
  A.pairs = (int2*)(base + o_pairs);
  A.pair_cap = cap;
  if (sizeof(SpadeCtl) > c->host_bytes) {
    if (c->host) cudaFreeHost(c->host);
    c->host = nullptr;
    c->host_bytes = 0;
    if (cudaMallocHost(&c->host, 4096) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "pinned host allocation failed");
    }
    c->host_bytes = 4096;
  }
  SpadeCtl* hc = (SpadeCtl*)c->host;
  KM_CUDA(cudaMemsetAsync(A.ctl, 0, sizeof(SpadeCtl), s));
  KM_CUDA(cudaEventRecord(c->ev0, s));
  KM_CUDA(launch_spade_init(A, s));
  KM_CUDA(cudaMemcpyAsync(hc, A.ctl, sizeof(SpadeCtl), cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (hc->nonfinite) return fail(KM_ENONFINITE, "X holds a NaN or Inf");
  // batches until one finds no candidate; every other batch settles at least one row,
  // so at most n + 1 batches run (read back every few batches)
  constexpr int kGroup = 4;
  int64_t launched = 0;
  for (int64_t b = 0; b <= n + kGroup; b += kGroup) {
    if ((rc = ensure_events(c, 2 * (size_t)(launched + kGroup)))) return rc;
    for (int g = 0; g < kGroup; ++g, ++launched)
      KM_CUDA(launch_spade_batch(A, s, c->prof[2 * launched], c->prof[2 * launched + 1]));
    KM_CUDA(cudaMemcpyAsync(hc, A.ctl, sizeof(SpadeCtl), cudaMemcpyDeviceToHost, s));
    KM_CUDA(cudaStreamSynchronize(s));
    if (hc->done) break;
  }
  float ms_pairs = 0.f;
  for (int64_t b = 0; b < launched; ++b) {
    float m = 0.f;
    KM_CUDA(cudaEventElapsedTime(&m, c->prof[2 * b], c->prof[2 * b + 1]));
    ms_pairs += m;
  }
  if (!hc->done) return fail(KM_ECUDA, "downsampling did not settle every row");
  KM_CUDA(launch_spade_density(A, densities, s));
  if (counts) KM_CUDA(cudaMemcpyAsync(counts, A.counts, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
  if (processed) KM_CUDA(cudaMemcpyAsync(processed, A.processed, (size_t)n, cudaMemcpyDeviceToDevice, s));
  KM_CUDA(cudaEventRecord(c->ev1, s));
  KM_CUDA(cudaMemcpyAsync(hc, A.ctl, sizeof(SpadeCtl), cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->n_evaluated = (int64_t)hc->n_evaluated;
    stats->n_computed = (int64_t)hc->n_computed;
    stats->n_found_pairs = (int64_t)hc->n_apprx;
    stats->n_exact = (int64_t)hc->n_exact;
    stats->batches = hc->batches;
    stats->overflow_batches = hc->overflow_batches;
    float ms = 0.f;
    KM_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    stats->ms = ms;
    stats->ms_pairs = ms_pairs;
  }
  return KM_OK;
}

KM_API const char* kmeans_last_error(void) { return g_err.c_str(); }

KM_API int32_t kmeans_version(void) { return 200; }

// ============================================================================ batched runs

namespace {

// Launch shape of a batch: chunk width, the order of the instances in the
// flattened tile space (0: as given, 1: by decreasing work per row tile), and
// whether the instances whose k spans several chunks run their tiles in the
// previous step's cluster-sorted order (1; a tile then mostly holds rows of one
// previous cluster, so its candidate tracking is cheap and starts with that
// cluster's chunk; their codes are copied in that order after each scatter) or
// every instance keeps the order of X (0). An instance with one chunk gains
// nothing from the order: its rows see every column in one block anyway.
struct BatchTune {
  int bn;
  int order;
  int sorted;
};

struct BatchPlan {
  std::vector<int> order;  // flattened position -> caller's instance index
  std::vector<BInst> inst;
  std::vector<int64_t> row_off, tile_off;
  std::vector<BChunk> sitems;     // work items of the segmented sum: about 96 KB of X each
  std::vector<int64_t> cta_tile;  // tile range of each CTA of the assignment launch
  std::vector<BChunk> rchunks;    // row chunks of the count and scatter stages
  std::vector<int32_t> kc_inst, kp_inst;  // instance of each flattened (padded) centroid
  int kmax = 0;
  int64_t R = 0, KC = 0, KP = 0, T = 0, SUMS = 0, XQ = 0, XQS = 0, CQ = 0, CSAVE = 0;
  int nkb_max = 1, kp_max = 0, stages = 0, abufs = 2, bn = 128, fp8 = 0, sorted = 1;
  int shape = 0;  // the tune, as km_stats.batch_shape reports it
};

// Work model of one 128-row tile of an instance, in units of a 128-column chunk
// with one 128-byte K block: epilogue work ~ the columns, MMA ~ columns x K, plus
// a fixed per-tile cost.
double tile_work(const BInst& I) {
  const double cols = (double)I.kp / 128.0;
  return cols * (0.5 + 0.5 * I.nkb * I.rowb / 128.0) + 1.5;
}

int plan_batch(const km_instance* in, int count, int precision, const BatchTune& tune, BatchPlan& P) {
  P = BatchPlan();
  P.fp8 = precision == KM_FP8E4M3;
  P.bn = tune.bn;
  P.sorted = tune.sorted;
  P.shape = tune.bn + 1000 * tune.order + 10000 * tune.sorted;
  const int esz = P.fp8 ? 1 : 2, kbe = 128 / esz;
  P.order.resize(count);
  for (int b = 0; b < count; ++b) P.order[b] = b;
  if (tune.order == 1) {
    std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) {
      return (int64_t)in[a].k * in[a].d > (int64_t)in[b].k * in[b].d;
    });
  }
  P.inst.resize(count);
  P.row_off.assign(count + 1, 0);
  P.tile_off.assign(count + 1, 0);
  for (int q = 0; q < count; ++q) {
    const km_instance& s = in[P.order[q]];
    BInst& I = P.inst[q];
    memset(&I, 0, sizeof I);
    I.X = s.X;
    I.C = s.C;
    I.assign = s.assign;
    I.sums = s.sums;
    I.counts = s.counts;
    I.n = s.n;
    I.d = s.d;
    I.k = s.k;
    // K: rows of 32 or 64 bytes (one MMA step or two, with the swizzle of that width) when d fits,
    // else whole 128-byte blocks; N: k rounded up to 32 columns when one chunk holds it
    if (s.d * esz <= 32) I.rowb = 32;
    else if (s.d * esz <= 64) I.rowb = 64;
    else I.rowb = 128;
    I.Kp = I.rowb < 128 ? I.rowb / esz : (s.d + kbe - 1) / kbe * kbe;
    I.nkb = I.rowb < 128 ? 1 : I.Kp / kbe;
    I.bn = s.k < P.bn ? (s.k + 31) / 32 * 32 : P.bn;
    I.kp = (s.k + I.bn - 1) / I.bn * I.bn;
    I.nchunks = I.kp / I.bn;
    I.gsort = tune.sorted && I.nchunks > 1;
    const double K = I.Kp;
    I.gam_tc = (float)(K * 0x1p-23 / (1.0 - K * 0x1p-23) * (1.0 + 1e-6));
    I.row_off = P.R;
    I.kc_off = P.KC;
    I.kp_off = P.KP;
    I.offs_off = P.KP + q;
    I.sum_off = P.SUMS;
    I.tile_off = P.T;
    I.xq_off = P.XQ;
    I.xqs_off = P.XQS;
    I.cq_off = P.CQ;
    P.R += s.n;
    P.KC += s.k;
    P.KP += I.kp;
    P.SUMS += (int64_t)s.k * s.d;
    P.CSAVE += (int64_t)s.k * s.d;
    P.T += (s.n + 127) / 128;
    P.XQ += align_up((size_t)s.n * I.Kp * esz, 256);
    if (I.gsort) P.XQS += align_up((size_t)s.n * I.Kp * esz, 256);
    P.CQ += align_up((size_t)I.kp * I.Kp * esz, 256);
    P.row_off[q + 1] = P.R;
    P.tile_off[q + 1] = P.T;
    {  // segmented-sum items: about 96 KB of rows, a multiple of 32 rows, at most 4096
      const int64_t per = std::min<int64_t>(4096, std::max<int64_t>(32, (98304 / (4 * s.d)) / 32 * 32));
      for (int64_t r = 0; r < s.n; r += per)
        P.sitems.push_back(BChunk{I.row_off + r, q, (int)std::min<int64_t>(per, s.n - r)});
    }
    P.nkb_max = std::max(P.nkb_max, I.nkb);
    P.kp_max = std::max(P.kp_max, I.kp);
    P.kmax = std::max(P.kmax, s.k);
    for (int64_t r = 0; r < s.n; r += kBRowChunk)
      P.rchunks.push_back(BChunk{I.row_off + r, q, (int)std::min<int64_t>(kBRowChunk, s.n - r)});
    P.kc_inst.insert(P.kc_inst.end(), (size_t)s.k, q);
    P.kp_inst.insert(P.kp_inst.end(), (size_t)I.kp, q);
  }
  P.stages = tc_pick_buffers(P.nkb_max, P.bn, P.kp_max, P.fp8, &P.abufs);
  if (P.stages < 2) return fail(KM_EUNSUPPORTED, "largest k of the batch does not fit the tensor-core pipeline");
  // contiguous tile ranges per CTA, balanced by a work model of a tile: MMA
  // and epilogue work ~ chunks x K blocks, plus a fixed per-tile cost
  const int grid = (int)std::min<int64_t>(P.T, num_sms());
  std::vector<double> wsum(count + 1, 0.0);
  for (int q = 0; q < count; ++q) {
    const BInst& I = P.inst[q];
    const double per_tile = tile_work(I);
    wsum[q + 1] = wsum[q] + per_tile * (double)(P.tile_off[q + 1] - P.tile_off[q]);
  }
  P.cta_tile.assign(grid + 1, P.T);
  P.cta_tile[0] = 0;
  int q = 0;
  for (int c = 1; c < grid; ++c) {
    const double target = wsum[count] * c / grid;
    while (q < count - 1 && wsum[q + 1] <= target) ++q;
    const BInst& I = P.inst[q];
    const double per_tile = tile_work(I);
    int64_t t = P.tile_off[q] + (int64_t)((target - wsum[q]) / per_tile);
    t = std::min(std::max(t, P.cta_tile[c - 1]), P.tile_off[q + 1]);
    P.cta_tile[c] = t;
  }
  return KM_OK;
}

struct BatchCache {
  uint64_t sig = 0;
  BatchTune tune{128, 0, 1};
};

struct BatchCtx {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* host = nullptr;
  size_t host_bytes = 0;
  cudaGraphExec_t gexec = nullptr;
  int graph_kernels = 0;  // kernel nodes of the cached graph
  std::vector<unsigned char> gkey;
  std::vector<unsigned char> tkey;  // the plan whose tables and tensor maps the workspace holds
  std::vector<BatchCache> tuned;
  // the last plan, reused while the caller's instances, precision and launch shape repeat
  BatchPlan plan;
  std::vector<km_instance> plan_in;
  BatchTune plan_tune{0, -1, -1};
  int plan_prec = -1;
};

BatchCtx g_batch[64];

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
  return h;
}

// Shape signature of a batch for the tuning cache: (n, d, k) of every instance.
uint64_t batch_signature(const km_instance* in, int count, int precision) {
  uint64_t h = fnv1a(&precision, sizeof precision);
  for (int b = 0; b < count; ++b) {
    h = fnv1a(&in[b].n, sizeof in[b].n, h);
    h = fnv1a(&in[b].d, sizeof in[b].d, h);
    h = fnv1a(&in[b].k, sizeof in[b].k, h);
  }
  return h;
}

// Byte offsets of the batch workspace.
struct BLayout {
  size_t ctl, inst, row, tile, seg, cta, rch, kci, kpi, maps, maps_s, slots, xs, xss, labs, perm, flags, offs, cur,
      sums, hq, scq, cst, xq, xqs, cq, csave, hist, total;
};

BLayout batch_layout(const BatchPlan& P, int iters) {
  BLayout L;
  const int nb = (int)P.inst.size();
  size_t off = 0;
  auto take = [&](size_t bytes, size_t al = 256) {
    off = (off + al - 1) / al * al;
    const size_t at = off;
    off += bytes;
    return at;
  };
  L.ctl = take(sizeof(Ctl) * nb);
  L.inst = take(sizeof(BInst) * nb);
  L.row = take(8 * (nb + 1));
  L.tile = take(8 * (nb + 1));
  L.seg = take(sizeof(BChunk) * P.sitems.size());
  L.cta = take(8 * P.cta_tile.size());
  L.rch = take(sizeof(BChunk) * P.rchunks.size());
  L.kci = take(4 * P.kc_inst.size());
  L.kpi = take(4 * P.kp_inst.size());
  L.maps = take(sizeof(CUtensorMap) * 2 * nb, 128);
  L.maps_s = take(sizeof(CUtensorMap) * nb, 128);
  L.slots = take(8);
  L.xs = take(16 * (size_t)P.R);
  L.xss = take(16 * (size_t)P.R);
  L.labs = take(4 * (size_t)P.R);
  L.perm = take(4 * (size_t)P.R);
  L.flags = take(sizeof(FlagRec) * (size_t)P.R);
  L.offs = take(4 * (size_t)(P.KP + nb));
  L.cur = take(4 * (size_t)P.KP);
  L.sums = take(8 * (size_t)P.SUMS);
  L.hq = take(4 * (size_t)P.KP);
  L.scq = take(4 * (size_t)P.KP);
  L.cst = take(16 * (size_t)P.KP);
  L.xq = take((size_t)P.XQ);
  L.xqs = take((size_t)P.XQS);
  L.cq = take((size_t)P.CQ);
  L.csave = take(4 * (size_t)P.CSAVE);
  L.hist = take((8 * 5 + 4) * (size_t)nb * iters);
  L.total = off;
  return L;
}

// Copies every instance's C back from the copy taken on entry of the last run.
int restore_batch_c(const BatchCtx& bc, const BatchPlan& P, int iters, cudaStream_t s) {
  const BLayout BL = batch_layout(P, iters);
  char* B = (char*)bc.ws;
  KM_CUDA(launch_b_copy_c((const BInst*)(B + BL.inst), (int)P.inst.size(), (float*)(B + BL.csave), 1, s));
  KM_CUDA(cudaStreamSynchronize(s));
  return KM_OK;
}

// Runs `iters` steps of the planned batch; the caller holds the device lock.
int run_batch_locked(DevCtx* c, BatchCtx& bc, const km_opts& o, const BatchPlan& P, int iters, double tol,
                     km_stats* per_inst, const int* caller_index, float* ms_out) {
  int rc = init_ctx(c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  const int nb = (int)P.inst.size();
  const BLayout BL = batch_layout(P, iters);
  const size_t o_ctl = BL.ctl, o_inst = BL.inst, o_row = BL.row, o_tile = BL.tile,
               o_maps = BL.maps, o_slots = BL.slots, o_xs = BL.xs, o_xss = BL.xss, o_labs = BL.labs,
               o_perm = BL.perm, o_flags = BL.flags, o_offs = BL.offs, o_cur = BL.cur, o_sums = BL.sums,
               o_hq = BL.hq, o_scq = BL.scq, o_xq = BL.xq, o_cq = BL.cq, o_csave = BL.csave, o_hist = BL.hist;
  const size_t off = BL.total;
  const size_t need = off;
  if (need > bc.ws_bytes) {
    if (bc.ws) {
      KM_CUDA(cudaDeviceSynchronize());
      cudaFree(bc.ws);
      bc.ws = nullptr;
      bc.ws_bytes = 0;
    }
    bc.gkey.clear();
    bc.tkey.clear();
    const size_t want = align_up(need + need / 4, 1 << 20);
    if (cudaMalloc(&bc.ws, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "batch workspace allocation of %zu bytes failed", want);
    }
    bc.ws_bytes = want;
  }
  char* B = (char*)bc.ws;
  BWork W;
  memset(&W, 0, sizeof W);
  W.inst = (const BInst*)(B + o_inst);
  W.nb = nb;
  W.iters = iters;
  W.row_off = (const int64_t*)(B + o_row);
  W.tile_off = (const int64_t*)(B + o_tile);
  W.sitems = (const BChunk*)(B + BL.seg);
  W.nsitems = (int64_t)P.sitems.size();
  W.cta_tile = (const int64_t*)(B + BL.cta);
  W.cta_grid = (int)P.cta_tile.size() - 1;
  W.rchunks = (const BChunk*)(B + BL.rch);
  W.nrchunks = (int)P.rchunks.size();
  W.kmax = P.kmax;
  W.kc_inst = (const int32_t*)(B + BL.kci);
  W.kp_inst = (const int32_t*)(B + BL.kpi);
  W.R = P.R;
  W.KC = P.KC;
  W.KP = P.KP;
  W.T = P.T;
  W.ctls = (Ctl*)(B + o_ctl);
  W.flag_slots = (unsigned long long*)(B + o_slots);
  W.maps = (const CUtensorMap*)(B + o_maps);
  W.maps_s = (const CUtensorMap*)(B + BL.maps_s);
  W.xs = (float4*)(B + o_xs);
  W.xs_sorted = (float4*)(B + o_xss);
  W.lab_sorted = (int32_t*)(B + o_labs);
  W.perm = (int32_t*)(B + o_perm);
  W.flags = (FlagRec*)(B + o_flags);
  W.offs = (int32_t*)(B + o_offs);
  W.cursor = (int32_t*)(B + o_cur);
  W.sums64 = (double*)(B + o_sums);
  W.hq = (float*)(B + o_hq);
  W.scq = (float*)(B + o_scq);
  W.cst = (float4*)(B + BL.cst);
  W.Xq = (uint8_t*)(B + o_xq);
  W.Xqs = (uint8_t*)(B + BL.xqs);
  W.Cq = (uint8_t*)(B + o_cq);
  char* hb = B + o_hist;
  W.obj_hist = (double*)hb;
  W.shift_hist = W.obj_hist + (size_t)nb * iters;
  W.changed_hist = (unsigned long long*)(W.shift_hist + (size_t)nb * iters);
  W.flagged_hist = W.changed_hist + (size_t)nb * iters;
  W.full_hist = W.flagged_hist + (size_t)nb * iters;
  W.empty_hist = (int*)(W.full_hist + (size_t)nb * iters);
  // Tables and tensor maps depend on the plan and the workspace only: they are
  // uploaded when either changed since the last call (nothing writes them on the device).
  std::vector<unsigned char> tk(sizeof(BInst) * nb);
  memcpy(tk.data(), P.inst.data(), tk.size());
  {
    auto tapp = [&](const void* v, size_t n) { tk.insert(tk.end(), (const unsigned char*)v, (const unsigned char*)v + n); };
    void* base = bc.ws;
    tapp(&base, sizeof base);
    tapp(&P.bn, sizeof P.bn);
    tapp(&P.sorted, sizeof P.sorted);
    tapp(&P.fp8, sizeof P.fp8);
    const size_t nt = P.cta_tile.size(), ns = P.sitems.size();
    tapp(&nt, sizeof nt);
    tapp(&ns, sizeof ns);
  }
  if (bc.tkey != tk) {
    bc.tkey.clear();
    // tensor maps of every instance's codes
    std::vector<CUtensorMap> maps(3 * nb);  // codes of X, codes of C; then the sorted copies
    memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
    const int esz = P.fp8 ? 1 : 2;
    for (int b = 0; b < nb; ++b) {
      const BInst& I = P.inst[b];
      if ((rc = encode_codes_map(&maps[2 * b], W.Xq + I.xq_off, I.n, I.Kp, esz, 128, I.rowb))) return rc;
      if ((rc = encode_codes_map(&maps[2 * b + 1], W.Cq + I.cq_off, I.kp, I.Kp, esz, I.bn, I.rowb))) return rc;
      if (I.gsort && (rc = encode_codes_map(&maps[2 * nb + b], W.Xqs + I.xqs_off, I.n, I.Kp, esz, 128, I.rowb)))
        return rc;
    }
    KM_CUDA(cudaMemcpyAsync(B + o_inst, P.inst.data(), sizeof(BInst) * nb, cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + o_row, P.row_off.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + o_tile, P.tile_off.data(), 8 * (nb + 1), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + BL.seg, P.sitems.data(), sizeof(BChunk) * P.sitems.size(), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + BL.cta, P.cta_tile.data(), 8 * P.cta_tile.size(), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + BL.rch, P.rchunks.data(), sizeof(BChunk) * P.rchunks.size(), cudaMemcpyHostToDevice,
                            s));
    KM_CUDA(cudaMemcpyAsync(B + BL.kci, P.kc_inst.data(), 4 * P.kc_inst.size(), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + BL.kpi, P.kp_inst.data(), 4 * P.kp_inst.size(), cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + o_maps, maps.data(), sizeof(CUtensorMap) * 2 * nb, cudaMemcpyHostToDevice, s));
    KM_CUDA(cudaMemcpyAsync(B + BL.maps_s, maps.data() + 2 * nb, sizeof(CUtensorMap) * nb, cudaMemcpyHostToDevice, s));
    // pageable sources: the copies are staged before cudaMemcpyAsync returns, so `maps` may go
    bc.tkey.swap(tk);
  }
  KM_CUDA(cudaMemsetAsync(W.ctls, 0, sizeof(Ctl) * nb, s));
  KM_CUDA(cudaMemsetAsync(W.sums64, 0, 8 * (size_t)P.SUMS, s));
  // C on entry, restored on error
  KM_CUDA(launch_b_copy_c(W.inst, nb, (float*)(B + o_csave), 0, s));
  if (o.profile && (rc = ensure_events(c, 2 + (size_t)iters * kEvPerStep))) return rc;
  KM_CUDA(cudaEventRecord(c->ev0, s));
  if (o.profile) KM_CUDA(cudaEventRecord(c->prof[0], s));
  KM_CUDA(launch_b_quant_x(W, P.fp8, s));
  if (o.profile) KM_CUDA(cudaEventRecord(c->prof[1], s));
  // graph of the iterations, cached while the batch and its workspace are unchanged
  std::vector<unsigned char> key(sizeof(BInst) * nb);
  memcpy(key.data(), P.inst.data(), key.size());
  auto app = [&](const void* v, size_t n) { key.insert(key.end(), (const unsigned char*)v, (const unsigned char*)v + n); };
  app(&iters, sizeof iters);
  app(&tol, sizeof tol);
  app(&o.recheck, sizeof o.recheck);
  app(&o.warm_start, sizeof o.warm_start);
  app(&P.bn, sizeof P.bn);
  app(&P.sorted, sizeof P.sorted);
  app(&o.profile, sizeof o.profile);
  void* base = bc.ws;
  app(&base, sizeof base);
  if (!(bc.gexec && bc.gkey == key)) {
    if (bc.gexec) {
      cudaGraphExecDestroy(bc.gexec);
      bc.gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    KM_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    const uint32_t idesc = tc::idesc_f32acc(P.fp8 ? 0u : 1u, 128, (uint32_t)P.bn);
    cudaStream_t cs = c->cap_stream;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
      // stage boundaries as in enqueue_step (events only when profiling)
      const cudaEvent_t* ev = step_events(c, o.profile != 0, it);
      auto at = [&](int i) { return ev ? mark(ev[i], cs) : cudaSuccess; };
      if (!e) e = launch_b_reset(W, cs);
      if (!e) e = at(0);
      if (!e) e = launch_b_quant_c(W, P.fp8, cs);
      if (!e) e = at(1);
      if (!e)
        e = launch_b_assign(W, P.fp8, it == 0 && !o.warm_start, it > 0 && P.sorted, P.nkb_max, P.kp_max, P.bn,
                            P.stages, P.abufs,
                            idesc, cs);
      if (!e) e = at(2);
      if (!e && o.recheck) e = launch_b_recheck(W, cs);
      if (!e) e = at(3);
      if (!e) e = launch_b_count(W, cs);
      if (!e) e = at(4);
      if (!e) e = launch_b_scan(W, cs);
      if (!e) e = at(5);
      if (!e) e = launch_b_scatter(W, cs);
      if (!e && P.sorted && it + 1 < iters) e = launch_b_permute(W, cs);  // the next step's sorted code copies
      if (!e) e = at(6);
      if (!e) e = launch_b_segsum(W, cs);
      if (!e) e = at(7);
      if (!e) e = launch_b_divide(W, tol, cs);
      if (!e) e = at(8);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return fail(KM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e ? e : e2));
    }
    bc.graph_kernels = kernel_nodes(g);
    e = cudaGraphInstantiate(&bc.gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      bc.gexec = nullptr;
      return fail(KM_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
    }
    bc.gkey = key;
  }
  KM_CUDA(cudaGraphLaunch(bc.gexec, s));
  KM_CUDA(cudaEventRecord(c->ev1, s));
  // read back control blocks and histories
  const size_t hist_bytes = (8 * 5 + 4) * (size_t)nb * iters, host_need = sizeof(Ctl) * nb + hist_bytes + 64;
  if (host_need > bc.host_bytes) {
    if (bc.host) cudaFreeHost(bc.host);
    bc.host = nullptr;
    bc.host_bytes = 0;
    if (cudaMallocHost(&bc.host, host_need) != cudaSuccess) {
      cudaGetLastError();
      return fail(KM_ENOMEM, "pinned host allocation failed");
    }
    bc.host_bytes = host_need;
  }
  Ctl* hc = (Ctl*)bc.host;
  char* hh = (char*)bc.host + align_up(sizeof(Ctl) * nb, 64);
  KM_CUDA(cudaMemcpyAsync(hc, W.ctls, sizeof(Ctl) * nb, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hh, hb, hist_bytes, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (ms_out) *ms_out = ms;
  float stage_ms[12] = {0.f};
  if (o.profile) {
    float t = 0.f;
    KM_CUDA(cudaEventElapsedTime(&t, c->prof[0], c->prof[1]));
    stage_ms[KM_STAGE_XNORM] = t;
    for (int it = 0; it < iters; ++it) {
      const cudaEvent_t* ev = step_events(c, true, it);
      for (int sg = 0; sg < kEvPerStep - 1; ++sg) {
        KM_CUDA(cudaEventElapsedTime(&t, ev[sg], ev[sg + 1]));
        stage_ms[KM_STAGE_PREP + sg] += t;
      }
    }
  }
  bool bad = false;
  int err = 0;
  for (int b = 0; b < nb; ++b) {
    if (hc[b].nonfinite) bad = true;
    if (hc[b].error) err = hc[b].error;
  }
  if (bad || err) {
    if ((rc = restore_batch_c(bc, P, iters, s))) return rc;
    if (bad) return fail(KM_ENONFINITE, "an instance holds a non-finite value (or a norm overflows FP32)");
    return fail(err, "device stage reported error %d", err);
  }
  if (per_inst) {
    const double* ho = (const double*)hh;
    const double* hs = ho + (size_t)nb * iters;
    const unsigned long long* hch = (const unsigned long long*)(hs + (size_t)nb * iters);
    const unsigned long long* hf = hch + (size_t)nb * iters;
    const unsigned long long* hfu = hf + (size_t)nb * iters;
    const int* he = (const int*)(hfu + (size_t)nb * iters);
    for (int b = 0; b < nb; ++b) {
      km_stats& st = per_inst[caller_index[b]];
      memset(&st, 0, sizeof st);
      st.iters_done = hc[b].iters_done;
      const int last = hc[b].iters_done - 1;
      if (last >= 0) {
        const size_t h = (size_t)b * iters + last;
        st.objective = ho[h];
        st.shift = hs[h];
        st.n_changed = (int64_t)hch[h];
        st.n_flagged = (int64_t)hf[h];
        st.n_full = (int64_t)hfu[h];
        st.n_empty = he[h];
      }
      st.ms = ms;
      st.launches = 1 + bc.graph_kernels;  // the whole batch's launches (point quantisation + graph),
                                           // reported for every instance
      memcpy(st.stage_ms, stage_ms, sizeof stage_ms);
      st.batch_shape = P.shape;
    }
  }
  return KM_OK;
}

}  // namespace

KM_API int kmeans_run_batched(const km_opts* opts, const km_instance* inst, int32_t count, int32_t iters,
                              double tol, km_stats* per_inst) {
  g_err.clear();
  const km_opts o = resolve(opts);
  if (!inst || count < 1) return fail(KM_EINVAL, "need count >= 1 instances");
  if (iters < 1) return fail(KM_EINVAL, "iters = %d < 1", iters);
  if (o.precision != KM_BF16 && o.precision != KM_FP8E4M3)
    return fail(o.precision == KM_FP32 || o.precision == KM_BF16X3 ? KM_EUNSUPPORTED : KM_EINVAL,
                "batched runs use the tensor-core path: precision must be KM_BF16 or KM_FP8E4M3");
  if (o.deterministic) return fail(KM_EUNSUPPORTED, "deterministic reduces are available for single-instance calls only");
  for (int b = 0; b < count; ++b) {
    const km_instance& s = inst[b];
    if (!s.X || !s.C || !s.assign || !s.sums || !s.counts) return fail(KM_EINVAL, "instance %d: null pointer", b);
    if (s.n < 1 || s.n > INT32_MAX || s.k < 1 || (int64_t)s.k > s.n || s.d < 1 || s.d > 128)
      return fail(KM_EINVAL, "instance %d: need 1 <= k <= n < 2^31 and 1 <= d <= 128", b);
  }
  int dev = 0;
  KM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(KM_EUNSUPPORTED, "device index %d", dev);
  for (int b = 0; b < count; ++b) {
    Problem p{inst[b].X, inst[b].n, inst[b].d, inst[b].C, inst[b].k, inst[b].assign, inst[b].sums, inst[b].counts};
    int rc = validate_device_ptrs(p, dev);
    if (rc) return fail(rc, "instance %d: %s", b, g_err.c_str());
  }
  DevCtx* c = get_ctx(dev);
  std::lock_guard<std::mutex> lk(c->mu);
  c->xc.valid = false;  // this call overwrites the workspace
  BatchCtx& bc = g_batch[dev];
  const uint64_t sig = batch_signature(inst, count, o.precision);
  BatchTune tune{128, 0, 1};
  bool known = false;
  for (const BatchCache& t : bc.tuned)
    if (t.sig == sig) {
      tune = t.tune;
      known = true;
    }
  // test knob: KM_BATCH_SHAPE="bn,order,sorted" runs that launch shape without tuning (every shape must
  // give the same results, so tests cover each one)
  if (const char* fs = getenv("KM_BATCH_SHAPE")) {
    BatchTune f{0, -1, -1};
    if (sscanf(fs, "%d,%d,%d", &f.bn, &f.order, &f.sorted) != 3 || (f.bn != 64 && f.bn != 128) || f.order < 0 ||
        f.order > 1 || f.sorted < 0 || f.sorted > 1)
      return fail(KM_EINVAL, "KM_BATCH_SHAPE must be \"bn,order,sorted\" with bn 64 or 128, order and sorted 0 or 1");
    tune = f;
    known = true;
  }
  int rc;
  if (!known) {
    // autotune: time three steps of every candidate shape on the caller's data, keep the fastest
    const BatchTune cands[8] = {{128, 0, 1}, {128, 1, 1}, {64, 0, 1}, {64, 1, 1},
                                {128, 0, 0}, {128, 1, 0}, {64, 0, 0}, {64, 1, 0}};
    float best = 1e30f;
    for (const BatchTune& cand : cands) {
      BatchPlan P;
      if (plan_batch(inst, count, o.precision, cand, P)) continue;
      std::vector<int> idx(P.order);
      float ms = 0.f;
      // three steps: the sorted order of the codes pays off from the second step on
      if ((rc = run_batch_locked(c, bc, o, P, 3, 0.0, nullptr, idx.data(), &ms))) return rc;
      // the trial steps moved C: put every instance back before the next candidate
      if ((rc = restore_batch_c(bc, P, 3, (cudaStream_t)o.stream))) return rc;
      if (ms < best) {
        best = ms;
        tune = cand;
      }
    }
    bc.tuned.push_back(BatchCache{sig, tune});
  }
  const bool same = bc.plan_prec == o.precision && bc.plan_tune.bn == tune.bn && bc.plan_tune.order == tune.order &&
                    bc.plan_tune.sorted == tune.sorted && bc.plan_in.size() == (size_t)count &&
                    memcmp(bc.plan_in.data(), inst, sizeof(km_instance) * count) == 0;
  if (!same) {
    bc.plan_prec = -1;
    if ((rc = plan_batch(inst, count, o.precision, tune, bc.plan))) return rc;
    bc.plan_in.assign(inst, inst + count);
    bc.plan_tune = tune;
    bc.plan_prec = o.precision;
  }
  return run_batch_locked(c, bc, o, bc.plan, iters, tol, per_inst, bc.plan.order.data(), nullptr);
}
