// C ABI of the fused Lloyd k-means library: argument validation, the per-device
// context and workspace, the stage sequence of one Lloyd step, graph capture of
// multi-step runs, and statistics. Declarations and contracts: include/kmeans.h.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
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
  size_t stage_bytes = 0;
  void* host = nullptr;   // pinned read-back of Ctl and the per-step history
  size_t host_bytes = 0;
  bool graph_valid = false;
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
  c->inited = true;
  return KM_OK;
}

size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

// Shape of the tensor-core path for (d, k, precision).
struct TcShape {
  int fp8, esz, Kp, nkb, bn, kp, nchunks, stages;
};

TcShape tc_shape(int precision, int d, int k) {
  TcShape t{};
  t.fp8 = precision == KM_FP8E4M3;
  t.esz = t.fp8 ? 1 : 2;
  const int kbe = 128 / t.esz;
  t.Kp = (d + kbe - 1) / kbe * kbe;
  t.nkb = t.Kp / kbe;
  t.bn = t.nkb <= 2 ? 128 : 64;
  t.kp = (k + t.bn - 1) / t.bn * t.bn;
  t.nchunks = t.kp / t.bn;
  // dynamic shared memory: 227 KB opt-in, minus 1 KB of alignment slack and 1 KB for static smem
  const size_t budget = 227 * 1024 - 1024 - 1024;
  const size_t a = 2 * (size_t)t.nkb * 128 * 128, b = (size_t)t.nkb * t.bn * 128;
  t.stages = a + 2 * b <= budget ? (int)std::min<size_t>(8, (budget - a) / b) : 0;
  return t;
}

struct Layout {
  size_t ctl, xnorm, flags, perm, offs, cursor, sums64, chalf, cnorm, Csave, obj, shift, changed,
      flagged, full, empty, Xq, xs, Cq, hsc, state, total;
};

Layout layout_for(int64_t n, int k, int d, int iters, int precision) {
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
  L.obj = take(8 * (size_t)iters);
  L.shift = take(8 * (size_t)iters);
  L.changed = take(8 * (size_t)iters);
  L.flagged = take(8 * (size_t)iters);
  L.full = take(8 * (size_t)iters);
  L.empty = take(4 * (size_t)iters);
  if (precision != KM_FP32) {
    const TcShape t = tc_shape(precision, d, k);
    L.Xq = take((size_t)n * t.Kp * t.esz);
    L.xs = take(16 * (size_t)n);
    L.Cq = take((size_t)t.kp * t.Kp * t.esz);
    L.hsc = take(8 * (size_t)t.kp);
    L.state = 0;
  } else {
    L.Xq = L.xs = L.Cq = L.hsc = 0;
    const int width = simt_slab_width(d);
    L.state = (width > 0 && width < k) ? take(16 * (size_t)n) : 0;
  }
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
  w.Xq = L.Xq ? (uint8_t*)(b + L.Xq) : nullptr;
  w.xs = L.xs ? (float4*)(b + L.xs) : nullptr;
  w.Cq = L.Cq ? (uint8_t*)(b + L.Cq) : nullptr;
  w.hsc = L.hsc ? (float2*)(b + L.hsc) : nullptr;
  w.state = L.state ? (float4*)(b + L.state) : nullptr;
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
int encode_codes_map(CUtensorMap* m, void* base, int64_t rows, int Kp, int esz, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(KM_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(KM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return KM_OK;
}

// Per-call state of a step sequence: precision, recheck switch, tensor-core launch data.
struct StepCfg {
  int precision;
  int recheck;
  int warm;  // assign holds a valid assignment on entry
  TcShape t;
  TcLaunch L;
  TcParams P;
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

// Argument checks that need no CUDA call.
int validate_args(const km_opts& o, const Problem& p, int iters) {
  if (!p.X || !p.C || !p.assign || !p.sums || !p.counts) return fail(KM_EINVAL, "null array pointer");
  if (p.n < 1 || p.n > INT32_MAX) return fail(KM_EINVAL, "n = %lld outside [1, 2^31)", (long long)p.n);
  if (p.k < 1 || (int64_t)p.k > p.n) return fail(KM_EINVAL, "k = %d outside [1, n]", p.k);
  if (p.d < 1 || p.d > kMaxD) return fail(KM_EINVAL, "d = %d outside [1, %d]", p.d, kMaxD);
  if (iters < 1) return fail(KM_EINVAL, "iters = %d < 1", iters);
  if (o.precision != KM_FP32 && o.precision != KM_BF16 && o.precision != KM_FP8E4M3)
    return fail(KM_EINVAL, "unknown precision %d", o.precision);
  if (o.precision != KM_FP32 && tc_shape(o.precision, p.d, p.k).stages < 2)
    return fail(KM_EUNSUPPORTED, "d = %d does not fit the tensor-core tile pipeline", p.d);
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
cudaError_t enqueue_step(const Problem& p, const Work& w, const StepCfg& cfg, int first, double tol,
                         cudaStream_t s, const cudaEvent_t* ev) {
  cudaError_t e;
  auto at = [&](int i) { return ev ? mark(ev[i], s) : cudaSuccess; };
  const bool tcp = cfg.precision != KM_FP32;
  if ((e = cudaMemsetAsync(w.ctl, 0, kCtlIterBytes, s))) return e;
  if ((e = at(0))) return e;
  if (tcp) e = launch_quant_c(p, w, cfg.t.fp8, cfg.t.kp, cfg.t.Kp, w.Cq, w.hsc, s);
  else e = launch_prep(p, w, s);
  if (e) return e;
  if ((e = at(1))) return e;
  if (tcp) {
    TcParams P = cfg.P;
    P.first = first;
    e = launch_assign_tc(p, cfg.L, P, s);
  } else {
    e = launch_assign_simt(p, w, first, s);
  }
  if (e) return e;
  if ((e = at(2))) return e;
  if (cfg.recheck && (e = launch_recheck(p, w, first, s))) return e;
  if ((e = at(3))) return e;
  if ((e = launch_count(p, w, s))) return e;
  if ((e = at(4))) return e;
  if ((e = launch_scan(p, w, s))) return e;
  if ((e = at(5))) return e;
  if ((e = launch_scatter(p, w, s))) return e;
  if ((e = at(6))) return e;
  if ((e = launch_segsum(p, w, s))) return e;
  if ((e = at(7))) return e;
  if ((e = launch_divide(p, w, first ? 0 : 1, tol, s))) return e;
  if ((e = at(8))) return e;
  return cudaSuccess;
}

const cudaEvent_t* step_events(DevCtx* c, bool profile, int it) {
  return profile ? c->prof.data() + 2 + (size_t)it * kEvPerStep : nullptr;
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
    e = enqueue_step(p, w, cfg, it == 0 && !cfg.warm, tol, c->cap_stream, step_events(c, profile, it));
  cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(KM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e ? e : e2));
  }
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

// Runs `iters` steps on device arrays. The caller holds c->mu.
int run_locked(DevCtx* c, const km_opts& o, const Problem& p, int iters, double tol, bool graph,
               km_stats* st) {
  int rc = init_ctx(c);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)o.stream;
  const Layout L = layout_for(p.n, p.k, p.d, iters, o.precision);
  if ((rc = ensure_ws(c, L, s))) return rc;
  const size_t host_need = sizeof(Ctl) + (size_t)iters * (8 * 5 + 4) + 64;
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
  const Work w = make_work(c, L);
  const bool profile = o.profile != 0;
  StepCfg cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.precision = o.precision;
  cfg.recheck = o.recheck;
  cfg.warm = o.warm_start;
  if (o.precision != KM_FP32) {
    cfg.t = tc_shape(o.precision, p.d, p.k);
    cfg.L.fp8 = cfg.t.fp8;
    if ((rc = encode_codes_map(&cfg.L.mapX, w.Xq, p.n, cfg.t.Kp, cfg.t.esz, 128))) return rc;
    if ((rc = encode_codes_map(&cfg.L.mapC, w.Cq, cfg.t.kp, cfg.t.Kp, cfg.t.esz, cfg.t.bn))) return rc;
    TcParams& P = cfg.P;
    P.hsc = w.hsc;
    P.xs = w.xs;
    P.Cq = w.Cq;
    P.assign = p.assign;
    P.flags = w.flags;
    P.ctl = w.ctl;
    P.n = p.n;
    P.k = p.k;
    P.Kp = cfg.t.Kp;
    P.nkb = cfg.t.nkb;
    P.bn = cfg.t.bn;
    P.nchunks = cfg.t.nchunks;
    P.stages = cfg.t.stages;
    P.idesc = tc::idesc_f32acc(cfg.t.fp8 ? 0u : 1u, 128, (uint32_t)cfg.t.bn);
    const double K = cfg.t.Kp;
    P.gam_tc = (float)(K * 0x1p-23 / (1.0 - K * 0x1p-23) * (1.0 + 1e-6));   // truncating FP32 accumulation
    P.gam_simt = (float)(K * 0x1p-24 / (1.0 - K * 0x1p-24) * (1.0 + 1e-6));
    P.wait_ns = 2000000000ull;
  }
  if (profile && (rc = ensure_events(c, 2 + (size_t)iters * kEvPerStep))) return rc;
  KM_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s));
  KM_CUDA(cudaMemsetAsync(w.sums64, 0, 8 * (size_t)p.k * p.d, s));
  KM_CUDA(cudaMemcpyAsync(w.Csave, p.C, (size_t)p.k * p.d * 4, cudaMemcpyDeviceToDevice, s));
  KM_CUDA(cudaEventRecord(c->ev0, s));
  if (profile) KM_CUDA(cudaEventRecord(c->prof[0], s));
  if (o.precision != KM_FP32) KM_CUDA(launch_quant_x(p, w, cfg.t.fp8, cfg.t.Kp, w.Xq, w.xs, s));
  else KM_CUDA(launch_xnorm(p, w, s));
  if (profile) KM_CUDA(cudaEventRecord(c->prof[1], s));
  if (graph && iters > 1) {
    GraphKey key;
    memset(&key, 0, sizeof key);
    key.X = p.X; key.C = p.C; key.assign = p.assign; key.sums = p.sums; key.counts = p.counts;
    key.n = p.n; key.d = p.d; key.k = p.k; key.iters = iters; key.prec = o.precision; key.tol = tol;
    key.profile = (profile ? 1 : 0) | (o.recheck ? 2 : 0) | (o.warm_start ? 4 : 0);
    key.ws_gen = c->ws_gen;
    cudaGraphExec_t ge = nullptr;
    if ((rc = get_graph(c, key, p, w, cfg, iters, tol, profile, &ge))) return rc;
    KM_CUDA(cudaGraphLaunch(ge, s));
  } else {
    for (int it = 0; it < iters; ++it)
      KM_CUDA(enqueue_step(p, w, cfg, it == 0 && !cfg.warm, tol, s, step_events(c, profile, it)));
  }
  KM_CUDA(cudaEventRecord(c->ev1, s));
  char* h = (char*)c->host;
  Ctl* hc = (Ctl*)h;
  double* hobj = (double*)(h + align_up(sizeof(Ctl), 64));
  double* hshift = hobj + iters;
  unsigned long long* hchanged = (unsigned long long*)(hshift + iters);
  unsigned long long* hflag = hchanged + iters;
  unsigned long long* hfull = hflag + iters;
  int* hempty = (int*)(hfull + iters);
  KM_CUDA(cudaMemcpyAsync(hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hobj, w.obj_hist, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hshift, w.shift_hist, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hchanged, w.changed_hist, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hflag, w.flagged_hist, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hfull, w.full_hist, 8 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaMemcpyAsync(hempty, w.empty_hist, 4 * (size_t)iters, cudaMemcpyDeviceToHost, s));
  KM_CUDA(cudaStreamSynchronize(s));
  if (hc->nonfinite || hc->error) {
    KM_CUDA(cudaMemcpyAsync(p.C, w.Csave, (size_t)p.k * p.d * 4, cudaMemcpyDeviceToDevice, s));
    KM_CUDA(cudaStreamSynchronize(s));
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
    if (last >= 0) {
      st->objective = hobj[last];
      st->shift = hshift[last];
      st->n_changed = (int64_t)hchanged[last];
      st->n_flagged = (int64_t)hflag[last];
      st->n_full = (int64_t)hfull[last];
      st->n_empty = hempty[last];
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

KM_API int kmeans_run_host(const km_opts* opts, const float* X, int64_t n, int32_t d, float* C,
                           int32_t k, int32_t* assign, float* sums, int32_t* counts, int32_t iters,
                           double tol, km_stats* stats) {
  g_err.clear();
  const km_opts o = resolve(opts);
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

KM_API const char* kmeans_last_error(void) { return g_err.c_str(); }

KM_API int32_t kmeans_version(void) { return 100; }
