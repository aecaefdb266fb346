// kmeans_reduce_noalloc: the keyed reduce of a Lloyd step (per-cluster counts,
// sums and the objective for a given assignment) for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are off limits --
// inside a host framework that owns every byte of device memory and forbids
// libraries from allocating (serving runtimes with a fixed memory budget,
// plugins of another runtime), and code on a latency-critical path that must
// not hit the device-wide synchronisation cudaFree implies. The regular entry
// points grow a cached workspace with cudaMalloc; this one uses only the
// fixed-size scratch array below, which every GPU that loads the library holds
// until the process exits.
//
// The stage kernels are the ones the regular Lloyd step launches (count, scan,
// scatter, segmented sum); only their scratch pointers point into the static
// array instead of the cudaMalloc'd workspace.
#include <cstring>
#include <mutex>

#include "km_internal.cuh"

#define KM_API extern "C" __attribute__((visibility("default")))

namespace km {
namespace {

// Limits of the no-allocation reduce (the scratch array is sized for them).
constexpr int64_t kNaMaxN = 1 << 20;   // points
constexpr int kNaMaxK = 8192;          // clusters
constexpr int64_t kNaMaxKD = 1 << 18;  // k * d (FP64 partial sums)

constexpr size_t a256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffOffs = a256(sizeof(Ctl));
constexpr size_t kOffCursor = kOffOffs + a256(4 * (kNaMaxK + 1));
constexpr size_t kOffPerm = kOffCursor + a256(4 * kNaMaxK);
constexpr size_t kOffSlab = kOffPerm + a256(4 * kNaMaxN);
constexpr size_t kOffSums = kOffSlab + a256(4 * kNaMaxN);
constexpr size_t kScratchBytes = kOffSums + a256(8 * kNaMaxKD);  // about 10.5 MB

static __device__ __align__(256) unsigned char km_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {nullptr};  // device address of the array, per device
bool g_kernels_ready[64] = {false};   // stage kernels' shared-memory limits raised on this device

int na_fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

// Flags any label outside [0, k); the later stages then return at entry.
__global__ void check_labels_kernel(const int32_t* __restrict__ assign, int64_t n, int k, Ctl* ctl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = assign[i];
    if (j < 0 || j >= k) {
      ctl->done = 1;
      ctl->error = KM_EINVAL;
    }
  }
}

// sums = RN32(FP64 partials); the partials are cleared for the next call.
__global__ void finish_sums_kernel(double* __restrict__ sums64, float* __restrict__ sums, int64_t kd,
                                   const Ctl* ctl) {
  if (ctl->done) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x) {
    sums[e] = (float)sums64[e];
    sums64[e] = 0.0;
  }
}

}  // namespace
}  // namespace km

/*
 * See include/kmeans.h. The first call on a device looks up the device
 * address of the static scratch array (cudaGetSymbolAddress with that device
 * current) and caches it: the address stays valid while the device's primary
 * context lives (a cudaDeviceReset ends it, and the cached address with it).
 * Every call ends with a device-to-host copy and a stream synchronisation, so
 * no call can be captured into a stream or graph.
 */
KM_API int kmeans_reduce_noalloc(const float* X, int64_t n, int32_t d, const float* C, int32_t k,
                                 const int32_t* assign, float* sums, int32_t* counts, double* objective,
                                 void* stream) {
  using namespace km;
  set_last_error("");
  if (!X || !C || !assign || !sums || !counts) return na_fail(KM_EINVAL, "null array pointer");
  if (n < 1 || k < 1 || d < 1 || d > kMaxD) return na_fail(KM_EINVAL, "need n >= 1, k >= 1, 1 <= d <= 256");
  if (n > kNaMaxN || k > kNaMaxK || (int64_t)k * d > kNaMaxKD)
    return na_fail(KM_EINVAL,
                   "size exceeds the no-allocation limit (n <= 1048576, k <= 8192, k*d <= 262144)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return na_fail(KM_ECUDA, "cudaGetDevice failed");
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, km_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return na_fail(KM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_scratch_ptr[dev] = p;
    }
    if (!g_kernels_ready[dev]) {
      if (init_segsum() != cudaSuccess) {
        cudaGetLastError();
        return na_fail(KM_ECUDA, "raising the segmented sum's shared-memory limit failed");
      }
      g_kernels_ready[dev] = true;
    }
    base = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  char* b = (char*)base;
  Work w;
  memset(&w, 0, sizeof w);
  w.ctl = (Ctl*)(b + kOffCtl);
  w.offs = (int32_t*)(b + kOffOffs);
  w.cursor = (int32_t*)(b + kOffCursor);
  w.perm = (int32_t*)(b + kOffPerm);
  w.lab_sorted = (int32_t*)(b + kOffSlab);
  w.sums64 = (double*)(b + kOffSums);
  Problem p{X, n, d, const_cast<float*>(C), k, const_cast<int32_t*>(assign), sums, counts};
  const size_t kd = (size_t)k * d;
  // the array keeps the previous call's contents: clear what must start at zero
  cudaError_t e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s);
  if (!e) e = cudaMemsetAsync(w.sums64, 0, 8 * kd, s);
  if (!e) e = cudaMemsetAsync(counts, 0, 4 * (size_t)k, s);
  if (!e) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > num_sms() * 4) blocks = num_sms() * 4;
    check_labels_kernel<<<blocks, 256, 0, s>>>(assign, n, k, w.ctl);
    e = cudaGetLastError();
  }
  if (!e) e = launch_count(p, w, s);
  if (!e) e = launch_scan(p, w, s);
  if (!e) e = launch_scatter(p, w, s);
  if (!e) e = launch_segsum(p, w, s);
  if (!e) {
    int blocks = (int)((kd + 255) / 256);
    if (blocks > num_sms() * 4) blocks = num_sms() * 4;
    finish_sums_kernel<<<blocks, 256, 0, s>>>(w.sums64, sums, (int64_t)kd, w.ctl);
    e = cudaGetLastError();
  }
  Ctl hc;
  if (!e) e = cudaMemcpyAsync(&hc, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) {
    cudaGetLastError();
    return na_fail(KM_ECUDA, cudaGetErrorString(e));
  }
  if (hc.error) return na_fail(KM_EINVAL, "assign holds a label outside [0, k)");
  if (objective) *objective = hc.objective;
  return KM_OK;
}
