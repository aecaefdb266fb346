// Diagnostics behind the library's accuracy argument and its roofline figures
// (declared in include/kmeans.h, section "Diagnostics"):
//
// kmeans_probe_mma -- one 128 x 128 output tile of the tensor-core contraction
//   exactly as the distance kernel forms it: K-major operands in the 128-byte
//   swizzled shared-memory layout, the same shared-memory and instruction
//   descriptors, one tcgen05.mma per 32 bytes of K accumulating into one FP32
//   TMEM accumulator, read back with tcgen05.ld. Tests use it to pin the
//   accumulator model that the near-tie margin rests on (23 kept mantissa bits,
//   truncation; gamma'_K = K 2^-23 / (1 - K 2^-23)) and the operand layout.
// kmeans_probe_ffma -- a device-wide loop of independent FP32 FMA chains
//   (scalar FFMA or packed FFMA2), timed with CUDA events: the measured FP32
//   SIMT peak that the FP32 assignment is compared against.
//
// Neither is on the Lloyd path.
#include <cstdio>

#include <cuda_bf16.h>

#include "km_internal.cuh"
#include "km_tc.cuh"

#define KM_API extern "C" __attribute__((visibility("default")))

namespace km {
namespace {

using namespace tc;

constexpr int PM = 128;          // rows of A (M) and of B (N)
constexpr uint32_t PROW = 128;   // bytes of one K block row
constexpr int PMAX_KB = 4;       // K blocks (128 bytes of K each)

// A: [128][nkb * 128 B] codes, B: [128][nkb * 128 B]; D: [128][128] FP32 (row m, column n).
template <int FP8>
__global__ void __launch_bounds__(128, 1)
probe_mma_kernel(const uint8_t* __restrict__ A, const uint8_t* __restrict__ B, int nkb, float* __restrict__ D,
                 int* __restrict__ status) {
  extern __shared__ uint8_t psmem_raw[];
  uint8_t* smem = psmem_raw + ((1024u - ((uint32_t)__cvta_generic_to_shared(psmem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t done_bar;
  __shared__ uint32_t tmem_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t blk = PM * PROW;  // one K block of one operand
  uint8_t* As = smem;
  uint8_t* Bs = smem + nkb * blk;
  const int rowb = nkb * (int)PROW;  // bytes of one global row

  // global rows -> shared K blocks, 16-byte chunk c of row r stored at chunk c ^ (r & 7)
  // (the 128-byte swizzle that TMA applies in the distance kernel)
  for (int e = threadIdx.x; e < 2 * PM * nkb * 8; e += blockDim.x) {
    const int op = e / (PM * nkb * 8);
    const int rem = e % (PM * nkb * 8);
    const int r = rem / (nkb * 8), kb = (rem / 8) % nkb, c = rem % 8;
    const uint8_t* src = (op ? B : A) + (size_t)r * rowb + kb * PROW + c * 16;
    uint8_t* dst = (op ? Bs : As) + kb * blk + r * PROW + ((c ^ (r & 7)) * 16);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
  }
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(&done_bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_s, 128);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_s;
  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_f32acc(FP8 ? 0u : 1u, 128, 128);
    const uint64_t a_desc = sdesc_k_sw128(smem_u32(As)), b_desc = sdesc_k_sw128(smem_u32(Bs));
    for (int kb = 0; kb < nkb; ++kb) {
      const uint64_t a_kb = a_desc + (uint64_t)((kb * blk) >> 4);
      const uint64_t b_kb = b_desc + (uint64_t)((kb * blk) >> 4);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K per instruction
        if constexpr (FP8) mma_fp8(tmem, a_kb + (uint64_t)(kk * 2), b_kb + (uint64_t)(kk * 2), idesc, (kb | kk) != 0);
        else mma_bf16(tmem, a_kb + (uint64_t)(kk * 2), b_kb + (uint64_t)(kk * 2), idesc, (kb | kk) != 0);
      }
    }
    mma_commit(&done_bar);
  }
  __syncwarp();
  int no_abort = 0;
  const bool ok = mbar_wait(&done_bar, 0, &no_abort, 1000000000ull);  // 1 s bound
  if (!ok && lane == 0) atomicExch(status, (int)KM_ETIMEOUT);
  tc_fence_after_sync();
  if (__all_sync(0xffffffffu, ok)) {
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t v[32];
    for (int cb = 0; cb < 4; ++cb) {
      tmem_ld_32x32b_x32(trow + (uint32_t)(cb * 32), v);
      tmem_ld_wait();
      float* out = D + (size_t)(warp * 32 + lane) * 128 + cb * 32;
#pragma unroll
      for (int t = 0; t < 32; ++t) out[t] = __uint_as_float(v[t]);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tmem, 128);
  }
}

// Independent FMA chains: 16 FP32 FMAs per thread and iteration (16 scalar
// chains, or 8 packed two-lane chains).
template <bool PACKED>
__global__ void __launch_bounds__(256)
ffma_peak_kernel(float* __restrict__ sink, int iters, float m, float c) {
  float acc = 0.f;
  if constexpr (PACKED) {
    float2 x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = make_float2(threadIdx.x * 1e-3f + u, 0.5f * u);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ffma2_rn(x[u], m2, c2);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += x[u].x + x[u].y;
  } else {
    float x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) x[u] = threadIdx.x * 1e-3f + u;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 16; ++u) x[u] = fmaf(x[u], m, c);
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) acc += x[u];
  }
  if (acc == -1.f) sink[blockIdx.x] = acc;  // never true for the inputs used: keeps the chains live
}

int probe_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
  set_last_error(buf);
  return code;
}

}  // namespace
}  // namespace km

using namespace km;

KM_API int kmeans_probe_mma(int32_t precision, const void* A, const void* B, int32_t K, float* D, void* stream) {
  set_last_error("");
  if (precision != KM_BF16 && precision != KM_FP8E4M3)
    return probe_fail(KM_EINVAL, "kmeans_probe_mma: precision must be KM_BF16 or KM_FP8E4M3");
  const int esz = precision == KM_BF16 ? 2 : 1;
  const int kbe = 128 / esz;
  if (K < kbe || K > PMAX_KB * kbe || K % kbe != 0)
    return probe_fail(KM_EINVAL, "kmeans_probe_mma: K must be 1 to 4 whole 128-byte K blocks");
  if (!A || !B || !D) return probe_fail(KM_EINVAL, "kmeans_probe_mma: null pointer");
  if (((uintptr_t)A | (uintptr_t)B) & 15u) return probe_fail(KM_EINVAL, "kmeans_probe_mma: A and B must be 16-byte aligned");
  const int nkb = K / kbe;
  cudaStream_t s = (cudaStream_t)stream;
  int* status = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&status, sizeof(int), s);
  if (e != cudaSuccess) return probe_fail(KM_ECUDA, "kmeans_probe_mma: status allocation", e);
  const size_t smem = 1024 + 2 * (size_t)nkb * PM * PROW;
  e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    if (esz == 1) {
      e = cudaFuncSetAttribute(probe_mma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        probe_mma_kernel<1><<<1, 128, smem, s>>>((const uint8_t*)A, (const uint8_t*)B, nkb, D, status);
    } else {
      e = cudaFuncSetAttribute(probe_mma_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        probe_mma_kernel<0><<<1, 128, smem, s>>>((const uint8_t*)A, (const uint8_t*)B, nkb, D, status);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(status, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return probe_fail(KM_ECUDA, "kmeans_probe_mma", e);
  if (hs) return probe_fail(hs, "kmeans_probe_mma: the MMA completion wait expired");
  return KM_OK;
}

KM_API int kmeans_probe_ffma(int32_t packed, int32_t iters, double* flops, float* ms, void* stream) {
  set_last_error("");
  if (iters < 1 || !flops || !ms) return probe_fail(KM_EINVAL, "kmeans_probe_ffma: iters >= 1, flops and ms required");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_fail(KM_ECUDA, "kmeans_probe_ffma", e);
  const int blocks = sms * 8;  // 8 CTAs of 256 threads: 64 warps per SM
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMallocAsync((void**)&sink, (size_t)blocks * sizeof(float), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    if (packed) ffma_peak_kernel<true><<<blocks, 256, 0, s>>>(sink, iters, 0.99999f, 1e-5f);
    else ffma_peak_kernel<false><<<blocks, 256, 0, s>>>(sink, iters, 0.99999f, 1e-5f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (sink) cudaFreeAsync(sink, s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return probe_fail(KM_ECUDA, "kmeans_probe_ffma", e);
  *ms = t;
  *flops = 2.0 * 16.0 * (double)iters * (double)blocks * 256.0;
  return KM_OK;
}
