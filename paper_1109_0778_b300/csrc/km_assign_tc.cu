// Tensor-core fused distance + argmin (BF16 or FP8-E4M3 operands, FP32 accumulate).
//
// One pass per 128-point row tile (vertical fusion with array contraction,
// Sec. 3.5): TMA stages the point codes (A, once per tile) and 128-centroid
// chunks of the centroid codes (B) into shared memory with the 128-byte
// swizzle; one thread issues tcgen05.mma into a TMEM accumulator (two buffers,
// so the MMA of chunk c+1 overlaps the epilogue of chunk c); four epilogue
// warps read their TMEM lane quarter with tcgen05.ld -- thread t of warp q
// owns point row 32q + t -- and fold the chunk's scores into a per-row
// candidate list in registers. The n x k score matrix never leaves TMEM.
//
// Roles (192 threads): warp 0 = TMA producer, warp 1 = MMA issuer and TMEM
// owner, warps 2-5 = epilogue. Every mbarrier wait is bounded in time; on
// expiry the kernel records KM_ETIMEOUT, drains what it issued, frees TMEM and
// returns.
//
// Scores. With codes q and power-of-two row scales (x~ = sx q_x, c~ = sc q_c;
// BF16 uses sx = sc = 1), the epilogue computes
//   s^_j = h_j - (sx sc_j) acc_j,  acc_j = sum_t q_x,t q_c,jt  (TMEM, FP32),
// whose argmin over j is the distance argmin up to the quantisation error.
//
// Error bound (u = 2^-24; the tensor core accumulates in FP32 with truncation,
// so gamma'_K = K 2^-23 / (1 - K 2^-23)): for every j
//   |s^_j - s_j| <= E_i = 3u H + (gamma'_K + 2u) ||x~_i|| C~max
//                       + ||dx_i|| Cmax + ||x_i|| DCmax + ||dx_i|| DCmax,
// where dx = x~ - x, dc = c~ - c, and H, Cmax, C~max, DCmax are the per-step
// maxima over the centroids (hoisted, Sec. 3.1). With margin_i = 2 E_i
// (1 + 2^-10), the true argmin is among the candidates {j : s^_j - s^_1 <=
// margin_i}. A row whose only candidate is j1 is final; otherwise its
// candidates (or, past 4 of them, all k) go to the FP32 re-check.
//
// Threshold. Rows keep the 4 smallest scores seen among elements <= thr, with
// thr = min(thr0, best + margin) rounded up. From the second step on thr0 is
// the score of the point's previous centroid, recomputed from the same codes
// in FP32 SIMT (plus its bound against the tensor-core sum and the margin), so
// a 32-column chunk costs one minimum unless it holds a candidate.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"
#include "km_tc.cuh"

namespace km {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int NTHREADS = 192;
constexpr uint32_t ROWB = 128;               // bytes of one K block row
constexpr uint32_t TMEM_COLS = 256;          // 2 accumulator buffers x up to 128 columns
constexpr int MAX_STAGES = 8;

struct Cand {
  float v;
  int i;
};

__device__ __forceinline__ void cand_insert(Cand (&top)[4], float v, int j) {
  // sorted ascending; strict comparisons keep the earlier (lower) index first
  if (v < top[3].v) {
    if (v < top[2].v) {
      top[3] = top[2];
      if (v < top[1].v) {
        top[2] = top[1];
        if (v < top[0].v) {
          top[1] = top[0];
          top[0] = Cand{v, j};
        } else {
          top[1] = Cand{v, j};
        }
      } else {
        top[2] = Cand{v, j};
      }
    } else {
      top[3] = Cand{v, j};
    }
  }
}

template <int FP8>
__device__ __forceinline__ float code_to_float(const uint8_t* p) {
  if constexpr (FP8) {
    __nv_fp8_e4m3 q;
    q.__x = *p;
    return (float)q;
  } else {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  }
}

template <int FP8>
__global__ void __launch_bounds__(NTHREADS, 1)
assign_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC,
                 const TcParams P) {
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int KBE = ROWB / ESZ;  // elements per 128-byte K block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t a_full[2], a_empty[2], b_full[MAX_STAGES], b_empty[MAX_STAGES], acc_full[2], acc_empty[2];
  __shared__ uint64_t drain_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ unsigned int changed_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = P.nkb, BN = P.bn, stages = P.stages, nchunks = P.nchunks;
  const uint32_t a_bytes = (uint32_t)nkb * BM * ROWB;        // one A buffer
  const uint32_t b_kblk = (uint32_t)BN * ROWB;               // one K block of a B stage
  const uint32_t b_bytes = (uint32_t)nkb * b_kblk;           // one B stage
  uint8_t* A0 = smem;
  uint8_t* B0 = smem + 2 * a_bytes;
  const int64_t ntiles = (P.n + BM - 1) / BM;
  Ctl* ctl = P.ctl;

  if (threadIdx.x == 0) {
    abort_s = 0;
    changed_s = 0;
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1 + 4);  // MMA commit + the 4 epilogue warps (seed reads)
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    for (int s = 0; s < stages; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(&drain_bar, 1);
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tensormap(&mapX);
    prefetch_tensormap(&mapC);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_s, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem_base = tmem_base_s;
  const bool stopped = ctl->done != 0;  // the run's stop rule fired: no work, but keep TMEM balanced

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0 && !stopped) {
      int lt = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const int ab = lt & 1;
        if (!mbar_wait(&a_empty[ab], ((lt >> 1) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
        mbar_arrive_expect_tx(&a_full[ab], a_bytes);
        for (int kb = 0; kb < nkb; ++kb)
          tma_load_2d(A0 + ab * a_bytes + kb * (BM * ROWB), &mapX, &a_full[ab], kb * KBE, (int)(tile * BM));
        for (int c = 0; c < nchunks; ++c) {
          const int g = lt * nchunks + c, s = g % stages;
          if (!mbar_wait(&b_empty[s], ((g / stages) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          mbar_arrive_expect_tx(&b_full[s], b_bytes);
          for (int kb = 0; kb < nkb; ++kb)
            tma_load_2d(B0 + s * b_bytes + kb * b_kblk, &mapC, &b_full[s], kb * KBE, c * BN);
        }
      }
      if (!ok) {
        abort_s = 1;
        atomicExch(&ctl->error, (int)KM_ETIMEOUT);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0 && !stopped) {
      int lt = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const int ab = lt & 1;
        if (!mbar_wait(&a_full[ab], (lt >> 1) & 1, &abort_s, P.wait_ns)) { ok = false; break; }
        tc_fence_after_sync();
        const uint32_t a_addr = smem_u32(A0 + ab * a_bytes);
        for (int c = 0; c < nchunks; ++c) {
          const int g = lt * nchunks + c, s = g % stages, buf = g & 1;
          if (!mbar_wait(&b_full[s], (g / stages) & 1, &abort_s, P.wait_ns)) { ok = false; break; }
          if (!mbar_wait(&acc_empty[buf], ((g >> 1) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          tc_fence_after_sync();
          const uint32_t b_addr = smem_u32(B0 + s * b_bytes);
          const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 128);
          for (int kb = 0; kb < nkb; ++kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sdesc_k_sw128(a_addr + kb * (BM * ROWB) + kk * 32);
              const uint64_t bd = sdesc_k_sw128(b_addr + kb * b_kblk + kk * 32);
              if constexpr (FP8) mma_fp8(d_tmem, ad, bd, P.idesc, (kb | kk) != 0);
              else mma_bf16(d_tmem, ad, bd, P.idesc, (kb | kk) != 0);
            }
          }
          mma_commit(&b_empty[s]);
          mma_commit(&acc_full[buf]);
        }
        if (ok) mma_commit(&a_empty[ab]);
      }
      if (!ok) {
        abort_s = 1;
        atomicExch(&ctl->error, (int)KM_ETIMEOUT);
      }
      // every MMA this thread issued has completed once drain_bar flips
      mma_commit(&drain_bar);
      int dummy = 0;
      mbar_wait(&drain_bar, 0, &dummy, P.wait_ns);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;
    const float H = __uint_as_float(ctl->hmax_bits);
    const float Cmax = __uint_as_float(ctl->cmax_bits);
    const float QCmax = __uint_as_float(ctl->qcmax_bits);
    const float DCmax = __uint_as_float(ctl->dcmax_bits);
    unsigned int changed = 0;
    int lt = 0;
    bool ok = !stopped;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
      const int ab = lt & 1;
      const int64_t i = tile * BM + r;
      const bool valid = i < P.n;
      float4 xs = make_float4(0.f, 0.f, 0.f, 0.f);
      int old = -1;
      if (valid) {
        xs = P.xs[i];
        if (!P.first) {
          old = P.assign[i];
          if (old < 0 || old >= P.k) old = -1;  // not a label: no seed
        }
      }
      // per-row error bound and margin
      const float E = fmaf(3.f * kU, H,
                           fmaf(P.gam_tc + 2.f * kU, xs.y * QCmax,
                                fmaf(xs.z, Cmax, fmaf(xs.w, DCmax, xs.z * DCmax))));
      const float margin = 2.f * E * (1.f + 0x1p-10f);
      float thr = INFINITY;
      if (!__all_sync(0xffffffffu, mbar_wait(&a_full[ab], (lt >> 1) & 1, &abort_s, P.wait_ns))) { ok = false; break; }
      if (old >= 0) {
        // seed: score of the previous centroid from the same codes, in FP32 SIMT
        const uint8_t* arow = A0 + ab * a_bytes + r * ROWB;
        const uint8_t* crow = P.Cq + (size_t)old * P.Kp * ESZ;
        float dot = 0.f;
        for (int kb = 0; kb < nkb; ++kb) {
          const uint8_t* ab_row = arow + kb * (BM * ROWB);
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {  // 16-byte chunks, stored at chunk ^ (row & 7)
            const uint4 av = *reinterpret_cast<const uint4*>(ab_row + ((ch ^ (r & 7)) << 4));
            const uint4 cv = __ldg(reinterpret_cast<const uint4*>(crow + kb * ROWB + ch * 16));
            const uint8_t* ap = reinterpret_cast<const uint8_t*>(&av);
            const uint8_t* cp = reinterpret_cast<const uint8_t*>(&cv);
#pragma unroll
            for (int e = 0; e < 16 / ESZ; ++e) dot = fmaf(code_to_float<FP8>(ap + e * ESZ), code_to_float<FP8>(cp + e * ESZ), dot);
          }
        }
        const float2 hs = __ldg(P.hsc + old);
        const float w = FP8 ? xs.x * hs.y : 1.f;
        const float s_seed = __fsub_rn(hs.x, w * dot);
        const float Eseed = fmaf(P.gam_tc + P.gam_simt, xs.y * QCmax, 2.f * kU * (H + 2.f * xs.y * QCmax));
        thr = __fadd_ru(__fadd_ru(s_seed, Eseed * (1.f + 0x1p-10f)), margin);
        if (!(thr == thr)) thr = INFINITY;  // NaN seed: scan everything
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&a_empty[ab]);  // this warp is done reading the A tile

      Cand top[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) top[t] = Cand{INFINITY, -1};
      const float nsx = FP8 ? -xs.x : -1.f;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int g = lt * nchunks + c, buf = g & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (g >> 1) & 1, &abort_s, P.wait_ns))) { ok = false; break; }
        tc_fence_after_sync();
        for (int sub = 0; sub < BN / 32; ++sub) {
          uint32_t v[32];
          tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 128 + sub * 32), v);
          tmem_ld_wait();
          const int j0 = c * BN + sub * 32;
          const float4* h4 = reinterpret_cast<const float4*>(P.hsc + j0);
          float s[32];
          float m = INFINITY;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const float4 hh = __ldg(h4 + t);  // (h, sc) of columns 2t, 2t+1
            if constexpr (FP8) {
              s[2 * t] = fmaf(nsx * hh.y, __uint_as_float(v[2 * t]), hh.x);
              s[2 * t + 1] = fmaf(nsx * hh.w, __uint_as_float(v[2 * t + 1]), hh.z);
            } else {
              s[2 * t] = __fsub_rn(hh.x, __uint_as_float(v[2 * t]));
              s[2 * t + 1] = __fsub_rn(hh.z, __uint_as_float(v[2 * t + 1]));
            }
            m = fminf(m, fminf(s[2 * t], s[2 * t + 1]));
          }
          if (__any_sync(0xffffffffu, m <= thr)) {
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              if (s[t] <= thr) {
                cand_insert(top, s[t], j0 + t);
                thr = fminf(thr, __fadd_ru(top[0].v, margin));
              }
            }
          }
        }
        tc_fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      if (valid) {
        int nc = -1;  // -1: final; 0: all k; >0: candidate count
        int cands[4];
        if (top[0].i < 0) {
          nc = 0;
        } else {
          int cnt = 1;
          cands[0] = top[0].i;
#pragma unroll
          for (int t = 1; t < 4; ++t)
            if (top[t].i >= 0 && __fsub_rn(top[t].v, top[0].v) <= margin) cands[cnt++] = top[t].i;
          if (cnt == 4) nc = 0;         // maybe more than 4 within the margin
          else if (cnt > 1) nc = cnt;
        }
        if (nc < 0) {
          P.assign[i] = top[0].i;
          changed += (old != top[0].i);
        } else {
          FlagRec rec;
          rec.i = (int32_t)i;
          rec.old = old;
          rec.nc = nc;
          rec.pad = 0;
          for (int t = 0; t < 4; ++t) rec.cand[t] = 0;
          if (nc > 0) {
            // increasing index order: the re-check breaks exact ties toward the lowest index
            for (int a = 0; a < nc; ++a) {
              int mn = a;
              for (int b = a + 1; b < nc; ++b)
                if (cands[b] < cands[mn]) mn = b;
              const int tmp = cands[a];
              cands[a] = cands[mn];
              cands[mn] = tmp;
              rec.cand[a] = cands[a];
            }
          }
          const unsigned long long slot = atomicAdd(&ctl->n_flagged, 1ull);
          P.flags[slot] = rec;
          if (nc == 0) atomicAdd(&ctl->n_full, 1ull);
          P.assign[i] = top[0].i >= 0 ? top[0].i : 0;
        }
      }
    }
    if (!ok && !stopped) {
      abort_s = 1;
      atomicExch(&ctl->error, (int)KM_ETIMEOUT);
    }
    if (changed) atomicAdd(&changed_s, changed);
  }

  tc_fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after_sync();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  if (threadIdx.x == 0 && changed_s) atomicAdd(&ctl->n_changed, (unsigned long long)changed_s);
}

}  // namespace

size_t tc_smem_bytes(int nkb, int bn, int stages) {
  return 1024 + 2 * (size_t)nkb * BM * ROWB + (size_t)stages * nkb * bn * ROWB;
}

// Raises the dynamic shared-memory limit of both instantiations to the
// device's opt-in maximum minus the kernel's static shared memory.
cudaError_t init_assign_tc() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, assign_tc_kernel<0>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(assign_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, assign_tc_kernel<1>);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(assign_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  return e;
}

cudaError_t launch_assign_tc(const Problem& p, const TcLaunch& L, const TcParams& P, cudaStream_t s) {
  const int64_t tiles = (p.n + BM - 1) / BM;
  const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
  const size_t smem = tc_smem_bytes(P.nkb, P.bn, P.stages);
  if (L.fp8)
    assign_tc_kernel<1><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, P);
  else
    assign_tc_kernel<0><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, P);
  return cudaGetLastError();
}

}  // namespace km
