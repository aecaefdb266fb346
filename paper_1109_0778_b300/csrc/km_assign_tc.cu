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
// Roles (320 threads): warp 0 = TMA producer, warp 1 = MMA issuer and TMEM
// owner, warps 2-9 = epilogue (two per TMEM lane quarter, each taking half of
// every chunk's columns; the two candidate lists of a row are merged through
// shared memory at the end of the tile). h_j (and the FP8 scales) are staged in
// shared memory once per CTA. Every mbarrier wait is bounded in time; on
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
// candidates (or, past 7 of them, all k) go to the FP32 re-check.
//
// Threshold. Rows keep the 8 smallest scores seen among elements <= thr, with
// thr = min(thr0, best + margin) rounded up. From the second step on thr0 is
// the score of the point's previous centroid, recomputed from the same codes
// in FP32 SIMT (plus its bound against the tensor-core sum and the margin), so
// a 32-column chunk costs one minimum unless it holds a candidate. From the
// second step of a call on, rows are the points in the previous step's
// cluster-sorted order (the codes are rewritten in that order by the reduce
// stage), so the 32 rows of a warp share their previous centroid and the
// candidate branch is taken in about one chunk per warp.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"
#include "km_tc.cuh"

#include <cstring>

namespace km {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int NEPI = 8;                      // epilogue warps: two per TMEM lane quarter
constexpr int NTHREADS = 64 + 32 * NEPI;
constexpr uint32_t ROWB = 128;               // bytes of one K block row
constexpr uint32_t TMEM_COLS = 512;          // 4 accumulator buffers x up to 128 columns
constexpr int NACC = 4;
constexpr int MAX_STAGES = 8;

constexpr int kT = kMaxCand;  // candidate slots per row

struct Cand {
  float v;
  int i;
};

// Sorted insert into the row's candidate list (ascending score; strict
// comparisons keep the earlier, lower index first among equal scores).
__device__ __forceinline__ void cand_insert(Cand (&top)[kT], float v, int j) {
  if (!(v < top[kT - 1].v)) return;
#pragma unroll
  for (int t = kT - 1; t > 0; --t) {
    if (v < top[t - 1].v) {
      top[t] = top[t - 1];
    } else {
      top[t] = Cand{v, j};
      return;
    }
  }
  top[0] = Cand{v, j};
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
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

// Per-tile parameters: one instance (single launches) or the instance that
// owns flattened tile gt (batched launches).
struct Item {
  int b;
  bool skip;        // the instance's stop rule fired
  int64_t tile;     // tile index within the instance
  int64_t n;
  int k, Kp, nkb, nchunks;
  const CUtensorMap* mapX;
  const CUtensorMap* mapC;
  const float* h;
  const float* sc;
  const int32_t* rows;
  const float4* xs;
  const float4* xs_sorted;
  const int32_t* lab_sorted;
  const uint8_t* Cq;
  int32_t* assign;
  Ctl* ctl;
  float gam_tc, gam_simt;
};

template <bool BATCH>
__device__ __forceinline__ Item get_item(const TcParams& P, const CUtensorMap* mx, const CUtensorMap* mc,
                                         int64_t gt) {
  Item it;
  if constexpr (!BATCH) {
    it.b = 0;
    it.tile = gt;
    it.n = P.n;
    it.k = P.k;
    it.Kp = P.Kp;
    it.nkb = P.nkb;
    it.nchunks = P.nchunks;
    it.mapX = mx;
    it.mapC = mc;
    it.h = P.h;
    it.sc = P.sc;
    it.rows = P.rows;
    it.xs = P.xs;
    it.xs_sorted = P.xs_sorted;
    it.lab_sorted = P.lab_sorted;
    it.Cq = P.Cq;
    it.assign = P.assign;
    it.ctl = P.ctl;
    it.gam_tc = P.gam_tc;
    it.gam_simt = P.gam_simt;
  } else {
    const int b = find_block(P.btile_off, P.nb, gt);
    const BInst& I = P.binst[b];
    it.b = b;
    it.tile = gt - I.tile_off;
    it.n = I.n;
    it.k = I.k;
    it.Kp = I.Kp;
    it.nkb = I.nkb;
    it.nchunks = I.nchunks;
    it.mapX = P.bmaps + 2 * b;
    it.mapC = P.bmaps + 2 * b + 1;
    it.h = P.bh + I.kp_off;
    it.sc = P.bsc + I.kp_off;
    it.rows = P.sorted ? P.bperm + I.row_off : nullptr;
    it.xs = P.bxs + I.row_off;
    it.xs_sorted = P.bxs_sorted + I.row_off;
    it.lab_sorted = P.blab_sorted + I.row_off;
    it.Cq = P.bCq + I.cq_off;
    it.assign = I.assign;
    it.ctl = P.bctls + b;
    it.gam_tc = I.gam_tc;
    it.gam_simt = I.gam_simt;
  }
  it.skip = it.ctl->done != 0;
  return it;
}

// A wait that ran out: the error goes to every control block of the launch, so
// that no later stage consumes the labels this step did not write.
template <bool BATCH>
__device__ void record_timeout(const TcParams& P) {
  if constexpr (BATCH) {
    for (int b = 0; b < P.nb; ++b) atomicExch(&P.bctls[b].error, (int)KM_ETIMEOUT);
  } else {
    atomicExch(&P.ctl->error, (int)KM_ETIMEOUT);
  }
}

template <int FP8, bool BATCH>
__global__ void __launch_bounds__(NTHREADS, 1)
assign_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC,
                 const TcParams P) {
  constexpr int ESZ = FP8 ? 1 : 2;
  constexpr int KBE = ROWB / ESZ;  // elements per 128-byte K block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t a_full[2], a_empty[2], b_full[MAX_STAGES], b_empty[MAX_STAGES], acc_full[NACC], acc_empty[NACC];
  __shared__ uint64_t drain_bar, never_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, halt_s;

  // an earlier launch of this step timed out: nothing to do (read once per CTA,
  // so that every role of the CTA takes the same decision)
  if (threadIdx.x == 0) halt_s = P.ctl->error != 0;
  __syncthreads();
  if (halt_s) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // buffer sizes follow the launch maxima (P.nkb, P.nchunks); a tile uses its own nkb, nchunks
  const int BN = P.bn, stages = P.stages;
  const uint32_t a_bytes = (uint32_t)P.nkb * BM * ROWB;      // one A buffer
  const uint32_t b_kblk = (uint32_t)BN * ROWB;               // one K block of a B stage
  const uint32_t b_bytes = (uint32_t)P.nkb * b_kblk;         // one B stage
  uint8_t* A0 = smem;
  const int nab = P.abufs;                                    // A buffers: 2 (double) or 1
  uint8_t* B0 = smem + nab * a_bytes;
  const int kpmax = P.nchunks * BN;
  float* Hs = reinterpret_cast<float*>(B0 + (size_t)stages * b_bytes);  // [kpmax]
  float* SCs = Hs + kpmax;                                               // [kpmax] (FP8)
  Cand* Ms = reinterpret_cast<Cand*>(SCs + (FP8 ? kpmax : 0));           // [BM][kT] merge buffer
  const int64_t ntiles = BATCH ? P.ntiles : (P.n + BM - 1) / BM;

  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1 + NEPI);  // MMA commit + the epilogue warps (seed reads)
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], NEPI);
    }
    for (int s = 0; s < stages; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(&drain_bar, 1);
    mbar_init(&never_bar, 1);  // nothing ever arrives: the timeout test waits on it
    fence_mbar_init();
  }
  if (!BATCH && warp == 0 && lane == 0) {
    prefetch_tensormap(&mapX);
    prefetch_tensormap(&mapC);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_s, TMEM_COLS);
    tmem_relinquish();
  }
  if (!BATCH && warp >= 2) {  // batched launches stage h per instance in the epilogue
    for (int j = threadIdx.x - 64; j < kpmax; j += 32 * NEPI) {
      Hs[j] = __ldg(P.h + j);
      if (FP8) SCs[j] = __ldg(P.sc + j);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem_base = tmem_base_s;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int lt = 0, gc = 0, cur_b = -1;  // tiles and chunks issued so far by this CTA
      int last_a = -1, last_s = -1;    // barrier slots of the most recent A and B loads
      uint32_t last_aph = 0, last_sph = 0;
      bool ok = true;
      for (int64_t gt = blockIdx.x; gt < ntiles && ok; gt += gridDim.x) {
        const Item it = get_item<BATCH>(P, &mapX, &mapC, gt);
        if (it.skip) continue;
        if (BATCH && it.b != cur_b) {
          // tensor maps in global memory: order the host's writes before the async proxy reads them
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(it.mapX) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(it.mapC) : "memory");
          cur_b = it.b;
        }
        const int ab = lt % nab;
        if (!mbar_wait(&a_empty[ab], ((lt / nab) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
        mbar_arrive_expect_tx(&a_full[ab], (uint32_t)it.nkb * BM * ROWB);
        for (int kb = 0; kb < it.nkb; ++kb)
          tma_load_2d(A0 + ab * a_bytes + kb * (BM * ROWB), it.mapX, &a_full[ab], kb * KBE, (int)(it.tile * BM));
        last_a = ab;
        last_aph = (lt / nab) & 1;
        for (int c = 0; c < it.nchunks; ++c, ++gc) {
          const int s = gc % stages;
          if (!mbar_wait(&b_empty[s], ((gc / stages) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          mbar_arrive_expect_tx(&b_full[s], (uint32_t)it.nkb * b_kblk);
          for (int kb = 0; kb < it.nkb; ++kb)
            tma_load_2d(B0 + s * b_bytes + kb * b_kblk, it.mapC, &b_full[s], kb * KBE, c * BN);
          last_s = s;
          last_sph = (gc / stages) & 1;
        }
        ++lt;
      }
      if (!ok) {
        abort_s = 1;
        record_timeout<BATCH>(P);
        // let the last loads land before the CTA can exit (bounded)
        int no_abort = 0;
        if (last_a >= 0) mbar_wait(&a_full[last_a], last_aph, &no_abort, 10000000ull);
        if (last_s >= 0) mbar_wait(&b_full[last_s], last_sph, &no_abort, 10000000ull);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int lt = 0, gc = 0;
      bool ok = true, issued = false;
      for (int64_t gt = blockIdx.x; gt < ntiles && ok; gt += gridDim.x) {
        const Item it = get_item<BATCH>(P, &mapX, &mapC, gt);
        if (it.skip) continue;
        const int ab = lt % nab;
        if (!mbar_wait(&a_full[ab], (lt / nab) & 1, &abort_s, P.wait_ns)) { ok = false; break; }
        tc_fence_after_sync();
        const uint32_t a_addr = smem_u32(A0 + ab * a_bytes);
        for (int c = 0; c < it.nchunks; ++c, ++gc) {
          const int s = gc % stages, buf = gc % NACC;
          if (!mbar_wait(&b_full[s], (gc / stages) & 1, &abort_s, P.wait_ns)) { ok = false; break; }
          if (!mbar_wait(&acc_empty[buf], ((gc / NACC) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          tc_fence_after_sync();
          const uint32_t b_addr = smem_u32(B0 + s * b_bytes);
          const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 128);
          for (int kb = 0; kb < it.nkb; ++kb) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sdesc_k_sw128(a_addr + kb * (BM * ROWB) + kk * 32);
              const uint64_t bd = sdesc_k_sw128(b_addr + kb * b_kblk + kk * 32);
              if constexpr (FP8) mma_fp8(d_tmem, ad, bd, P.idesc, (kb | kk) != 0);
              else mma_bf16(d_tmem, ad, bd, P.idesc, (kb | kk) != 0);
            }
          }
          issued = true;
          mma_commit(&b_empty[s]);
          mma_commit(&acc_full[buf]);
        }
        if (ok) mma_commit(&a_empty[ab]);
        ++lt;
      }
      if (!ok) {
        abort_s = 1;
        record_timeout<BATCH>(P);
      }
      if (issued) {  // every MMA this thread issued has completed once drain_bar flips
        mma_commit(&drain_bar);
        int dummy = 0;
        mbar_wait(&drain_bar, 0, &dummy, P.wait_ns);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..9)
    const int q = warp & 3;            // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;  // which half of each chunk's columns
    const int r = q * 32 + lane;
    const int nsub = BN / 64;          // 32-column sub-chunks per half
    int lt = 0, gc = 0, cur_b = -1;
    bool ok = true;
    unsigned int changed = 0;
    // Every epilogue warp runs every tile to the end, even after a timeout (then
    // skipping waits and work), so that all of them reach the named barriers of
    // the candidate merge the same number of times.
    for (int64_t gt = blockIdx.x; gt < ntiles; gt += gridDim.x) {
      const Item it = get_item<BATCH>(P, &mapX, &mapC, gt);
      if (it.skip) continue;
      if (BATCH && it.b != cur_b) {
        // this instance's h_j (and scales) into shared memory
        asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
        if (cur_b >= 0 && changed) {
          atomicAdd(&P.bctls[cur_b].n_changed, (unsigned long long)changed);
          changed = 0;
        }
        for (int j = threadIdx.x - 64; j < it.nchunks * BN; j += 32 * NEPI) {
          Hs[j] = __ldg(it.h + j);
          if (FP8) SCs[j] = __ldg(it.sc + j);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
        cur_b = it.b;
      }
      const Ctl* ctl = it.ctl;
      const float H = __uint_as_float(ctl->hmax_bits);
      const float Cmax = __uint_as_float(ctl->cmax_bits);
      const float QCmax = __uint_as_float(ctl->qcmax_bits);
      const float DCmax = __uint_as_float(ctl->dcmax_bits);
      const int ab = lt % nab;
      const int64_t prow = it.tile * BM + r;  // row of the code matrix
      const bool valid = prow < it.n;
      int64_t i = 0;                          // point of this row
      float4 xs = make_float4(0.f, 0.f, 0.f, 0.f);
      int old = -1;
      if (valid) {
        if (it.rows) {  // cluster-sorted order: contiguous metadata written by the reduce stage
          i = it.rows[prow];
          xs = it.xs_sorted[prow];
          if (!P.first) old = it.lab_sorted[prow];
        } else {
          i = prow;
          xs = it.xs[prow];
          if (!P.first) old = it.assign[prow];
        }
      }
      if (old < 0 || old >= it.k) old = -1;  // not a label: no seed
      // per-row error bound and margin
      const float E = fmaf(3.f * kU, H,
                           fmaf(it.gam_tc + 2.f * kU, xs.y * QCmax,
                                fmaf(xs.z, Cmax, fmaf(xs.w, DCmax, xs.z * DCmax))));
      const float margin = 2.f * E * (1.f + 0x1p-10f);
      float thr = INFINITY;
      if (ok && !__all_sync(0xffffffffu, mbar_wait(&a_full[ab], (lt / nab) & 1, &abort_s, P.wait_ns))) ok = false;
      if (ok && P.debug_stall && !__all_sync(0xffffffffu, mbar_wait(&never_bar, 0, &abort_s, P.wait_ns))) ok = false;
      if (ok && old >= 0) {
        // seed: score of the previous centroid from the same codes, in FP32 SIMT
        const uint8_t* arow = A0 + ab * a_bytes + r * ROWB;
        const uint8_t* crow = it.Cq + (size_t)old * it.Kp * ESZ;
        float dot = 0.f;
        for (int kb = 0; kb < it.nkb; ++kb) {
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
        const float w = FP8 ? xs.x * SCs[old] : 1.f;
        const float s_seed = __fsub_rn(Hs[old], w * dot);
        const float Eseed = fmaf(it.gam_tc + it.gam_simt, xs.y * QCmax, 2.f * kU * (H + 2.f * xs.y * QCmax));
        thr = __fadd_ru(__fadd_ru(s_seed, Eseed * (1.f + 0x1p-10f)), margin);
        if (!(thr == thr)) thr = INFINITY;  // NaN seed: scan everything
      }
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&a_empty[ab]);  // this warp is done reading the A tile

      Cand top[kT];
#pragma unroll
      for (int t = 0; t < kT; ++t) top[t] = Cand{INFINITY, -1};
      const float nsx = -xs.x;
      for (int c = 0; c < it.nchunks; ++c, ++gc) {
        if (!ok) continue;
        const int buf = gc % NACC;
        if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (gc / NACC) & 1, &abort_s, P.wait_ns))) {
          ok = false;
          continue;
        }
        tc_fence_after_sync();
        const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 128 + half * (BN / 2));
        uint32_t v[32];
        tmem_ld_32x32b_x32(tbase, v);
        for (int sub = 0; sub < nsub; ++sub) {
          tmem_ld_wait();
          const int j0 = c * BN + half * (BN / 2) + sub * 32;
          // scores s_j = h_j - (sx sc_j) acc_j, two columns per packed operation
          float s[32];
          const float4* h4 = reinterpret_cast<const float4*>(Hs + j0);
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float4 hh = h4[t];
            float2 a0 = make_float2(__uint_as_float(v[4 * t]), __uint_as_float(v[4 * t + 1]));
            float2 a1 = make_float2(__uint_as_float(v[4 * t + 2]), __uint_as_float(v[4 * t + 3]));
            float2 w0, w1;
            if constexpr (FP8) {
              const float4 sc4 = reinterpret_cast<const float4*>(SCs + j0)[t];
              w0 = __fmul2_rn(make_float2(nsx, nsx), make_float2(sc4.x, sc4.y));
              w1 = __fmul2_rn(make_float2(nsx, nsx), make_float2(sc4.z, sc4.w));
            } else {
              w0 = make_float2(-1.f, -1.f);
              w1 = w0;
            }
            const float2 s0 = __ffma2_rn(w0, a0, make_float2(hh.x, hh.y));
            const float2 s1 = __ffma2_rn(w1, a1, make_float2(hh.z, hh.w));
            s[4 * t] = s0.x;
            s[4 * t + 1] = s0.y;
            s[4 * t + 2] = s1.x;
            s[4 * t + 3] = s1.y;
          }
          if (sub + 1 < nsub) tmem_ld_32x32b_x32(tbase + (uint32_t)((sub + 1) * 32), v);  // next sub-chunk in flight
          float m = INFINITY;
#pragma unroll
          for (int t = 0; t < 32; t += 2) m = min3f(m, s[t], s[t + 1]);
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
      // merge the second half's list into the first half's (named barrier of the epilogue warps)
      if (half == 1) {
#pragma unroll
        for (int t = 0; t < kT; ++t) Ms[r * kT + t] = top[t];
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (half == 0) {
#pragma unroll
        for (int t = 0; t < kT; ++t) {
          const Cand o = Ms[r * kT + t];
          if (o.i >= 0) cand_insert(top, o.v, o.i);
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
      if (ok && valid && half == 0) {
        int nc = -1;  // -1: final; 0: all k; >0: candidate count
        int cands[kT];
        if (top[0].i < 0) {
          nc = 0;
        } else {
          int cnt = 1;
          cands[0] = top[0].i;
#pragma unroll
          for (int t = 1; t < kT; ++t)
            if (top[t].i >= 0 && __fsub_rn(top[t].v, top[0].v) <= margin) cands[cnt++] = top[t].i;
          if (cnt == kT) nc = 0;        // maybe more than kT within the margin
          else if (cnt > 1) nc = cnt;
        }
        if (nc < 0) {
          it.assign[i] = top[0].i;
          changed += (old != top[0].i);
        } else {
          FlagRec rec;
          rec.i = (int32_t)i;
          rec.old = old;
          rec.nc = nc;
          rec.pad = it.b;
#pragma unroll
          for (int t = 0; t < kT; ++t) rec.cand[t] = 0;
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
          const unsigned long long slot = atomicAdd(P.flag_slots, 1ull);
          if (slot < (unsigned long long)P.flag_cap) P.flags[slot] = rec;
          if (BATCH) atomicAdd(&it.ctl->n_flagged, 1ull);
          if (nc == 0) atomicAdd(&it.ctl->n_full, 1ull);
          it.assign[i] = top[0].i >= 0 ? top[0].i : 0;
        }
      }
      ++lt;
    }
    if (!ok) {
      abort_s = 1;
      record_timeout<BATCH>(P);
    }
    if (changed) {
      Ctl* cc = BATCH ? (cur_b >= 0 ? P.bctls + cur_b : nullptr) : P.ctl;
      if (cc) atomicAdd(&cc->n_changed, (unsigned long long)changed);
    }
  }

  tc_fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after_sync();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace

size_t tc_smem_bytes(int nkb, int bn, int stages, int kp, int fp8, int abufs) {
  return 1024 + (size_t)abufs * nkb * BM * ROWB + (size_t)stages * nkb * bn * ROWB + (size_t)kp * 4 * (fp8 ? 2 : 1) +
         (size_t)BM * kT * sizeof(Cand);
}

// Raises the dynamic shared-memory limit of both instantiations to the
// device's opt-in maximum minus the kernel's static shared memory.
template <typename K>
cudaError_t raise_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  return e;
}

cudaError_t init_assign_tc() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<0, false>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<1, false>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<0, true>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<1, true>, optin);
  return e;
}

cudaError_t launch_assign_tc(const Problem& p, const TcLaunch& L, const TcParams& P, cudaStream_t s) {
  const int64_t tiles = (p.n + BM - 1) / BM;
  const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
  const size_t smem = tc_smem_bytes(P.nkb, P.bn, P.stages, P.nchunks * P.bn, L.fp8, P.abufs);
  if (L.fp8)
    assign_tc_kernel<1, false><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, P);
  else
    assign_tc_kernel<0, false><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, P);
  return cudaGetLastError();
}

// One launch over the flattened tiles of every instance of a batch (BF16 or
// E4M3, d <= 128 so nkb <= 2, chunk width bn = 64 or 128).
cudaError_t launch_b_assign(const BWork& W, int fp8, int first, int sorted, int nkb_max, int kp_max, int bn,
                            int stages, int abufs, uint32_t idesc, cudaStream_t s) {
  TcParams P;
  memset(&P, 0, sizeof P);
  P.nkb = nkb_max;
  P.bn = bn;
  P.nchunks = kp_max / bn;
  P.stages = stages;
  P.abufs = abufs;
  P.first = first;
  P.idesc = idesc;
  P.wait_ns = 2000000000ull;
  P.ctl = W.ctls;  // timeouts are reported in the first instance's control block
  P.flags = W.flags;
  P.flag_slots = W.flag_slots;
  P.flag_cap = W.R;
  P.binst = W.inst;
  P.btile_off = W.tile_off;
  P.nb = W.nb;
  P.sorted = sorted;
  P.ntiles = W.T;
  P.bctls = W.ctls;
  P.bmaps = W.maps;
  P.bh = W.hq;
  P.bsc = W.scq;
  P.bCq = W.Cq;
  P.bxs = W.xs;
  P.bxs_sorted = W.xs_sorted;
  P.blab_sorted = W.lab_sorted;
  P.bperm = W.perm;
  const int grid = (int)(W.T < num_sms() ? W.T : num_sms());
  const size_t smem = tc_smem_bytes(nkb_max, bn, stages, kp_max, fp8, abufs);
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof dummy);
  if (fp8) assign_tc_kernel<1, true><<<grid, NTHREADS, smem, s>>>(dummy, dummy, P);
  else assign_tc_kernel<0, true><<<grid, NTHREADS, smem, s>>>(dummy, dummy, P);
  return cudaGetLastError();
}

}  // namespace km
