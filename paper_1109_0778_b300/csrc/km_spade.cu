// SPADE density downsampling (Sec. 4.1, "Downsampling in Bioinformatics").
//
// The paper's loop visits the rows in order and evaluates a row only while its
// density is still 0: one fused pass over the row's L1 distances finds the rows
// within apprx_width and counts the rows within kernel_width, and the found
// rows take the count as their density (so they are skipped later). The
// evaluated rows form the greedy set P: row i is in P exactly when no earlier
// row of P lies within apprx_width of it.
//
// Here the rows are evaluated in batches of up to kSB candidates, the first
// kSB rows (from a cursor) that no evaluated row has found yet:
//   select   one block collects the candidates in index order;
//   pairs    a tile pass computes every candidate's distances to all n rows:
//            its count, the rows it finds (a list), and which earlier
//            candidates of the batch it finds (a bit matrix);
//   resolve  one block settles, in index order, which candidates the loop
//            evaluates: a candidate found by an evaluated earlier candidate of
//            the batch is skipped (its row was computed speculatively);
//   apply    every row found by an evaluated candidate records it as a writer:
//            the highest (policy 0, the generated code's overwriting bulk
//            update) or lowest (policy 1, the C++ snippet's fill-if-zero)
//            index; when the list overflowed, a second tile pass over the
//            evaluated candidates records the writers directly;
//   finish   counts and flags of the evaluated rows, cursor bookkeeping.
// At the end a row's density is the count of its writer.
//
// Distances. The FP32 sum D^ of |x_t - y_t| (d terms, each difference rounded
// once) satisfies |D^ - D| <= gamma_d D for the exact D (u = 2^-24), and the
// loop's FP64 distance D64 (columns in order) satisfies |D64 - D| <= g64 D.
// So D64 < w is certain when D^ < w (1 - gamma)/(1 + g64) and impossible when
// D^ > w (1 + gamma)/(1 - g64); in between the pair is re-evaluated in FP64
// exactly as the loop does (same operations, same order), so every decision
// equals the FP64 loop's.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "km_gather.cuh"
#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kTile = 128;   // candidates x rows per tile
constexpr int kKC = 32;      // feature columns per shared-memory stage
constexpr int kPad = 36;     // floats per staged row (16-byte aligned, spreads banks)
constexpr int kThreads = 256;
constexpr int kSideFloats = kTile * kPad;

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// The loop's distance: FP64, columns in increasing order.
__device__ __forceinline__ double l1_fp64(const float* __restrict__ x, const float* __restrict__ y, int d) {
  double s = 0.0;
  for (int t = 0; t < d; ++t) s += fabs((double)x[t] - (double)y[t]);
  return s;
}

__device__ __forceinline__ void cp_async16_zfill(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

// Stages columns [c0, c0 + NC) of 128 rows into side (row r at side + r * rs
// floats): row r < nrows is X row rowof(r); columns past d and rows past
// nrows are zero. 16-byte copies when every row starts on a 16-byte boundary
// (vec), else 4-byte. Issues the copies; the caller commits the group.
template <int NC, typename RowOf>
__device__ __forceinline__ void stage_cols(float* side, int rs, const float* __restrict__ X, int d, int vec, int c0,
                                           int nrows, RowOf rowof, int tid) {
  if (vec) {
#pragma unroll
    for (int m = 0; m < (kTile * NC / 4) / kThreads; ++m) {
      const int p = tid + m * kThreads, r = p / (NC / 4), c = 4 * (p % (NC / 4));
      const bool ok = r < nrows && c0 + c < d;
      const float* src = ok ? X + (int64_t)rowof(r) * d + c0 + c : X;
      cp_async16_zfill(side + r * rs + c, src, ok);
    }
  } else {
#pragma unroll 4
    for (int m = 0; m < (kTile * NC) / kThreads; ++m) {
      const int p = tid + m * kThreads, r = p / NC, c = p % NC;
      const bool ok = r < nrows && c0 + c < d;
      const float* src = ok ? X + (int64_t)rowof(r) * d + c0 + c : X;
      cp_async4_zfill(side + r * rs + c, src, ok);
    }
  }
}

// The slow path of one (candidate k, row j) pair whose FP32 distance D lies in
// a decision band or below apprx_width's: FP64 re-evaluation where the band
// requires it (nex counts them), then the found-row record (APPLY = 0: list
// entry and in-batch bit; APPLY = 1: writer, evaluated candidates only).
// Returns 1 when the pair adds to the candidate's count beyond D < w_lo.
template <int APPLY>
__device__ __noinline__ int settle_pair(const SpadeArgs& A, int k, int64_t j, float D, int& nex) {
  if (APPLY && !A.inP[k]) return 0;
  const int d = A.d;
  const int32_t ci = A.cand[k];
  int add = 0;
  double D64 = -1.0;  // FP64 distance once evaluated
  if (!APPLY && D >= A.w_lo && D <= A.w_hi) {
    D64 = l1_fp64(A.X + (int64_t)ci * d, A.X + j * d, d);
    ++nex;
    add = D64 < A.cw ? 1 : 0;
  }
  bool near = D < A.a_lo;
  if (!near && D <= A.a_hi) {
    if (D64 < 0.0) {
      D64 = l1_fp64(A.X + (int64_t)ci * d, A.X + j * d, d);
      ++nex;
    }
    near = D64 < A.apprx;
  }
  if (!near) return add;
  if (APPLY) {
    if (A.policy == 0) atomicMax(&A.q[j], ci);
    else atomicMin(&A.q[j], ci);
  } else {
    SpadeCtl* ctl = A.ctl;
    const unsigned long long at = atomicAdd(&ctl->n_pairs, 1ull);
    if (at < (unsigned long long)A.pair_cap) A.pairs[at] = make_int2(k, (int)j);
    else ctl->overflow = 1;
    const int kj = A.slot[j];
    if (kj >= 0 && kj < k) atomicOr(&A.nbr[(size_t)k * (kSB / 32) + (kj >> 5)], 1u << (kj & 31));
  }
  return add;
}

// The slow path of a thread's 8 x 8 pairs (candidates k0 + 16 a, rows j0 + 16 b):
// the pairs whose D lies at or below a_hi or in the counting band go through
// settle_pair, one at a time (D read through select trees, so acc stays in
// registers). With count_certain the certain counts (D < w_lo) are added too
// (tiles whose fast path did not count).
template <int APPLY>
__device__ __forceinline__ void slow_pairs(const SpadeArgs& A, const float (&acc)[8][8], int k0, int64_t j0, bool full,
                                           bool count_certain, int nb, int64_t n, int (&cnt)[8], int& nex) {
  uint32_t msk[2] = {0u, 0u};  // bit (a % 4) * 8 + b of word a / 4
#pragma unroll
  for (int a = 0; a < 8; ++a) {
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float D = acc[a][b];
      const bool valid = full || (k0 + 16 * a < nb && j0 + 16 * b < n);
      if (count_certain) cnt[a] += (valid && D < A.w_lo) ? 1 : 0;
      const bool sl = valid && (D <= A.a_hi || fabsf(D - A.w_mid) <= A.w_half);
      msk[a >> 2] |= (sl ? 1u : 0u) << ((a & 3) * 8 + b);
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t m = msk[h];
#pragma unroll 1
    while (m) {
      const int bit = __ffs(m) - 1;
      m &= m - 1;
      const int a = h * 4 + (bit >> 3), b = bit & 7;
      float ra[8];
#pragma unroll
      for (int aa = 0; aa < 8; ++aa) {
        const float b0 = (b & 1) ? acc[aa][1] : acc[aa][0], b1 = (b & 1) ? acc[aa][3] : acc[aa][2];
        const float b2 = (b & 1) ? acc[aa][5] : acc[aa][4], b3 = (b & 1) ? acc[aa][7] : acc[aa][6];
        const float c0 = (b & 2) ? b1 : b0, c1 = (b & 2) ? b3 : b2;
        ra[aa] = (b & 4) ? c1 : c0;
      }
      const float e0 = (a & 1) ? ra[1] : ra[0], e1 = (a & 1) ? ra[3] : ra[2];
      const float e2 = (a & 1) ? ra[5] : ra[4], e3 = (a & 1) ? ra[7] : ra[6];
      const float f0 = (a & 2) ? e1 : e0, f1 = (a & 2) ? e3 : e2;
      const float D = (a & 4) ? f1 : f0;
      const int add = settle_pair<APPLY>(A, k0 + 16 * a, j0 + 16 * b, D, nex);
#pragma unroll
      for (int aa = 0; aa < 8; ++aa) cnt[aa] += aa == a ? add : 0;
    }
  }
}

// acc[a][b] += sum over the staged columns [0, 4 nq) of |xa - yb| for candidate
// rows ty + 16 a of sa and rows tx + 16 b of sb (row stride rs floats): the
// differences two columns at a time (packed), the absolute values added in order.
__device__ __forceinline__ void accumulate_l1(float (&acc)[8][8], const float* sa, const float* sb, int rs, int nq,
                                              int tx, int ty) {
  for (int q = 0; q < nq; ++q) {
    float4 xa[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) xa[a] = *reinterpret_cast<const float4*>(sa + (ty + 16 * a) * rs + 4 * q);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const float4 yb = *reinterpret_cast<const float4*>(sb + (tx + 16 * b) * rs + 4 * q);
      const float2 ny01 = make_float2(-yb.x, -yb.y), ny23 = make_float2(-yb.z, -yb.w);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const float2 d01 = __fadd2_rn(make_float2(xa[a].x, xa[a].y), ny01);
        const float2 d23 = __fadd2_rn(make_float2(xa[a].z, xa[a].w), ny23);
        float v = acc[a][b];
        v += fabsf(d01.x);
        v += fabsf(d01.y);
        v += fabsf(d23.x);
        v += fabsf(d23.y);
        acc[a][b] = v;
      }
    }
  }
}

// Tile pass over (candidate, row) pairs. APPLY = 0: counts, found-row list and
// in-batch bits of every candidate. APPLY = 1 (only after a list overflow):
// the evaluated candidates record themselves as writers of their found rows.
template <int APPLY>
__global__ void __launch_bounds__(kThreads, 2) spade_pairs_kernel(SpadeArgs A) {
  extern __shared__ __align__(16) float sp_smem[];
  __shared__ int s_cnt[kTile];
  SpadeCtl* ctl = A.ctl;
  const int nb = ctl->nb;
  if (nb == 0 || (APPLY && !ctl->overflow)) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t n = A.n;
  const int d = A.d;
  const int nct = (nb + kTile - 1) / kTile;
  const int nrt = (int)((n + kTile - 1) / kTile);
  const int64_t ntiles = (int64_t)nct * nrt;
  const int nkc = (d + kKC - 1) / kKC;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nsteps = my_tiles * nkc;
  if (nsteps == 0) return;

  // this CTA's steps: tiles t = blockIdx.x + m gridDim.x (candidate tile ct = t / nrt, row
  // tile rt = t % nrt), each in nkc column chunks; positions advance without division
  struct Pos {
    int ct, rt, kc;
  };
  auto advance = [&](Pos& p) {
    if (++p.kc == nkc) {
      p.kc = 0;
      p.rt += gridDim.x;
      while (p.rt >= nrt) {
        p.rt -= nrt;
        ++p.ct;
      }
    }
  };
  auto stage_step = [&](const Pos& p, int buf) {
    const int c0 = p.kc * kKC;
    float* sa = sp_smem + (size_t)buf * 2 * kSideFloats;
    float* sb = sa + kSideFloats;
    const int32_t* cand = A.cand + p.ct * kTile;
    const int64_t r0 = (int64_t)p.rt * kTile;
    stage_cols<kKC>(sa, kPad, A.X, d, A.vec, c0, min(kTile, nb - p.ct * kTile), [&](int r) { return cand[r]; }, tid);
    stage_cols<kKC>(sb, kPad, A.X, d, A.vec, c0, (int)min((int64_t)kTile, n - r0), [&](int r) { return r0 + r; },
                    tid);
    cp_async_commit();
  };

  for (int r = tid; r < kTile; r += kThreads) s_cnt[r] = 0;
  int cur_ct = -1;
  float acc[8][8];
  Pos ld{(int)(blockIdx.x / nrt), (int)(blockIdx.x % nrt), 0};
  Pos cp = ld;
  stage_step(ld, 0);
  advance(ld);
  for (int64_t s = 0; s < nsteps; ++s, advance(cp)) {
    const int buf = (int)(s & 1);
    if (s + 1 < nsteps) {
      stage_step(ld, buf ^ 1);
      advance(ld);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int kc = cp.kc;
    if (kc == 0) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    }
    {
      const float* sa = sp_smem + (size_t)buf * 2 * kSideFloats;
      accumulate_l1(acc, sa, sa + kSideFloats, kPad, (min(kKC, d - kc * kKC) + 3) >> 2, tx, ty);
    }
    __syncthreads();  // the stage is consumed before it is refilled
    if (kc != nkc - 1) continue;

    // ---------------------------------------------------------------- tile epilogue
    const int ct = cp.ct;
    const int64_t rt = cp.rt;
    if (!APPLY && ct != cur_ct) {  // candidate counts accumulate while the candidate tile stays
      if (cur_ct >= 0) {
        for (int r = tid; r < kTile; r += kThreads) {
          const int k = cur_ct * kTile + r;
          if (k < nb && s_cnt[r]) atomicAdd(&A.ccount[k], s_cnt[r]);
        }
        __syncthreads();
        for (int r = tid; r < kTile; r += kThreads) s_cnt[r] = 0;
        __syncthreads();
      }
      cur_ct = ct;
    }
    // certain counts (D < w_lo); pairs at or below a_hi or in the counting band take the slow path
    int cnt[8];
    bool slow = false;
    const bool full = (ct + 1) * kTile <= nb && (rt + 1) * kTile <= n;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      cnt[a] = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const float D = acc[a][b];
        const bool valid = full || (ct * kTile + ty + 16 * a < nb && rt * kTile + tx + 16 * b < n);
        cnt[a] += (valid && D < A.w_lo) ? 1 : 0;
        slow |= valid && (D <= A.a_hi || fabsf(D - A.w_mid) <= A.w_half);
      }
    }
    if (__any_sync(0xffffffffu, slow) && slow) {
      int nex = 0;
      slow_pairs<APPLY>(A, acc, ct * kTile + ty, rt * kTile + tx, full, false, nb, n, cnt, nex);
      if (nex) atomicAdd(&ctl->n_exact, (unsigned long long)nex);
    }
    if (!APPLY) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        int v = cnt[a];
#pragma unroll
        for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tx == 0) s_cnt[ty + 16 * a] += v;  // one writer per candidate row
      }
    }
  }
  if (!APPLY && cur_ct >= 0) {
    __syncthreads();
    for (int r = tid; r < kTile; r += kThreads) {
      const int k = cur_ct * kTile + r;
      if (k < nb && s_cnt[r]) atomicAdd(&A.ccount[k], s_cnt[r]);
    }
  }
}

// The counting pass with the candidate tile resident in shared memory (d <=
// DMAX): CTA b keeps candidate tile ct = b % nct and streams the row tiles
// rt = b / nct + m G (G = gridDim.x / nct) through an NST-stage cp.async ring
// (with three stages one barrier per tile suffices: the stage refilled after
// iteration m's barrier was last read at iteration m - 1);
// the candidates' counts stay in registers until the CTA ends. Full tiles test
// the slow-path conditions on the 64 pairs' minima (of D and of |D - w_mid|).
template <int DMAX, int NST>
__global__ void __launch_bounds__(kThreads, 2) spade_pairs_res_kernel(SpadeArgs A) {
  static_assert(NST == 2 || NST == 3, "two or three row stages");
  constexpr int RS = DMAX + 4;  // floats per staged row (16-byte aligned, spreads banks)
  extern __shared__ __align__(16) float sp_smem[];
  __shared__ int s_cnt[kTile];
  SpadeCtl* ctl = A.ctl;
  const int nb = ctl->nb;
  if (nb == 0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t n = A.n;
  const int d = A.d;
  const int nct = (nb + kTile - 1) / kTile;
  const int G = (int)gridDim.x / nct;
  if ((int)blockIdx.x >= nct * G) return;
  const int ct = (int)blockIdx.x % nct, g = (int)blockIdx.x / nct;
  const int nrt = (int)((n + kTile - 1) / kTile);
  if (g >= nrt) return;
  const int my = (nrt - 1 - g) / G + 1;  // row tiles of this CTA
  float* sa = sp_smem;
  float* sb0 = sa + kTile * RS;
  const int32_t* cand = A.cand + ct * kTile;
  stage_cols<DMAX>(sa, RS, A.X, d, A.vec, 0, min(kTile, nb - ct * kTile), [&](int r) { return cand[r]; }, tid);
  auto stage_b = [&](int rt, float* dst) {
    const int64_t r0 = (int64_t)rt * kTile;
    stage_cols<DMAX>(dst, RS, A.X, d, A.vec, 0, (int)min((int64_t)kTile, n - r0), [&](int r) { return r0 + r; },
                     tid);
  };
  stage_b(g, sb0);
  cp_async_commit();
  if (NST == 3 && my > 1) stage_b(g + G, sb0 + kTile * RS);
  if (NST == 3) cp_async_commit();  // (possibly empty) group of the second row tile
  int cnt[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) cnt[a] = 0;
  int nex = 0;
  const int nq = (d + 3) >> 2;
  const int k0 = ct * kTile + ty;
  for (int m = 0; m < my; ++m) {
    const int rt = g + m * G;
    if (NST == 2) {
      if (m + 1 < my) {
        stage_b(rt + G, sb0 + ((m + 1) & 1) * kTile * RS);
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      cp_async_wait<1>();  // every group but the newest (row tile m + 1): row tile m has landed
    }
    __syncthreads();
    if (NST == 3) {
      // every thread is past iteration m - 1, the last reader of stage (m + 2) % 3
      if (m + 2 < my) stage_b(rt + 2 * G, sb0 + ((m + 2) % 3) * kTile * RS);
      cp_async_commit();  // one group per iteration (empty near the end) keeps the count uniform
    }
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    accumulate_l1(acc, sa, sb0 + (m % NST) * kTile * RS, RS, nq, tx, ty);
    if (NST == 2) __syncthreads();  // this stage is refilled by the next iteration's prefetch

    const int64_t j0 = (int64_t)rt * kTile + tx;
    const bool full = (ct + 1) * kTile <= nb && (int64_t)(rt + 1) * kTile <= n;
    bool slow = !full;
    if (full) {
      float mnD = INFINITY, mnB = INFINITY;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
#pragma unroll
        for (int b = 0; b < 8; b += 2) {
          const float D0 = acc[a][b], D1 = acc[a][b + 1];
          cnt[a] += (D0 < A.w_lo ? 1 : 0) + (D1 < A.w_lo ? 1 : 0);
          mnD = min3f(mnD, D0, D1);
          mnB = min3f(mnB, fabsf(D0 - A.w_mid), fabsf(D1 - A.w_mid));
        }
      }
      slow = mnD <= A.a_hi || mnB <= A.w_half;
    }
    if (__any_sync(0xffffffffu, slow) && slow) slow_pairs<0>(A, acc, k0, j0, full, !full, nb, n, cnt, nex);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int v = cnt[a];
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tx == 0) s_cnt[ty + 16 * a] = v;  // one writer per candidate row
  }
  __syncthreads();
  for (int r = tid; r < kTile; r += kThreads) {
    const int k = ct * kTile + r;
    if (k < nb && s_cnt[r]) atomicAdd(&A.ccount[k], s_cnt[r]);
  }
  if (nex) atomicAdd(&ctl->n_exact, (unsigned long long)nex);
}

// Rows not yet found by any evaluated row, from the cursor, become the next
// batch's candidates (in index order). One block of kSB threads.
__global__ void __launch_bounds__(kSB) spade_select_kernel(SpadeArgs A) {
  __shared__ int s_warp[kSB / 32];
  __shared__ int s_found;
  __shared__ int64_t s_next;
  SpadeCtl* ctl = A.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t start = ctl->cursor;
  if (tid == 0) {
    s_found = 0;
    s_next = A.n;
  }
  // clear the batch state
  A.ccount[tid] = 0;
  A.inP[tid] = 0;
  uint4* nbr4 = reinterpret_cast<uint4*>(A.nbr);  // coalesced: consecutive threads, consecutive 16 bytes
  for (int w = tid; w < kSB * (kSB / 32) / 4; w += kSB) nbr4[w] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int64_t base = start; base < A.n; base += kSB) {
    const int found = s_found;
    if (found >= kSB) break;
    const int64_t row = base + tid;
    const bool f = row < A.n && A.q[row] == A.none;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kSB / 32; ++w) {
      const int c = s_warp[w];
      before += w < warp ? c : 0;
      total += c;
    }
    const int pos = found + before + __popc(bal & ((1u << lane) - 1u));
    if (f && pos < kSB) {
      A.cand[pos] = (int32_t)row;
      A.slot[row] = pos;
      if (pos == kSB - 1) s_next = row + 1;  // the batch is full: the next one starts after this row
    }
    __syncthreads();
    if (tid == 0) s_found = min(kSB, found + total);
    __syncthreads();
  }
  if (tid == 0) {
    ctl->nb = s_found;
    ctl->cursor = s_found >= kSB ? s_next : A.n;
    ctl->n_pairs = 0;
    ctl->overflow = 0;
  }
}

// Settles which candidates the loop evaluates: candidate k is evaluated exactly
// when no evaluated candidate k' < k of the batch finds it. Rounds over the
// batch: a candidate decides once every earlier candidate that finds it has
// decided; the lowest undecided one always can, so at most nb rounds run.
__global__ void __launch_bounds__(kSB) spade_resolve_kernel(SpadeArgs A) {
  __shared__ unsigned s_in[kSB / 32], s_und[kSB / 32];
  const int nb = A.ctl->nb;
  if (nb == 0) return;
  const int k = threadIdx.x, lane = k & 31, warp = k >> 5;
  uint32_t w[kSB / 32];
  {
    const uint4* row = reinterpret_cast<const uint4*>(A.nbr + (size_t)k * (kSB / 32));
#pragma unroll
    for (int i = 0; i < kSB / 128; ++i) {
      const uint4 v = k < nb ? row[i] : make_uint4(0u, 0u, 0u, 0u);
      w[4 * i] = v.x;
      w[4 * i + 1] = v.y;
      w[4 * i + 2] = v.z;
      w[4 * i + 3] = v.w;
    }
  }
  int st = k < nb ? 0 : 2;  // 0 undecided, 1 evaluated, 2 skipped
  {
    const unsigned u = __ballot_sync(0xffffffffu, st == 0);
    if (lane == 0) {
      s_und[warp] = u;
      s_in[warp] = 0u;
    }
  }
  __syncthreads();
  for (int round = 0; round <= kSB; ++round) {
    if (st == 0) {
      uint32_t any_in = 0, any_und = 0;
#pragma unroll
      for (int i = 0; i < kSB / 32; ++i) {
        any_in |= w[i] & s_in[i];
        any_und |= w[i] & s_und[i];
      }
      if (any_in) st = 2;
      else if (!any_und) st = 1;
    }
    __syncthreads();
    const unsigned bi = __ballot_sync(0xffffffffu, st == 1), bu = __ballot_sync(0xffffffffu, st == 0);
    if (lane == 0) {
      s_in[warp] = bi;
      s_und[warp] = bu;
    }
    if (!__syncthreads_or(st == 0)) break;
  }
  if (k < nb) A.inP[k] = st == 1;
}

// Every row found by an evaluated candidate records it as a writer.
__global__ void __launch_bounds__(256) spade_apply_kernel(SpadeArgs A) {
  const SpadeCtl* ctl = A.ctl;
  if (ctl->nb == 0 || ctl->overflow) return;
  const int64_t np = (int64_t)min(ctl->n_pairs, (unsigned long long)A.pair_cap);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < np; e += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = A.pairs[e];
    if (!A.inP[p.x]) continue;
    const int32_t ci = A.cand[p.x];
    if (A.policy == 0) atomicMax(&A.q[p.y], ci);
    else atomicMin(&A.q[p.y], ci);
  }
}

// Counts and flags of the evaluated candidates; releases the batch slots.
__global__ void __launch_bounds__(kSB) spade_finish_kernel(SpadeArgs A) {
  SpadeCtl* ctl = A.ctl;
  const int nb = ctl->nb, k = threadIdx.x;
  const bool ev = k < nb && A.inP[k];
  if (k < nb) {
    const int32_t r = A.cand[k];
    A.slot[r] = -1;
    if (ev) {
      A.processed[r] = 1;
      A.counts[r] = A.ccount[k];
    }
  }
  const int nev = __syncthreads_count(ev);
  if (k == 0) {
    ctl->n_computed += (unsigned long long)nb;
    ctl->n_evaluated += (unsigned long long)nev;
    ctl->n_apprx += ctl->n_pairs;
    ctl->overflow_batches += ctl->overflow ? 1 : 0;
    ctl->batches += nb > 0 ? 1 : 0;
    if (nb == 0) ctl->done = 1;
  }
}

__global__ void __launch_bounds__(256) spade_init_kernel(SpadeArgs A) {
  const int64_t nd = A.n * (int64_t)A.d;
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nd; e += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(A.X[e]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) A.ctl->nonfinite = 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    A.q[i] = A.none;
    A.slot[i] = -1;
    A.counts[i] = -1;
    A.processed[i] = 0;
  }
}

// densities[i] = count of row i's writer.
__global__ void __launch_bounds__(256) spade_density_kernel(SpadeArgs A, int32_t* __restrict__ dens) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t w = A.q[i];
    dens[i] = (w >= 0 && w < A.n) ? A.counts[w] : 0;
  }
}

constexpr size_t kPairSmem = (size_t)2 * 2 * kSideFloats * sizeof(float);
template <int DMAX, int NST>
constexpr size_t res_smem() {
  return (size_t)(1 + NST) * kTile * (DMAX + 4) * sizeof(float);  // candidates + NST row stages
}

}  // namespace

size_t spade_pairs_smem() { return kPairSmem; }

cudaError_t init_spade() {
  cudaError_t e = cudaFuncSetAttribute(spade_pairs_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPairSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spade_pairs_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spade_pairs_res_kernel<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)res_smem<32, 2>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(spade_pairs_res_kernel<64, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)res_smem<64, 2>());
  return e;
}

cudaError_t launch_spade_init(const SpadeArgs& A, cudaStream_t s) {
  int64_t blocks = (A.n * A.d + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  spade_init_kernel<<<(int)blocks, 256, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_spade_batch(const SpadeArgs& A, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  spade_select_kernel<<<1, kSB, 0, s>>>(A);
  const int64_t tiles = (int64_t)(kSB / kTile) * ((A.n + kTile - 1) / kTile);
  const int grid = (int)std::min<int64_t>(tiles, 2 * (int64_t)num_sms());
  cudaError_t e;
  if (e0 && (e = cudaEventRecord(e0, s)) != cudaSuccess) return e;
  if (A.d <= 32) spade_pairs_res_kernel<32, 2><<<grid, kThreads, res_smem<32, 2>(), s>>>(A);
  else if (A.d <= 64) spade_pairs_res_kernel<64, 2><<<grid, kThreads, res_smem<64, 2>(), s>>>(A);
  else spade_pairs_kernel<0><<<grid, kThreads, kPairSmem, s>>>(A);
  if (e1 && (e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
  spade_resolve_kernel<<<1, kSB, 0, s>>>(A);
  int ab = (int)std::min<int64_t>((A.pair_cap + 255) / 256, num_sms() * 8);
  spade_apply_kernel<<<ab, 256, 0, s>>>(A);
  spade_pairs_kernel<1><<<grid, kThreads, kPairSmem, s>>>(A);
  spade_finish_kernel<<<1, kSB, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_spade_density(const SpadeArgs& A, int32_t* dens, cudaStream_t s) {
  int64_t blocks = (A.n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  spade_density_kernel<<<(int)blocks, 256, 0, s>>>(A, dens);
  return cudaGetLastError();
}

}  // namespace km
