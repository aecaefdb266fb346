// FP32 fused distance + argmin on the SIMT FFMA pipes.
//
// The distance loop, the argmin and the error test are one pass over a
// 128-point row tile (vertical fusion with array contraction, Sec. 3.5): the
// n x k score matrix lives only in registers, one 128 x 128 chunk at a time,
// the way the Stream of Sec. 4.1 evaluates its distance matrix chunk by chunk
// into the consumer.
//
// Score. With h_j = ||c_j||^2 / 2 (prepared once per iteration, Sec. 3.1),
//   ||x - c_j||^2 = ||x||^2 + 2 (h_j - x.c_j),
// so the argmin over j of s_j = h_j - x.c_j is the distance argmin, and
// ||x||^2 never has to be added.
//
// Error bound (u = 2^-24, gamma_m = m u / (1 - m u)). The dot product is an
// FMA chain over d terms: |fl(x.c) - x.c| <= gamma_d sum_t |x_t c_t|
// <= gamma_d ||x|| ||c||. h_j carries <= 2u h_j (FP64 norm rounded to FP32),
// and the subtraction one more rounding, so for every j
//   |s^_j - s_j| <= E_i = 3u H + gamma_{d+1} ||x_i|| Cmax,
// with H = max_j h_j and Cmax = max_j ||c_j|| (rounded up). If the computed
// top-2 scores satisfy s^_2 - s^_1 > 2 E_i, every other centroid is strictly
// farther than j1 in exact arithmetic, so j1 is the exact argmin. Otherwise
// the point is flagged and re-checked with compensated FP32 distances. The
// FMA chain is the same whether it runs as scalar or paired (FFMA2) FMAs: each
// accumulator takes one rounding per term, so the bound does not change.
#include <type_traits>

#include "km_internal.cuh"

namespace km {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, PAD = 4;
constexpr int THREADS = 256;
// Slab kernel: 8 rows x 4 columns of scores per thread. The 32 lanes of a warp
// take the 128 columns of a chunk (4 adjacent columns each) and share its 8
// rows: a centroid load is 32 distinct 16-byte words, a point load one
// broadcast word holding 4 rows of one dimension (the point tile is staged
// transposed), and each paired FMA takes two adjacent rows against one
// centroid coordinate.
constexpr int SR = 8;
// Slab kernel geometries: G = 0, 512 threads on 128-row tiles, one CTA per SM
// (the largest slab); G = 1, 256 threads on 64-row tiles, two CTAs per SM (half
// the slab each; their barriers and epilogues no longer line up).
template <int G>
struct SlabGeo {
  static constexpr int T = G ? 256 : 512, M = G ? 64 : 128, CTAS = G ? 2 : 1;
};
__device__ __forceinline__ int srow_of(int wq, int r) { return wq * SR + r; }

__device__ __forceinline__ int row_of(int ty, int r) { return r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4); }
__device__ __forceinline__ int col_of(int tx, int c) { return c < 4 ? tx * 4 + c : 64 + tx * 4 + (c - 4); }

// Best score and index of a row, and the second-best score (its index is not
// needed: a flagged point is re-checked against every centroid).
struct Top2 {
  float b1, b2;
  int i1;
};

__device__ __forceinline__ void top2_push(Top2& t, float s, int j) {
  // Columns arrive in increasing j, so strict comparisons keep the lowest
  // index among equal scores. Branch-free: a NaN score changes nothing.
  const bool lt1 = s < t.b1;
  t.b2 = lt1 ? t.b1 : fminf(t.b2, s);
  t.i1 = lt1 ? j : t.i1;
  t.b1 = lt1 ? s : t.b1;
}

__device__ __forceinline__ Top2 top2_merge(const Top2& a, const Top2& b) {
  Top2 r;
  if (lex_less(b.b1, b.i1, a.b1, a.i1)) {
    r.b1 = b.b1; r.i1 = b.i1;
    r.b2 = fminf(a.b1, b.b2);
  } else {
    r.b1 = a.b1; r.i1 = a.i1;
    r.b2 = fminf(b.b1, a.b2);
  }
  return r;
}

// Re-check passes over gathered rows keep the best two (score, index) pairs
// and the third-best score: when the third lies outside the margin, the two
// are the complete candidate list of the point.
struct Top3s {
  float b1, b2, b3;
  int i1, i2;
};

__device__ __forceinline__ void top_push(Top2& t, float s, int j) { top2_push(t, s, j); }
__device__ __forceinline__ void top_push(Top3s& t, float s, int j) {
  // branch-free sorted insert; columns arrive in increasing j, so strict
  // comparisons keep the lowest index first; a NaN score changes nothing
  const bool lt1 = s < t.b1, lt2 = s < t.b2;
  t.b3 = lt2 ? t.b2 : fminf(t.b3, s);
  t.i2 = lt1 ? t.i1 : (lt2 ? j : t.i2);
  t.b2 = lt1 ? t.b1 : (lt2 ? s : t.b2);
  t.i1 = lt1 ? j : t.i1;
  t.b1 = lt1 ? s : t.b1;
}

__device__ __forceinline__ Top3s top_merge(Top3s a, Top3s b) {
  if (lex_less(b.b1, b.i1, a.b1, a.i1)) {
    const Top3s t = a;
    a = b;
    b = t;
  }
  Top3s r;
  r.b1 = a.b1;
  r.i1 = a.i1;
  if (lex_less(b.b1, b.i1, a.b2, a.i2)) {
    r.b2 = b.b1;
    r.i2 = b.i1;
    r.b3 = fminf(a.b2, b.b2);
  } else {
    r.b2 = a.b2;
    r.i2 = a.i2;
    r.b3 = fminf(a.b3, b.b1);
  }
  return r;
}

// Order-preserving integer key of a score (-0 first made +0, so equal scores
// give equal keys; scores here are never NaN).
__device__ __forceinline__ int score_key(float x) {
  const int k = __float_as_int(x + 0.f);
  return k ^ ((k >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_score(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }

// The merged top-2 of a warp's 32 lanes for one row: the best score, its
// lowest index among equal scores, and the second-best score (three full-warp
// minimum reductions over order-preserving keys).
__device__ __forceinline__ Top2 warp_top2(const Top2& t) {
  const int k1 = score_key(t.b1);
  const int m1 = __reduce_min_sync(0xffffffffu, k1);
  const bool win = k1 == m1;
  const int i1 = __reduce_min_sync(0xffffffffu, win ? t.i1 : INT_MAX);
  const bool me = win && t.i1 == i1;  // the lane holding the winner (indices are distinct across lanes)
  const int m2 = __reduce_min_sync(0xffffffffu, score_key(me ? t.b2 : t.b1));
  return Top2{key_score(m1), key_score(m2), i1};
}

__device__ __forceinline__ Top3s top_shfl_xor(const Top3s& t, int o) {
  Top3s p;
  p.b1 = __shfl_xor_sync(0xffffffffu, t.b1, o);
  p.b2 = __shfl_xor_sync(0xffffffffu, t.b2, o);
  p.b3 = __shfl_xor_sync(0xffffffffu, t.b3, o);
  p.i1 = __shfl_xor_sync(0xffffffffu, t.i1, o);
  p.i2 = __shfl_xor_sync(0xffffffffu, t.i2, o);
  return p;
}

// Loads a BK-wide slice [k0, k0+BK) of `rows` rows starting at r0 of a
// row-major (nrows x d) matrix into registers (coalesced along d).
__device__ __forceinline__ void load_slice(const float* __restrict__ M, int64_t nrows, int d,
                                           int64_t r0, int k0, float (&v)[BM * BK / THREADS]) {
#pragma unroll
  for (int q = 0; q < BM * BK / THREADS; ++q) {
    int e = threadIdx.x + q * THREADS;
    int r = e / BK, c = e % BK;
    int64_t row = r0 + r;
    int col = k0 + c;
    v[q] = (row < nrows && col < d) ? __ldg(M + row * d + col) : 0.f;
  }
}

__device__ __forceinline__ void store_slice(float (*S)[BM + PAD], const float (&v)[BM * BK / THREADS]) {
#pragma unroll
  for (int q = 0; q < BM * BK / THREADS; ++q) {
    int e = threadIdx.x + q * THREADS;
    S[e % BK][e / BK] = v[q];
  }
}

__global__ void __launch_bounds__(THREADS, 1)
assign_simt_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ C, int k,
                   const float* __restrict__ chalf, const float* __restrict__ xnorm, Ctl* ctl,
                   int32_t* __restrict__ assign, FlagRec* __restrict__ flags, int first, float gam,
                   const SubRows sr) {
  if (halted(ctl)) return;
  if (sr.n_dev) n = min(n, (int64_t)*sr.n_dev);  // gathered rows of the re-check stage (n = capacity)
  extern __shared__ __align__(16) float smem[];
  float (*As)[BM + PAD] = reinterpret_cast<float (*)[BM + PAD]>(smem);
  float (*Bs)[BM + PAD] = reinterpret_cast<float (*)[BM + PAD]>(smem + BK * (BM + PAD));
  __shared__ unsigned int s_changed;

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float H = __uint_as_float(ctl->hmax_bits);
  const float Cmax = __uint_as_float(ctl->cmax_bits);
  const int64_t ntiles = (n + BM - 1) / BM;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t m0 = tile * BM;
    Top2 top[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) top[r] = Top2{INFINITY, INFINITY, 0};

    for (int j0 = 0; j0 < k; j0 += BN) {
      float2 acc2[8][4];  // (acc[r][2c], acc[r][2c + 1]): one paired FMA per two columns
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[r][c] = make_float2(0.f, 0.f);

      float va[BM * BK / THREADS], vb[BM * BK / THREADS];
      load_slice(X, n, d, m0, 0, va);
      load_slice(C, k, d, j0, 0, vb);
      for (int k0 = 0; k0 < d; k0 += BK) {
        __syncthreads();
        store_slice(As, va);
        store_slice(Bs, vb);
        __syncthreads();
        if (k0 + BK < d) {  // prefetch the next slice while this one is consumed
          load_slice(X, n, d, m0, k0 + BK, va);
          load_slice(C, k, d, j0, k0 + BK, vb);
        }
        const int kend = min(BK, d - k0);
#pragma unroll 8
        for (int kk = 0; kk < kend; ++kk) {
          float a[8], b[8];
          *reinterpret_cast<float4*>(&a[0]) = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
          *reinterpret_cast<float4*>(&a[4]) = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
          *reinterpret_cast<float4*>(&b[0]) = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
          *reinterpret_cast<float4*>(&b[4]) = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float2 ar = make_float2(a[r], a[r]);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc2[r][c] = __ffma2_rn(ar, make_float2(b[2 * c], b[2 * c + 1]), acc2[r][c]);
          }
        }
      }
      float acc[8][8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][2 * c] = acc2[r][c].x;
          acc[r][2 * c + 1] = acc2[r][c].y;
        }
      // epilogue of this chunk: scores and running top-2 per row
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = j0 + col_of(tx, c);
        if (j < k) {
          const float hj = __ldg(chalf + j);
#pragma unroll
          for (int r = 0; r < 8; ++r) top2_push(top[r], __fsub_rn(hj, acc[r][c]), j);
        }
      }
    }

    // merge the 16 column-threads that share each row (lanes differ in tx only)
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int o = 8; o; o >>= 1) {
        Top2 p;
        p.b1 = __shfl_xor_sync(0xffffffffu, top[r].b1, o);
        p.b2 = __shfl_xor_sync(0xffffffffu, top[r].b2, o);
        p.i1 = __shfl_xor_sync(0xffffffffu, top[r].i1, o);
        top[r] = top2_merge(top[r], p);
      }
    }
    if (tid == 0) s_changed = 0;
    __syncthreads();
    if (tx == 0) {
      unsigned int changed = 0;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t i = m0 + row_of(ty, r);
        if (i < n) {
          const int64_t pt = sr.rows ? (int64_t)sr.rows[i] : i;  // the point of row i
          int old = sr.rows ? sr.old[i] : (first ? -1 : assign[pt]);
          if (old < 0 || old >= k) old = -1;
          const float E = fmaf(3.f * kU, H, gam * xnorm[i] * Cmax);
          const float margin = 2.f * E * (1.f + 0x1p-10f);
          const int j1 = top[r].i1;
          if (__fsub_rn(top[r].b2, top[r].b1) <= margin) {
            unsigned long long slot = atomicAdd(sr.nflag ? sr.nflag : &ctl->n_flagged, 1ull);
            FlagRec rec;
            rec.i = (int32_t)pt; rec.old = old; rec.nc = 0; rec.pad = 0;
            rec.cand[0] = rec.cand[1] = rec.cand[2] = rec.cand[3] = 0;
            (sr.flags ? sr.flags : flags)[slot] = rec;
            if (!sr.rows) atomicAdd(&ctl->n_full, 1ull);
          } else {
            changed += (old != j1);
          }
          assign[pt] = j1;
        }
      }
      if (changed) atomicAdd(&s_changed, changed);
    }
    __syncthreads();
    if (tid == 0 && s_changed) atomicAdd(&ctl->n_changed, (unsigned long long)s_changed);
  }
}


// ---------------------------------------------------------------------------
// Slab-resident variant (d <= 128). A slab of up to kSlab centroids is loaded
// into shared memory once per CTA (transposed, with its h_j); point tiles
// stream through a cp.async double buffer, staged transposed, and each thread
// keeps 8 rows x 4 columns of scores. A row's running (best, index, second) lives in
// registers within a slab and in `state` between slabs; the last slab applies
// the same error-bound test as the streaming kernel above.
constexpr int kSlabMaxD = 128;
// Floats between consecutive K rows of a staged centroid chunk (BN columns +
// 4): 4 modulo 32, so that the slab fill (8 dimensions of 4 centroids per warp
// copy) meets 32 distinct banks; rows stay 16-byte aligned.
constexpr int BNP = BN + 4;

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Issues the copies of point tile `tile` into XsT, transposed: dimension t of
// tile row r goes to XsT[t * xs_stride + r] (xs_stride = tile rows + 4). A warp
// copies 8 consecutive dimensions of 4 rows per instruction: 4 fully used
// 32-byte sectors from global memory, and 32 distinct banks in shared memory
// (xs_stride is 4 modulo 32). Rows past n are not copied.
template <int G>
__device__ __forceinline__ void load_tile_async(float* XsT, int xs_stride, const float* __restrict__ X, int64_t n,
                                                int d, int64_t tile) {
  constexpr int SBM = SlabGeo<G>::M, ST = SlabGeo<G>::T;
  const int64_t m0 = tile * SBM;
  const int rows = (int)(n - m0 < SBM ? n - m0 : SBM);
  const int lane = threadIdx.x & 31, tl = lane & 7;
  // warp: groups of 4 rows; lane: row lane / 8 of the group, dimensions lane % 8 + 8 m
  for (int r = (threadIdx.x >> 5) * 4 + (lane >> 3); r < rows; r += ST / 8) {
    const float* src = X + (m0 + r) * d + tl;
    float* dst = XsT + tl * xs_stride + r;
    for (int t = tl; t < d; t += 8, src += 8, dst += 8 * xs_stride) cp_async4(dst, src);
  }
}

// T3 (re-check passes over gathered rows): the best two candidates and the
// third-best score are kept, and a flagged row whose third-best score lies
// outside the margin is recorded with its two candidates; the third-best
// score crosses slabs in state3.
template <bool T3, int G>
__global__ void __launch_bounds__(SlabGeo<G>::T, SlabGeo<G>::CTAS)
assign_slab_kernel(const float* __restrict__ X, int64_t n, int d, int dp, const float* __restrict__ C, int k,
                   int j_lo, int ns, const float* __restrict__ chalf, const float* __restrict__ xnorm, Ctl* ctl,
                   int32_t* __restrict__ assign, FlagRec* __restrict__ flags, float4* __restrict__ state,
                   float* __restrict__ state3, int first, int first_slab, int last_slab, float gam,
                   const SubRows sr) {
  using TopT = typename std::conditional<T3, Top3s, Top2>::type;
  constexpr int ST = SlabGeo<G>::T, SBM = SlabGeo<G>::M;
  if (halted(ctl)) return;
  if (sr.n_dev) n = min(n, (int64_t)*sr.n_dev);  // gathered rows of the re-check stage (n = capacity)
  if ((int64_t)blockIdx.x * SBM >= n) return;    // no tile for this CTA: skip the slab load
  extern __shared__ __align__(16) float smem[];
  const int nsp = (ns + BN - 1) / BN * BN;  // slab columns padded to whole chunks
  const int xs_stride = SBM + 4;            // floats per staged dimension (a row of the transposed tile)
  float* Cs = smem;                          // [nsp / BN][dp][BNP]: per chunk, K rows BNP floats apart
  float* Hs = Cs + (size_t)dp * (nsp / BN) * BNP;  // [nsp]
  float* Xs0 = Hs + nsp;                     // 2 x [dp][xs_stride]: point tiles, transposed
  __shared__ unsigned int s_changed;

  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  // slab of centroids, transposed, by 4-byte cp.async (every load in flight at once; the first
  // tile's wait completes them): a warp copies 8 dimensions of 4 centroids per instruction;
  // zero padding in [d, dp) and [ns, nsp)
  for (int j = (tid >> 5) * 4 + (lane >> 3); j < nsp; j += ST / 8) {
    float* dst = Cs + (size_t)(j / BN) * dp * BNP + (j % BN);
    const float* src = C + (int64_t)(j_lo + (j < ns ? j : 0)) * d;
    for (int t = lane & 7; t < dp; t += 8) {
      if (j < ns && t < d) cp_async4(dst + t * BNP, src + t);
      else dst[t * BNP] = 0.f;
    }
  }
  cp_async_commit();
  for (int j = tid; j < nsp; j += ST) Hs[j] = j < ns ? __ldg(chalf + j_lo + j) : INFINITY;
  // zero both point buffers once: padding dimensions [d, dp) stay zero
  for (int e = tid; e < 2 * dp * xs_stride; e += ST) Xs0[e] = 0.f;
  __syncthreads();

  const float H = __uint_as_float(ctl->hmax_bits);
  const float Cmax = __uint_as_float(ctl->cmax_bits);
  const int64_t ntiles = (n + SBM - 1) / SBM;
  int buf = 0;
  if ((int64_t)blockIdx.x < ntiles) load_tile_async<G>(Xs0, xs_stride, X, n, d, blockIdx.x);
  cp_async_commit();
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    float* Xs = Xs0 + buf * dp * xs_stride;
    if (next < ntiles) load_tile_async<G>(Xs0 + (buf ^ 1) * dp * xs_stride, xs_stride, X, n, d, next);
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();

    const int64_t m0 = tile * SBM;
    TopT top[SR];
#pragma unroll
    for (int r = 0; r < SR; ++r) {
      const int64_t i = m0 + srow_of(wq, r);
      // the carried state enters through one of the 32 lanes sharing the row,
      // so the cross-thread merge sees it once
      if constexpr (T3) {
        if (!first_slab && lane == 0 && i < n) {
          const float4 st = state[i];
          top[r] = Top3s{st.x, st.z, state3[i], __float_as_int(st.y), __float_as_int(st.w)};
        } else {
          top[r] = Top3s{INFINITY, INFINITY, INFINITY, 0, 0};
        }
      } else {
        if (!first_slab && lane == 0 && i < n) {
          const float4 st = state[i];
          top[r] = Top2{st.x, st.z, __float_as_int(st.y)};
        } else {
          top[r] = Top2{INFINITY, INFINITY, 0};
        }
      }
    }
    for (int j0 = 0; j0 < nsp; j0 += BN) {
      const float* Cc = Cs + (size_t)(j0 / BN) * dp * BNP;  // this chunk's [dp][BNP] block
      float2 acc2[SR / 2][4];  // (acc[2p][c], acc[2p + 1][c]): one paired FMA per two rows
#pragma unroll
      for (int p = 0; p < SR / 2; ++p)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[p][c] = make_float2(0.f, 0.f);
      const float* xr = Xs + wq * SR;
      const float* cr = Cc + lane * 4;
#pragma unroll 8
      for (int kk = 0; kk < dp; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(xr + kk * xs_stride);
        const float4 a1 = *reinterpret_cast<const float4*>(xr + kk * xs_stride + 4);
        const float4 b = *reinterpret_cast<const float4*>(cr + kk * BNP);
        const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                              make_float2(a1.z, a1.w)};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 bc = make_float2(bv[c], bv[c]);
#pragma unroll
          for (int p = 0; p < SR / 2; ++p) acc2[p][c] = __ffma2_rn(ap[p], bc, acc2[p][c]);
        }
      }
      const float4 h4 = *reinterpret_cast<const float4*>(Hs + j0 + lane * 4);
      const float hj[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j_lo + j0 + lane * 4 + c;
#pragma unroll
        for (int p = 0; p < SR / 2; ++p) {
          top_push(top[2 * p], __fsub_rn(hj[c], acc2[p][c].x), j);
          top_push(top[2 * p + 1], __fsub_rn(hj[c], acc2[p][c].y), j);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < SR; ++r) {
      if constexpr (T3) {
#pragma unroll
        for (int o = 16; o; o >>= 1) top[r] = top_merge(top[r], top_shfl_xor(top[r], o));
      } else {
        top[r] = warp_top2(top[r]);
      }
    }
    if (tid == 0) s_changed = 0;
    __syncthreads();  // also: every thread is done reading Xs before it is refilled
    // after the merge every lane of the warp holds its rows' results: lane r < SR settles row r
    if (lane < SR) {
      unsigned int changed = 0;
      TopT tr = top[0];
#pragma unroll
      for (int q = 1; q < SR; ++q)
        if (lane == q) tr = top[q];
      {
        const int r = lane;
        const int64_t i = m0 + srow_of(wq, r);
        if (i >= n) goto row_done;
        if (!last_slab) {
          if constexpr (T3) {
            state[i] = make_float4(tr.b1, __int_as_float(tr.i1), tr.b2, __int_as_float(tr.i2));
            state3[i] = tr.b3;
          } else {
            state[i] = make_float4(tr.b1, __int_as_float(tr.i1), tr.b2, 0.f);
          }
          goto row_done;
        }
        const int64_t pt = sr.rows ? (int64_t)sr.rows[i] : i;  // the point of row i
        int old = sr.rows ? sr.old[i] : (first ? -1 : assign[pt]);
        if (old < 0 || old >= k) old = -1;
        const float E = fmaf(3.f * kU, H, gam * xnorm[i] * Cmax);
        const float margin = 2.f * E * (1.f + 0x1p-10f);
        const int j1 = tr.i1;
        if (__fsub_rn(tr.b2, tr.b1) <= margin) {
          const unsigned long long slot = atomicAdd(sr.nflag ? sr.nflag : &ctl->n_flagged, 1ull);
          FlagRec rec;
          rec.i = (int32_t)pt; rec.old = old; rec.nc = 0; rec.pad = 0;
          rec.cand[0] = rec.cand[1] = rec.cand[2] = rec.cand[3] = 0;
          if constexpr (T3) {
            if (__fsub_rn(tr.b3, tr.b1) > margin) {  // no third centroid can be the nearest
              rec.nc = 2;
              rec.cand[0] = min(j1, tr.i2);
              rec.cand[1] = max(j1, tr.i2);
            }
          }
          (sr.flags ? sr.flags : flags)[slot] = rec;
          if (!sr.rows) atomicAdd(&ctl->n_full, 1ull);
        } else {
          changed += (old != j1);
        }
        assign[pt] = j1;
      }
    row_done:
      if (changed) atomicAdd(&s_changed, changed);
    }
    __syncthreads();
    if (tid == 0 && s_changed) atomicAdd(&ctl->n_changed, (unsigned long long)s_changed);
    buf ^= 1;
  }
  cp_async_wait_1();
}

size_t slab_smem_bytes(int dp, int nsp, int rows) {
  return ((size_t)dp * (nsp / BN) * BNP + nsp + 2 * (size_t)dp * (rows + 4)) * sizeof(float);
}

// Centroids per slab of geometry G for dimension d (0: does not fit).
int slab_width_g(int d, int G) {
  if (d > kSlabMaxD) return 0;
  const int dp = (d + 3) / 4 * 4;
  const size_t budget = (G ? 113 : 227) * 1024 - 2048;  // per CTA
  const size_t fixed = 2 * (size_t)dp * ((G ? SlabGeo<1>::M : SlabGeo<0>::M) + 4) * sizeof(float);
  if (fixed >= budget) return 0;
  const size_t per_chunk = ((size_t)dp * BNP + BN) * sizeof(float);  // one chunk of BN centroids and its h_j
  const int ns = (int)((budget - fixed) / per_chunk) * BN;
  return ns >= BN ? ns : 0;
}

}  // namespace

cudaError_t init_assign_simt() {
  cudaError_t e = cudaFuncSetAttribute(assign_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * BK * (BM + PAD) * sizeof(float)));
  int dev = 0, optin = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  auto raise = [&](auto kernel) {
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  };
  raise(assign_slab_kernel<false, 0>);
  raise(assign_slab_kernel<true, 0>);
  raise(assign_slab_kernel<false, 1>);
  raise(assign_slab_kernel<true, 1>);
  return e;
}

// Centroids per slab for dimension d (0: the slab kernel does not apply).
int simt_slab_width(int d) { return slab_width_g(d, 0); }

// p.X / p.n: the rows to assign (the gathered rows and their capacity for a
// re-check pass); chalf, xnorm: h_j and the rows' norm bounds.
cudaError_t launch_assign_slab(const Problem& p, const Work& w, const float* chalf, const float* xnorm, int first,
                               const SubRows& sr, cudaStream_t s) {
  const double u = 1.0 / 16777216.0;
  const double m = p.d + 1;
  const float gam = (float)(m * u / (1.0 - m * u) * (1.0 + 1e-6));
  const int dp = (p.d + 3) / 4 * 4;
  // two CTAs per SM when all k centroids fit the half-size slab, else one CTA with the larger slab
  const int G = (slab_width_g(p.d, 1) >= p.k) ? 1 : 0;
  const int width = slab_width_g(p.d, G), rows = G ? SlabGeo<1>::M : SlabGeo<0>::M;
  const int64_t tiles = (p.n + rows - 1) / rows;
  const int64_t cap = (int64_t)num_sms() * (G ? SlabGeo<1>::CTAS : SlabGeo<0>::CTAS);
  const int blocks = (int)(tiles < cap ? tiles : cap);
  for (int j_lo = 0; j_lo < p.k; j_lo += width) {
    const int ns = p.k - j_lo < width ? p.k - j_lo : width;
    const int nsp = (ns + BN - 1) / BN * BN;
    const size_t smem = slab_smem_bytes(dp, nsp, rows);
    const int first_slab = j_lo == 0, last_slab = j_lo + width >= p.k;
    // passes over gathered re-check rows keep a third score (candidate lists of two)
    const bool t3 = sr.rows != nullptr;
#define KM_SLAB(T3_, G_)                                                                                    \
  assign_slab_kernel<T3_, G_><<<blocks, SlabGeo<G_>::T, smem, s>>>(                                         \
      p.X, p.n, p.d, dp, p.C, p.k, j_lo, ns, chalf, xnorm, w.ctl, p.assign, w.flags, w.state, w.state3, first, \
      first_slab, last_slab, gam, sr)
    if (G) {
      if (t3) KM_SLAB(true, 1);
      else KM_SLAB(false, 1);
    } else {
      if (t3) KM_SLAB(true, 0);
      else KM_SLAB(false, 0);
    }
#undef KM_SLAB
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_assign_any(const Problem& p, const Work& w, const float* chalf, const float* xnorm, int first,
                              const SubRows& sr, cudaStream_t s) {
  if (simt_slab_width(p.d) > 0) return launch_assign_slab(p, w, chalf, xnorm, first, sr, s);
  const size_t smem = 2 * BK * (BM + PAD) * sizeof(float);
  const double u = 1.0 / 16777216.0;
  const double m = p.d + 1;
  const float gam = (float)(m * u / (1.0 - m * u) * (1.0 + 1e-6));
  int64_t tiles = (p.n + BM - 1) / BM;
  int64_t cap = (int64_t)num_sms();
  int blocks = (int)(tiles < cap ? tiles : cap);
  assign_simt_kernel<<<blocks, THREADS, smem, s>>>(p.X, p.n, p.d, p.C, p.k, chalf, xnorm, w.ctl, p.assign, w.flags,
                                                   first, gam, sr);
  return cudaGetLastError();
}

cudaError_t launch_assign_simt(const Problem& p, const Work& w, int first, cudaStream_t s) {
  const SubRows none{nullptr, nullptr, nullptr, nullptr, nullptr};
  return launch_assign_any(p, w, w.chalf, w.xnorm, first, none, s);
}

cudaError_t launch_assign_simt_sub(const Problem& p, const Work& w, const float* h, cudaStream_t s) {
  const SubRows sr{w.fq_rows, w.fq_old, &w.ctl->n_fullq, &w.ctl->n_flagged2, w.flags2};
  Problem q = p;
  q.X = w.X_sub;
  q.n = w.fq_cap;
  return launch_assign_any(q, w, h, w.xn_sub, 0, sr, s);
}

}  // namespace km
