// Tensor-core fused distance + argmin (BF16 or FP8-E4M3 operands, FP32 accumulate).
//
// One pass per 128-point row tile (vertical fusion with array contraction,
// Sec. 3.5): TMA stages the point codes (A, once per tile) and 128-centroid
// chunks of the centroid codes (B) into shared memory with the 128-byte
// swizzle; one thread issues tcgen05.mma into TMEM accumulators (four buffers,
// so the MMAs of the next chunks overlap the epilogue of chunk c); the
// epilogue warps read their TMEM lane quarter with tcgen05.ld -- thread t of a
// warp of quarter q owns point row 32q + t -- and fold the chunk's scores into
// a per-row candidate list in registers. The n x k score matrix never leaves
// TMEM.
//
// Tiles. A single-instance launch deals row tiles round-robin to the CTAs; a
// batched launch gives each CTA one contiguous range of the flattened tiles
// (ranges balanced by MMA + epilogue work on the host), so a CTA meets each
// instance once and walks its tiles in order. The epilogue loads the row
// metadata of the CTA's next tile while it works on the current one.
//
// Roles (352 threads): warp 0 = TMA producer, warp 1 = MMA issuer of the first
// tile of each pair and TMEM owner, warps 2-9 = epilogue in two groups of four
// (one warp per TMEM lane quarter), warp 10 = MMA issuer of the second tile.
// Row tiles go in pairs: each B chunk is loaded once and multiplied with both
// tiles of the pair (each issuer commits the B stage, so it is refilled after
// both), group u scores tile u (accumulators in TMEM buffers u and u + 2), and
// each row has a single owner thread that sees all of
// its columns. h_j (and the FP8 scales) are staged in shared memory once per
// CTA. Every mbarrier wait is bounded in time; on
// expiry the kernel records KM_ETIMEOUT, drains what it issued, frees TMEM and
// returns.
//
// Scores. With codes q and power-of-two scales (x~ = sx q_x with a scale per
// point row, c~ = sc q_c with one scale for all centroids of the step; BF16
// uses sx = sc = 1), the epilogue computes
//   s^_j = h_j - (sx sc) acc_j,  acc_j = sum_t q_x,t q_c,jt  (TMEM, FP32),
// whose argmin over j is the distance argmin up to the quantisation error.
//
// Error bound (u = 2^-24; the tensor core accumulates in FP32 with truncation,
// so gamma'_K = K 2^-23 / (1 - K 2^-23)): for every j
//   |s^_j - s_j| <= e_ij = 3u h_j + (gamma'_K + 2u) ||x~_i|| ||c~_j||
//                        + ||dx_i|| ||c_j|| + ||x_i|| ||dc_j|| + ||dx_i|| ||dc_j||,
// where dx = x~ - x, dc = c~ - c (the centroid's own terms come from a table
// the centroid quantisation writes), and e_ij <= E_i, the same expression with
// the per-step maxima H, C~max, Cmax, DCmax (hoisted, Sec. 3.1); both carry a
// factor 1 + 2^-10 for the rounding of their evaluation. The exact minimum is
// at most U_i = min_j (s^_j + e_ij), so the true argmin is among the
// candidates {j : s^_j - e_ij <= U_i}. A row whose only candidate is j1 is
// final; otherwise its candidates (or, past 7 of them, all k) go to the FP32
// re-check. On centroid sets of widely different norms the per-centroid terms
// keep the candidates of rows near small centroids few where E_i, set by the
// largest centroids, would flag them all. Codes may be those of x - mu and
// c - mu for a fixed centring vector mu (distances unchanged); every norm and
// residual above is then that of the centred rows, and the centring's
// rounding is inside the residual bounds the quantisation stages write.
//
// Threshold. Columns are examined only below thr = U + E_i (rounded up;
// FLT_MAX before the first), a superset of the candidates, so a 32-column block
// costs one minimum unless it holds one; an examined column gets its own e_ij,
// tightens U, and enters the row's list of 7 (ordered by lower bound) while its
// lower bound is <= U. The list's prefix with lower bound <= U at the end is the
// candidate set; a dropped entry that qualifies too sends the row to the
// all-centroid re-check. From the
// second step of a call on, rows are the points in the previous step's
// cluster-sorted order (the codes are rewritten in that order by the reduce
// stage) and a tile's chunks are visited starting with the chunk of its first
// row's previous centroid: most rows of the tile meet their nearest centroid in
// the first chunk, and the later chunks rarely hold a candidate.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_internal.cuh"
#include "km_tc.cuh"

#include <cfloat>
#include <cstring>

namespace km {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int NEPI = 8;                      // epilogue warps: two per TMEM lane quarter
constexpr int NTHREADS = 96 + 32 * NEPI;  // producer, MMA issuer 0, epilogue, MMA issuer 1
constexpr uint32_t ROWB = 128;               // bytes of one K block row
constexpr uint32_t TMEM_COLS = 512;          // 4 accumulator buffers x up to 128 columns
constexpr int NACC = 4;
constexpr int MAX_STAGES = 8;
constexpr int MAX_ABUF = 4;                  // A slots (row tiles) in the smem ring

constexpr int kT = kMaxCand - 1;  // candidate slots per row (a flag record holds up to kMaxCand)

struct Cand {
  float v;
  int i;
};

// Sorted insert into the row's candidate list (ascending score; strict
// comparisons keep the earlier, lower index first among equal scores). Written
// without branches so that the list stays in registers.
__device__ __forceinline__ void cand_insert(Cand (&top)[kT], float v, int j) {
#pragma unroll
  for (int t = kT - 1; t >= 0; --t) {
    const bool here = (t == 0) || !(v < top[t > 0 ? t - 1 : 0].v);
    if (v < top[t].v) top[t] = here ? Cand{v, j} : top[t > 0 ? t - 1 : 0];
  }
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Per-instance parameters of the tiles a role is working on: the only
// instance (single launches) or the instance that owns the current flattened
// tile (batched launches).
struct Item {
  int b;
  bool skip;        // the instance's stop rule fired
  int64_t tile0;    // first flattened tile of the instance
  int64_t tend;     // one past its last flattened tile
  int64_t n;
  int k, Kp, nkb, nchunks;
  int rowb;  // bytes of a code row of one K block (32, 64 or 128; batched instances may be narrower)
  int bn;    // centroid chunk width
  const CUtensorMap* mapX;
  const CUtensorMap* mapC;
  const float* h;
  const float* sc;
  const float4* cst;  // per-centroid error-bound terms
  const int32_t* rows;
  const float4* xs;
  const float4* xs_sorted;
  const int32_t* lab_sorted;
  const uint8_t* Cq;
  int32_t* assign;
  Ctl* ctl;
  float gam_tc;
};

template <bool BATCH>
__device__ __forceinline__ void set_instance(const TcParams& P, const CUtensorMap* mx, const CUtensorMap* mc, int b,
                                             Item& it) {
  if constexpr (!BATCH) {
    it.b = 0;
    it.tile0 = 0;
    it.tend = INT64_MAX;
    it.n = P.n_dev ? min(P.n, (int64_t)*P.n_dev) : P.n;
    it.k = P.k;
    it.Kp = P.Kp;
    it.nkb = P.nkb;
    it.nchunks = P.nchunks;
    it.rowb = (int)ROWB;
    it.bn = P.bn;
    it.mapX = mx;
    it.mapC = mc;
    it.h = P.h;
    it.sc = P.sc;
    it.cst = P.cst;
    it.rows = P.rows;
    it.xs = P.xs;
    it.xs_sorted = P.xs_sorted;
    it.lab_sorted = P.lab_sorted;
    it.Cq = P.Cq;
    it.assign = P.assign;
    it.ctl = P.ctl;
    it.gam_tc = P.gam_tc;
  } else {
    const BInst& I = P.binst[b];
    it.b = b;
    it.tile0 = I.tile_off;
    it.tend = P.btile_off[b + 1];
    it.n = I.n;
    it.k = I.k;
    it.Kp = I.Kp;
    it.nkb = I.nkb;
    it.nchunks = I.nchunks;
    it.rowb = I.rowb;
    it.bn = I.bn;
    // an instance whose tiles run in cluster-sorted order reads the sorted copy of its codes
    const bool srt = P.sorted && I.gsort;
    it.mapX = srt ? P.bmaps_s + b : P.bmaps + 2 * b;
    it.mapC = P.bmaps + 2 * b + 1;
    it.h = P.bh + I.kp_off;
    it.sc = P.bsc + I.kp_off;
    it.cst = P.bcst + I.kp_off;
    it.rows = srt ? P.bperm + I.row_off : nullptr;
    it.xs = P.bxs + I.row_off;
    it.xs_sorted = P.bxs_sorted + I.row_off;
    it.lab_sorted = P.blab_sorted + I.row_off;
    it.Cq = P.bCq + I.cq_off;
    it.assign = I.assign;
    it.ctl = P.bctls + b;
    it.gam_tc = I.gam_tc;
  }
  it.skip = it.ctl->done != 0;
}

// Tile range of this CTA: [t0, t1) with stride ts.
struct TileRange {
  int64_t t0, t1, ts;
};

template <bool BATCH>
__device__ __forceinline__ TileRange tile_range(const TcParams& P) {
  if constexpr (BATCH) return TileRange{P.bcta[blockIdx.x], P.bcta[blockIdx.x + 1], 1};
  else return TileRange{blockIdx.x, ((P.n_dev ? min(P.n, (int64_t)*P.n_dev) : P.n) + BM - 1) / BM, gridDim.x};
}

// Moves `it` to the instance of flattened tile gt (tiles are visited in
// increasing order). Returns true when the instance changed.
template <bool BATCH>
__device__ __forceinline__ bool seek(const TcParams& P, const CUtensorMap* mx, const CUtensorMap* mc, int64_t gt,
                                     Item& it) {
  if constexpr (!BATCH) {
    if (it.b >= 0) return false;
    set_instance<false>(P, mx, mc, 0, it);
    return true;
  } else {
    if (it.b >= 0 && gt < it.tend) return false;
    int b = it.b < 0 ? find_block(P.btile_off, P.nb, gt) : it.b + 1;
    while (P.btile_off[b + 1] <= gt) ++b;
    set_instance<true>(P, mx, mc, b, it);
    return true;
  }
}

template <bool BATCH>
__device__ void record_timeout(const TcParams& P) {
  if constexpr (BATCH) {
    for (int b = 0; b < P.nb; ++b) atomicExch(&P.bctls[b].error, (int)KM_ETIMEOUT);
  } else {
    atomicExch(&P.ctl->error, (int)KM_ETIMEOUT);
  }
}

// Row metadata of one tile row: the point, its norm bounds and its previous label.
struct RowMeta {
  int64_t i;
  float4 xs;
  int old;
};

template <bool BATCH>
__device__ __forceinline__ RowMeta fetch_meta(const TcParams& P, const Item& it, int64_t tile, int r) {
  RowMeta m{0, make_float4(0.f, 0.f, 0.f, 0.f), -1};
  const int64_t prow = tile * BM + r;
  if (prow < it.n) {
    if (it.rows) {  // cluster-sorted order: contiguous metadata written by the reduce stage
      m.i = __ldg(it.rows + prow);
      m.xs = __ldg(it.xs_sorted + prow);
      if (!P.first) m.old = __ldg(it.lab_sorted + prow);
    } else {
      m.i = prow;
      m.xs = __ldg(it.xs + prow);
      if (!P.first) m.old = it.assign[prow];
    }
  }
  return m;
}

// Chunk order of a tile. In cluster-sorted order the tile's rows mostly share
// the previous label of its first row; its chunks are visited starting with the
// chunk that holds that centroid, so that the first chunk already gives most
// rows a tight threshold. Any order gives the same candidates. Every role of
// the CTA derives the order from the same label.
__device__ __forceinline__ int tile_label(const TcParams& P, const Item& it, int64_t tile) {
  if (P.first || !it.rows || it.nchunks == 1) return -1;
  return __ldg(it.lab_sorted + tile * BM);
}

__device__ __forceinline__ int first_chunk(int lab, const Item& it, int bn) {
  return (lab >= 0 && lab < it.k) ? lab / bn : 0;
}

template <bool NEG>
__device__ __forceinline__ float score_of(float x) { return NEG ? -x : x; }
template <bool NEG>
__device__ __forceinline__ float score_of(uint32_t x) { return NEG ? -__uint_as_float(x) : __uint_as_float(x); }

// Per-centroid error bound of a row. Column j's computed score s^_j is within
//   e_j = (a0 h_j + a1 ||c~_j|| + a2 ||c_j|| + a3 ||c~_j - c_j||) ks
// of its exact value (the terms of E_i with the centroid's own values in place
// of the step's maxima; cst[j] holds them; ks = 1 + 2^-10 covers the rounding
// of this evaluation, times the folded E4M3 accumulator scale). U = min over
// the columns seen of s^_j + e_j bounds the row's exact minimum from above, so
// the true argmin is among {j : s^_j - e_j <= U} (its lower bound cannot exceed
// any column's upper bound). err(j) is monotone in the four terms, so
// errv(step maxima) >= e_j for every j.
struct RowErr {
  const float4* cst;
  float a0, a1, a2, a3, ks;
  float U;    // running upper bound of the row's exact minimum score
  float Lev;  // smallest lower bound dropped from a full candidate list (+inf: none)
  bool perc;  // per-centroid bounds this step (else the step maxima, candidates within the margin of the best)
  __device__ __forceinline__ float errv(float h, float q, float c, float dc) const {
    return fmaf(a0, h, fmaf(a1, q, fmaf(a2, c, a3 * dc))) * ks;
  }
  __device__ __forceinline__ float err(int j) const {
    const float4 v = __ldg(cst + j);
    return errv(v.x, v.y, v.z, v.w);
  }
};

// Folds a 32-column score block into the row's candidate list: the columns
// within min(thr, mn + margin) of the block minimum mn, in index order. With
// per-centroid bounds (a superset of the columns whose lower bound can end
// below U) each gets its own error bound e_j, tightens U, and enters the list
// (ordered by lower bound) while its lower bound is <= U; thr = U + margin / 2
// >= U + e_j for every j. Otherwise the list holds the smallest scores and thr =
// best + margin. NEG: the block holds accumulator bits whose negation is the
// score (folded BF16).
template <bool NEG = false, typename T>
__device__ __forceinline__ void fold_block(Cand (&top)[kT], const T (&s)[32], float mn, int j0, float& thr,
                                           float margin, RowErr& re) {
  const float lim = fminf(thr, __fadd_ru(mn, margin));
  unsigned mask = 0;
#pragma unroll
  for (int t = 0; t < 32; ++t) mask |= (score_of<NEG>(s[t]) <= lim ? 1u : 0u) << t;
#pragma unroll 1
  while (mask) {
    const int t = __ffs(mask) - 1;
    mask &= mask - 1;
    // s[t] through a 5-level select tree
    float x16[16], x8[8], x4[4];
#pragma unroll
    for (int u = 0; u < 16; ++u) x16[u] = (t & 1) ? score_of<NEG>(s[2 * u + 1]) : score_of<NEG>(s[2 * u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) x8[u] = (t & 2) ? x16[2 * u + 1] : x16[2 * u];
#pragma unroll
    for (int u = 0; u < 4; ++u) x4[u] = (t & 4) ? x8[2 * u + 1] : x8[2 * u];
    const float x2a = (t & 8) ? x4[1] : x4[0], x2b = (t & 8) ? x4[3] : x4[2];
    const float v = (t & 16) ? x2b : x2a;
    if (v <= thr && !re.perc) {
      cand_insert(top, v, j0 + t);
      thr = fminf(thr, __fadd_ru(top[0].v, margin));
    } else if (v <= thr) {
      const float ej = re.err(j0 + t);
      re.U = fminf(re.U, __fadd_ru(v, ej));
      thr = fminf(thr, __fadd_ru(re.U, 0.5f * margin));
      const float lo = __fsub_rd(v, ej);
      if (lo <= re.U) {
        const float last = top[kT - 1].v;  // dropped when the list is full (+inf: it has room)
        if (lo < last) {
          re.Lev = fminf(re.Lev, last);
          cand_insert(top, lo, j0 + t);
        } else {
          re.Lev = fminf(re.Lev, lo);
        }
      }
    }
  }
}

// Scores of one 32-column block from its TMEM accumulators,
// s_j = h_j + w acc_j with the row's factor w = -(sx sc) (two columns per
// packed operation), their minimum, and the fold of the block's candidates
// (rare once thr is tight).
__device__ __forceinline__ void score_block(const uint32_t (&v)[32], const float* hb, float w, Cand (&top)[kT],
                                            int j0, float& thr, float margin, RowErr& re) {
  float s[32];
  const float4* h4 = reinterpret_cast<const float4*>(hb);
  const float2 w2 = make_float2(w, w);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const float4 hh = h4[t];
    const float2 a0 = make_float2(__uint_as_float(v[4 * t]), __uint_as_float(v[4 * t + 1]));
    const float2 a1 = make_float2(__uint_as_float(v[4 * t + 2]), __uint_as_float(v[4 * t + 3]));
    const float2 s0 = __ffma2_rn(w2, a0, make_float2(hh.x, hh.y));
    const float2 s1 = __ffma2_rn(w2, a1, make_float2(hh.z, hh.w));
    s[4 * t] = s0.x;
    s[4 * t + 1] = s0.y;
    s[4 * t + 2] = s1.x;
    s[4 * t + 3] = s1.y;
  }
  // block minimum by a 4-level tree of 3-input minima
  float m11[11];
#pragma unroll
  for (int u = 0; u < 10; ++u) m11[u] = min3f(s[3 * u], s[3 * u + 1], s[3 * u + 2]);
  m11[10] = fminf(s[30], s[31]);
  const float mn = fminf(min3f(min3f(m11[0], m11[1], m11[2]), min3f(m11[3], m11[4], m11[5]),
                               min3f(m11[6], m11[7], m11[8])),
                         fminf(m11[9], m11[10]));
  if (__any_sync(0xffffffffu, mn <= thr))
    if (mn <= thr) fold_block(top, s, mn, j0, thr, margin, re);
}

// Two consecutive 32-column blocks: both score sets, one vote on the smaller
// block minimum, then the folds in column order (the first may tighten thr).
__device__ __forceinline__ void score_block2(const uint32_t (&v)[32], const uint32_t (&v2)[32], const float* hb,
                                             float w, Cand (&top)[kT], int j0, float& thr, float margin, RowErr& re) {
  float s[32], s2[32];
  const float4* h4 = reinterpret_cast<const float4*>(hb);
  const float2 w2 = make_float2(w, w);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const float4 hh = h4[t], hg = h4[t + 8];
    const float2 a0 = make_float2(__uint_as_float(v[4 * t]), __uint_as_float(v[4 * t + 1]));
    const float2 a1 = make_float2(__uint_as_float(v[4 * t + 2]), __uint_as_float(v[4 * t + 3]));
    const float2 c0 = make_float2(__uint_as_float(v2[4 * t]), __uint_as_float(v2[4 * t + 1]));
    const float2 c1 = make_float2(__uint_as_float(v2[4 * t + 2]), __uint_as_float(v2[4 * t + 3]));
    const float2 s0 = __ffma2_rn(w2, a0, make_float2(hh.x, hh.y));
    const float2 s1 = __ffma2_rn(w2, a1, make_float2(hh.z, hh.w));
    const float2 t0 = __ffma2_rn(w2, c0, make_float2(hg.x, hg.y));
    const float2 t1 = __ffma2_rn(w2, c1, make_float2(hg.z, hg.w));
    s[4 * t] = s0.x;
    s[4 * t + 1] = s0.y;
    s[4 * t + 2] = s1.x;
    s[4 * t + 3] = s1.y;
    s2[4 * t] = t0.x;
    s2[4 * t + 1] = t0.y;
    s2[4 * t + 2] = t1.x;
    s2[4 * t + 3] = t1.y;
  }
  float m11[11], n11[11];
#pragma unroll
  for (int u = 0; u < 10; ++u) {
    m11[u] = min3f(s[3 * u], s[3 * u + 1], s[3 * u + 2]);
    n11[u] = min3f(s2[3 * u], s2[3 * u + 1], s2[3 * u + 2]);
  }
  m11[10] = fminf(s[30], s[31]);
  n11[10] = fminf(s2[30], s2[31]);
  const float mn = fminf(min3f(min3f(m11[0], m11[1], m11[2]), min3f(m11[3], m11[4], m11[5]),
                               min3f(m11[6], m11[7], m11[8])),
                         fminf(m11[9], m11[10]));
  const float mn2 = fminf(min3f(min3f(n11[0], n11[1], n11[2]), min3f(n11[3], n11[4], n11[5]),
                                min3f(n11[6], n11[7], n11[8])),
                          fminf(n11[9], n11[10]));
  if (__any_sync(0xffffffffu, fminf(mn, mn2) <= thr)) {
    // no candidate lies above the pair's minimum + margin (the row's best is at most that minimum),
    // so a block whose minimum is above it needs no fold
    thr = fminf(thr, __fadd_ru(fminf(mn, mn2), margin));
    if (mn <= thr) fold_block(top, s, mn, j0, thr, margin, re);
    if (mn2 <= thr) fold_block(top, s2, mn2, j0 + 32, thr, margin, re);
  }
}

// Folded BF16 (the accumulators hold acc_j = x.c_j - h_j, the score is -acc_j):
// the block minimum of the scores is minus the maximum of the accumulators, so
// a 64-column half costs two trees of 3-input maxima and a vote.
__device__ __forceinline__ void score_block2_fold(const uint32_t (&v)[32], const uint32_t (&v2)[32], Cand (&top)[kT],
                                                  int j0, float& thr, float margin, RowErr& re) {
  float m11[11], n11[11];
#pragma unroll
  for (int u = 0; u < 10; ++u) {
    m11[u] = max3f(__uint_as_float(v[3 * u]), __uint_as_float(v[3 * u + 1]), __uint_as_float(v[3 * u + 2]));
    n11[u] = max3f(__uint_as_float(v2[3 * u]), __uint_as_float(v2[3 * u + 1]), __uint_as_float(v2[3 * u + 2]));
  }
  m11[10] = fmaxf(__uint_as_float(v[30]), __uint_as_float(v[31]));
  n11[10] = fmaxf(__uint_as_float(v2[30]), __uint_as_float(v2[31]));
  const float mn = -fmaxf(max3f(max3f(m11[0], m11[1], m11[2]), max3f(m11[3], m11[4], m11[5]),
                                max3f(m11[6], m11[7], m11[8])),
                          fmaxf(m11[9], m11[10]));
  const float mn2 = -fmaxf(max3f(max3f(n11[0], n11[1], n11[2]), max3f(n11[3], n11[4], n11[5]),
                                 max3f(n11[6], n11[7], n11[8])),
                           fmaxf(n11[9], n11[10]));
  if (__any_sync(0xffffffffu, fminf(mn, mn2) <= thr)) {
    thr = fminf(thr, __fadd_ru(fminf(mn, mn2), margin));  // (as in score_block2)
    if (mn <= thr) fold_block<true>(top, v, mn, j0, thr, margin, re);
    if (mn2 <= thr) fold_block<true>(top, v2, mn2, j0 + 32, thr, margin, re);
  }
}

// The constant A operand of the folded -h_j slice: 128 rows of 16 BF16
// [1, 1, 1, 0, ...] in the 32-byte swizzled K-major layout (row r at byte
// 32 r, its 16-byte chunk c at chunk c ^ ((r >> 2) & 1)), one K = 16 MMA step.
constexpr uint32_t HROWB = 32;  // bytes of one row of the -h_j slice
__device__ __forceinline__ void fill_ones_block(uint8_t* blk) {
  for (int e = threadIdx.x; e < BM * 2; e += blockDim.x) {
    const int r = e >> 1, c = e & 1;
    const uint4 ones = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);  // BF16 1.0, 1.0, 1.0, 0, 0, ...
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(blk + r * HROWB + ((c ^ ((r >> 2) & 1)) << 4)) = c == 0 ? ones : zero;
  }
}

template <int FP8, bool BATCH, bool FOLD>
__global__ void __launch_bounds__(NTHREADS, 1)
assign_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC,
                 const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapXh,
                 const TcParams P) {
  constexpr int KBE = ROWB / (FP8 ? 1 : 2);  // elements per 128-byte K block
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned by an offset into the shared array (not an integer round trip), so that
  // accesses through derived pointers (h_j in the epilogue) compile to shared-memory loads
  uint8_t* smem = smem_raw + ((1024u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t a_full[MAX_ABUF], a_empty[MAX_ABUF], b_full[MAX_STAGES], b_empty[MAX_STAGES];
  __shared__ uint64_t acc_full[NACC], acc_empty[NACC], drain_bar, drain_bar1, never_bar;
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
  constexpr bool AXS = FP8 && FOLD;                          // A slots carry each row's 1/s_x slice
  const uint32_t a_bytes = (uint32_t)P.nkb * BM * ROWB + (AXS ? BM * HROWB : 0);  // one A slot
  const uint32_t b_kblk = (uint32_t)BN * ROWB;               // one K block of a B stage
  const uint32_t b_bytes = (uint32_t)P.nkb * b_kblk + (FOLD ? BN * HROWB : 0);  // one B stage (+ -h_j slice)
  const int nab = P.abufs;                                    // A slots (ring)
  const bool pairs = nab >= 2;                                // two row tiles per B chunk
  uint8_t* A0 = smem;
  uint8_t* B0 = smem + nab * a_bytes;
  const int kpmax = P.nchunks * BN;
  uint8_t* Aex = B0 + (size_t)stages * b_bytes;                         // folded BF16: the constant ones slice
  float* Hs = reinterpret_cast<float*>(Aex + (FOLD && !FP8 ? BM * HROWB : 0));  // [kpmax] (unfolded launches)
  const TileRange tr = tile_range<BATCH>(P);

  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int b = 0; b < nab; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1);  // the MMA commit after the tile's last chunk
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], NEPI / 2);  // the four warps of the buffer's group
    }
    for (int s = 0; s < stages; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], pairs ? 2 : 1);  // one commit per MMA issuer
    }
    mbar_init(&drain_bar, 1);
    mbar_init(&drain_bar1, 1);
    mbar_init(&never_bar, 1);  // nothing ever arrives: the timeout test waits on it
    fence_mbar_init();
  }
  if (!BATCH && warp == 0 && lane == 0) {
    prefetch_tensormap(&mapX);
    prefetch_tensormap(&mapC);
    if (FOLD) prefetch_tensormap(&mapH);
    if (AXS) prefetch_tensormap(&mapXh);
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_s, TMEM_COLS);
    tmem_relinquish();
  }
  if (!BATCH && !FOLD && warp >= 2 && warp < 2 + NEPI) {  // batched launches stage h per instance in the epilogue
    for (int j = threadIdx.x - 64; j < kpmax; j += 32 * NEPI) Hs[j] = __ldg(P.h + j);
  }
  if (FOLD && !FP8) {  // generic-proxy writes the MMA (async proxy) reads after the barrier
    fill_ones_block(Aex);
    fence_proxy_async_smem();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem_base = tmem_base_s;

  // Every role walks the same sequence of tile pairs: the CTA's tiles in order,
  // two consecutive ones of the same instance at a time (one when the next
  // tile is absent or belongs to another instance). Tile u of a pair is read
  // by epilogue group u; its accumulators are TMEM buffers u and u + 2.
  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      int lt = 0, gc = 0;              // tiles and chunks loaded so far by this CTA
      int last_a = -1, last_s = -1;    // barrier slots of the most recent A and B loads
      uint32_t last_aph = 0, last_sph = 0;
      bool ok = true;
      Item it;
      it.b = -1;
      int labn = -2;                   // label of the next pair's first row, loaded a pair ahead (-2: not loaded)
      int ab = 0, sb = 0;              // next A slot and B stage (lt % nab, gc % stages, kept incrementally)
      uint32_t aph = 0, sph = 0;       // and their phase bits ((lt / nab) & 1, (gc / stages) & 1)
      for (int64_t ga = tr.t0; ga < tr.t1 && ok;) {
        if (seek<BATCH>(P, &mapX, &mapC, ga, it)) {
          labn = -2;
          if (BATCH && !it.skip) {
            // tensor maps in global memory: order the host's writes before the async proxy reads them
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(it.mapX) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(it.mapC) : "memory");
          }
        }
        if (it.skip) {
          ga += tr.ts;
          continue;
        }
        const int64_t gb = ga + tr.ts;
        const int ntp = (pairs && gb < tr.t1 && gb < it.tend) ? 2 : 1;
        const int64_t tile0 = ga - it.tile0;
        const int c0 = first_chunk(labn != -2 ? labn : tile_label(P, it, tile0), it, it.bn);
        {
          const int64_t gn = ntp == 2 ? gb + tr.ts : gb;
          labn = (gn < tr.t1 && gn < it.tend) ? tile_label(P, it, gn - it.tile0) : -2;
        }
        for (int u = 0; u < ntp && ok; ++u, ++lt) {
          if (!mbar_wait(&a_empty[ab], aph ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          const uint32_t rowb = BATCH ? (uint32_t)it.rowb : ROWB;  // (narrower rows come as one K block: x = 0)
          mbar_arrive_expect_tx(&a_full[ab], (uint32_t)it.nkb * BM * rowb + (AXS ? BM * HROWB : 0u));
          const int row0 = (int)((u ? gb - it.tile0 : tile0) * BM);
          for (int kb = 0; kb < it.nkb; ++kb)
            tma_load_2d(A0 + ab * a_bytes + kb * (BM * rowb), it.mapX, &a_full[ab], kb * KBE, row0);
          if (AXS) tma_load_2d(A0 + ab * a_bytes + it.nkb * (BM * ROWB), &mapXh, &a_full[ab], 0, row0);
          last_a = ab;
          last_aph = aph;
          if (++ab == nab) {
            ab = 0;
            aph ^= 1;
          }
        }
        for (int cc = 0, c = c0; cc < it.nchunks && ok; ++cc, ++gc, c = (c + 1 == it.nchunks) ? 0 : c + 1) {
          const int s = sb;
          if (!mbar_wait(&b_empty[s], sph ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
          mbar_arrive_expect_tx(&b_full[s], (BATCH ? (uint32_t)(it.nkb * it.bn * it.rowb) : (uint32_t)it.nkb * b_kblk) +
                                                (FOLD ? BN * HROWB : 0u));
          for (int kb = 0; kb < it.nkb; ++kb)
            tma_load_2d(B0 + s * b_bytes + kb * b_kblk, it.mapC, &b_full[s], kb * KBE, c * (BATCH ? it.bn : BN));
          if (FOLD) tma_load_2d(B0 + s * b_bytes + it.nkb * b_kblk, &mapH, &b_full[s], 0, c * BN);
          last_s = s;
          last_sph = sph;
          if (++sb == stages) {
            sb = 0;
            sph ^= 1;
          }
        }
        ga = ntp == 2 ? gb + tr.ts : gb;
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
  } else if (warp == 1 || warp == 2 + NEPI) {
    // ---------------------------------------------------------------- MMA issuers
    // Two issuers, each one thread: issuer me (warp 1, or the warp after the epilogue) issues the
    // MMAs of tile u = me of every pair, so that the two tiles' instruction streams run side by
    // side (one issuing thread was the limiter); both walk every chunk and each commits the B stage.
    const int me = warp == 1 ? 0 : 1;
    if (lane == 0 && (me == 0 || pairs)) {
      int lt = 0;
      int gu = 0;          // chunks issued for this issuer's epilogue group
      int sb = 0;          // B stage and its phase, kept incrementally
      uint32_t sph = 0;
      bool ok = true, issued = false;
      const bool split = !BATCH && !FP8 && P.split;
      Item it;
      it.b = -1;
      for (int64_t ga = tr.t0; ga < tr.t1 && ok;) {
        seek<BATCH>(P, &mapX, &mapC, ga, it);
        if (it.skip) {
          ga += tr.ts;
          continue;
        }
        const int64_t gb = ga + tr.ts;
        const int ntp = (pairs && gb < tr.t1 && gb < it.tend) ? 2 : 1;
        const bool mine = me < ntp;
        const int ab = (lt + me) % nab;
        if (mine && !mbar_wait(&a_full[ab], ((lt + me) / nab) & 1, &abort_s, P.wait_ns)) { ok = false; break; }
        tc_fence_after_sync();
        for (int cc = 0; cc < it.nchunks && ok; ++cc) {
          const int s = sb;
          if (!mbar_wait(&b_full[s], sph, &abort_s, P.wait_ns)) { ok = false; break; }
          if (++sb == stages) {
            sb = 0;
            sph ^= 1;
          }
          tc_fence_after_sync();
          if (mine) {
            const uint32_t b_addr = smem_u32(B0 + s * b_bytes);
            const int buf = 2 * (gu & 1) + me;
            if (!mbar_wait(&acc_empty[buf], ((gu >> 1) & 1) ^ 1, &abort_s, P.wait_ns)) { ok = false; break; }
            tc_fence_after_sync();
            const uint32_t a_addr = smem_u32(A0 + ab * a_bytes);
            const uint32_t d_tmem = tmem_base + (uint32_t)(buf * 128);
            const uint64_t a_desc = BATCH ? sdesc_k(a_addr, (uint32_t)it.rowb) : sdesc_k_sw128(a_addr);
            const uint64_t b_desc = BATCH ? sdesc_k(b_addr, (uint32_t)it.rowb) : sdesc_k_sw128(b_addr);
            // a batched instance's N is its own chunk width
            const uint32_t idesc = BATCH ? ((P.idesc & ~(0x3Fu << 17)) | ((uint32_t)(it.bn >> 3) << 17)) : P.idesc;
            const int ksteps = BATCH ? it.rowb >> 5 : 4;  // 32-byte MMA steps per K block row
            const int mk = split ? it.nkb >> 1 : it.nkb;
            for (int seg = 0; seg < (split ? 3 : 1); ++seg) {
              const int ka = seg == 1 ? mk : 0, kc = seg == 2 ? mk : 0;
              for (int kb = 0; kb < mk; ++kb) {
                const uint64_t a_kb = a_desc + (uint64_t)(((ka + kb) * (BM * (BATCH ? (uint32_t)it.rowb : ROWB))) >> 4);
                const uint64_t b_kb = b_desc + (uint64_t)(((kc + kb) * b_kblk) >> 4);
#pragma unroll
                for (int kk = 0; kk < (BATCH ? ksteps : 4); ++kk) {
                  const uint64_t ad = a_kb + (uint64_t)(kk * 2);  // + 32 bytes
                  const uint64_t bd = b_kb + (uint64_t)(kk * 2);
                  if constexpr (FP8) mma_fp8(d_tmem, ad, bd, idesc, (seg | kb | kk) != 0);
                  else mma_bf16(d_tmem, ad, bd, idesc, (seg | kb | kk) != 0);
                }
              }
            }
            if constexpr (FOLD) {  // + [r, r, r, 0, ...] . [-h1, -h2, -h3, 0, ...]: one BF16 K = 16 step (r = 1, or
                                   // 1 / s_x of the row for E4M3, whose accumulator it adds to)
              const uint32_t ax = AXS ? a_addr + (uint32_t)it.nkb * (BM * ROWB) : smem_u32(Aex);
              mma_bf16(d_tmem, sdesc_k_sw32(ax), sdesc_k_sw32(b_addr + it.nkb * b_kblk), AXS ? P.idesc16 : P.idesc, 1u);
            }
            issued = true;
            mma_commit(&acc_full[buf]);
            ++gu;
          }
          mma_commit(&b_empty[s]);
        }
        if (ok && mine) mma_commit(&a_empty[ab]);
        lt += ntp;
        ga = ntp == 2 ? gb + tr.ts : gb;
      }
      if (!ok) {
        abort_s = 1;
        record_timeout<BATCH>(P);
      }
      if (issued) {  // every MMA this thread issued has completed once its drain barrier flips
        uint64_t* db = me ? &drain_bar1 : &drain_bar;
        mma_commit(db);
        int dummy = 0;
        mbar_wait(db, 0, &dummy, P.wait_ns);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..9)
    const int q = warp & 3;                // TMEM lane quarter this warp may access
    const int grp = (warp - 2) >> 2;       // epilogue group: tile u = grp of each pair
    const int r = q * 32 + lane;           // row of the tile this thread owns
    int gu = 0;                            // chunks of this group consumed so far
    bool ok = true;
    unsigned int changed = 0;
    Item it;
    it.b = -1;
    float H = 0.f, Cmax = 0.f, QCmax = 0.f, DCmax = 0.f;  // per-step maxima of the instance
    bool perc = false;                                    // per-centroid error bounds this step
    float csc = 1.f;                                      // the instance's centroid code scale (E4M3)
    RowMeta nxt;
    bool have_nxt = false;
    int labn = -2;  // label of the next pair's first row, loaded a pair ahead (-2: not loaded)
    // Every epilogue warp walks every pair to the end, even after a timeout
    // (then skipping waits and work), so that all of them reach the named
    // barrier of the batched h staging the same number of times.
    for (int64_t ga = tr.t0; ga < tr.t1;) {
      if (seek<BATCH>(P, &mapX, &mapC, ga, it)) {
        have_nxt = false;
        labn = -2;
        if (BATCH && !it.skip) {
          // this instance's h_j (and scales) into shared memory
          asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
          for (int j = threadIdx.x - 64; j < it.nchunks * it.bn; j += 32 * NEPI) Hs[j] = __ldg(it.h + j);
          asm volatile("bar.sync 1, %0;" ::"n"(32 * NEPI) : "memory");
        }
        if (!it.skip) {
          const Ctl* ctl = it.ctl;
          H = __uint_as_float(ctl->hmax_c_bits);  // (the centred centroids' maxima)
          // per-centroid bounds pay when the centroids' h_j spread over more than a factor 64 (norms 8):
          // below that their candidate-by-candidate evaluation costs more than the re-checks it saves
          perc = H > 64.f * __uint_as_float(0x7f800000u - ctl->hmin_neg);
          Cmax = __uint_as_float(ctl->cmax_c_bits);
          QCmax = __uint_as_float(!BATCH && P.stats16 ? ctl->qcmax16_bits : ctl->qcmax_bits);
          DCmax = __uint_as_float(!BATCH && P.stats16 ? ctl->dcmax16_bits : ctl->dcmax_bits);
          if (FP8) csc = __ldg(it.sc);  // the same for every centroid of the step
        }
      }
      if (it.skip) {
        ga += tr.ts;
        continue;
      }
      const int64_t gb = ga + tr.ts;
      const int ntp = (pairs && gb < tr.t1 && gb < it.tend) ? 2 : 1;
      const int64_t ga_next = ntp == 2 ? gb + tr.ts : gb;
      const int64_t tile0 = ga - it.tile0;
      const int lab = labn != -2 ? labn : tile_label(P, it, tile0);
      labn = (ga_next < tr.t1 && ga_next < it.tend) ? tile_label(P, it, ga_next - it.tile0) : -2;
      if (grp >= ntp) {  // no tile for this group in this pair
        ga = ga_next;
        continue;
      }
      const int64_t tile = grp ? gb - it.tile0 : tile0;
      const int c0 = first_chunk(lab, it, it.bn);
      const int nblk = it.bn / 32;  // 32-column blocks per chunk
      const RowMeta m = have_nxt ? nxt : fetch_meta<BATCH>(P, it, tile, r);
      // this group's tile of the next pair, when it belongs to the same instance: its loads overlap this tile
      {
        const int64_t na = ga_next, nb2 = ga_next + tr.ts;
        const int64_t ntile = grp ? nb2 : na;
        have_nxt = na < tr.t1 && na < it.tend && ntile < tr.t1 && ntile < it.tend &&
                   (grp == 0 || (pairs && nb2 < tr.t1 && nb2 < it.tend));
        if (have_nxt) nxt = fetch_meta<BATCH>(P, it, ntile - it.tile0, r);
      }
      const bool valid = tile * BM + r < it.n;
      const int64_t i = m.i;
      const float4 xs = m.xs;
      int old = m.old;
      if (old < 0 || old >= it.k) old = -1;
      // per-row error bounds: each centroid's own (candidates), and the step maxima's (margin / 2 >= e_j
      // for every j; folded E4M3 launches compare accumulators, scores / (s_x s_c), an exact power of two)
      RowErr re;
      re.cst = BATCH ? it.cst : P.cst;  // (single launches: read from the parameter space)
      re.a0 = BATCH ? 3.f * kU : P.hcoef;
      re.a1 = (it.gam_tc + 2.f * kU) * xs.y;
      re.a2 = xs.z;
      re.a3 = xs.w + xs.z;
      re.ks = (1.f + 0x1p-10f) * (FP8 && FOLD ? __frcp_rn(xs.x * csc) : 1.f);
      re.U = INFINITY;
      re.Lev = INFINITY;
      re.perc = perc;
      const float margin = 2.f * re.errv(H, QCmax, Cmax, DCmax);
      float thr = FLT_MAX;  // finite: padding columns (score +inf) never become candidates
      if (ok && P.debug_stall && !__all_sync(0xffffffffu, mbar_wait(&never_bar, 0, &abort_s, P.wait_ns))) ok = false;

      Cand top[kT];
#pragma unroll
      for (int t = 0; t < kT; ++t) top[t] = Cand{INFINITY, -1};
      const float wrow = FP8 ? -xs.x * csc : -1.f;  // exact: a product of powers of two
      const uint32_t trow = tmem_base + ((uint32_t)(q * 32) << 16);
      // the tile's 32-column blocks in chunk order
      const int nall = it.nchunks * nblk;
      uint32_t v[32], v2[32];
      int c = c0;
      if (!BATCH && BN == 128) {
        // 128-column chunks in straight-line code: two 64-column halves, each two TMEM loads and
        // one wait; the buffer is released once the second half is in registers
#pragma unroll 1
        for (int cc = 0; cc < it.nchunks && ok; ++cc) {
          const int buf = 2 * (gu & 1) + grp;
          if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (gu >> 1) & 1, &abort_s, P.wait_ns))) {
            ok = false;
            break;
          }
          tc_fence_after_sync();
          const uint32_t ta = trow + (uint32_t)(buf * 128);
          const int j0 = c * 128;
          tmem_ld_32x32b_x32(ta, v);
          tmem_ld_32x32b_x32(ta + 32u, v2);
          tmem_ld_wait();
          if constexpr (FOLD) score_block2_fold(v, v2, top, j0, thr, margin, re);
          else score_block2(v, v2, Hs + j0, wrow, top, j0, thr, margin, re);
          tmem_ld_32x32b_x32(ta + 64u, v);
          tmem_ld_32x32b_x32(ta + 96u, v2);
          tmem_ld_wait();
          tc_fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
          if constexpr (FOLD) score_block2_fold(v, v2, top, j0 + 64, thr, margin, re);
          else score_block2(v, v2, Hs + j0 + 64, wrow, top, j0 + 64, thr, margin, re);
          ++gu;
          c = (c + 1 == it.nchunks) ? 0 : c + 1;
        }
      }
      int blk = 0;  // 32-column block within the current chunk
#pragma unroll 1
      for (int kb = (!BATCH && BN == 128) ? nall : 0; kb < nall && ok;) {
        const int buf = 2 * (gu & 1) + grp;
        if (blk == 0) {  // a new chunk: wait for its accumulators
          if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[buf], (gu >> 1) & 1, &abort_s, P.wait_ns))) {
            ok = false;
            break;
          }
          tc_fence_after_sync();
        }
        // two blocks of this chunk per load and vote (single launches: the batched kernel keeps one,
        // for registers)
        const bool two = !BATCH && blk + 1 < nblk;
        tmem_ld_32x32b_x32(trow + (uint32_t)(buf * 128 + blk * 32), v);
        if (two) tmem_ld_32x32b_x32(trow + (uint32_t)(buf * 128 + blk * 32 + 32), v2);
        tmem_ld_wait();
        const int lastb = two ? blk + 1 : blk;
        if (lastb == nblk - 1) {  // the chunk's accumulators are all in registers: release the buffer
          tc_fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
        const int j0 = c * it.bn + blk * 32;
        if (two) score_block2(v, v2, Hs + j0, wrow, top, j0, thr, margin, re);
        else score_block(v, Hs + j0, wrow, top, j0, thr, margin, re);
        kb += two ? 2 : 1;
        blk = lastb + 1;
        if (lastb == nblk - 1) {
          blk = 0;
          ++gu;
          c = (c + 1 == it.nchunks) ? 0 : c + 1;
        }
      }
      {  // warp-uniform: the flag slots are reserved once per warp
        const bool live = ok && valid;
        int nc = -1;  // -1: final; 0: all k; >0: candidate count
        if (live && perc) {
          // the candidates: the list's prefix with lower bound <= U (ordered by lower bound); a
          // dropped entry that qualifies too means the list cannot hold them all
          int cnt = 0;
#pragma unroll
          for (int t = 0; t < kT; ++t) cnt += (top[t].i >= 0 && top[t].v <= re.U) ? 1 : 0;
          if (cnt == 0 || re.Lev <= re.U) nc = 0;
          else if (cnt > 1) nc = cnt;
        } else if (live) {  // the scores within the margin of the best
          if (top[0].i < 0) {
            nc = 0;
          } else {
            int cnt = 1;
#pragma unroll
            for (int t = 1; t < kT; ++t) cnt += (top[t].i >= 0 && __fsub_rn(top[t].v, top[0].v) <= margin) ? 1 : 0;
            if (cnt == kT) nc = 0;  // maybe more than kT within the margin
            else if (cnt > 1) nc = cnt;
          }
        }
        const bool flag = live && nc >= 0;
        const unsigned fm = __ballot_sync(0xffffffffu, flag);
        unsigned long long slot = 0;
        if (fm) {
          const unsigned fullm = __ballot_sync(0xffffffffu, flag && nc == 0);
          const int leader = __ffs(fm) - 1;
          if (lane == leader) {
            slot = atomicAdd(P.flag_slots, (unsigned long long)__popc(fm));
            if (BATCH) atomicAdd(&it.ctl->n_flagged, (unsigned long long)__popc(fm));
            if (fullm && (BATCH || !P.n_dev))  // a re-check pass does not count its points again
              atomicAdd(&it.ctl->n_full, (unsigned long long)__popc(fullm));
          }
          slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(fm & ((1u << lane) - 1u));
        }
        if (live && !flag) {
          it.assign[i] = top[0].i;
          changed += (old != top[0].i);
        } else if (flag) {
          FlagRec rec;
          rec.i = (int32_t)i;
          rec.old = old;
          rec.nc = nc;
          rec.pad = it.b;
          // the candidates: the list's first nc entries, in list order (the
          // re-check gives exact ties to the lowest index itself)
#pragma unroll
          for (int a = 0; a < kT; ++a) rec.cand[a] = (a < nc) ? top[a].i : 0;
#pragma unroll
          for (int a = kT; a < kMaxCand; ++a) rec.cand[a] = 0;
          if (slot < (unsigned long long)P.flag_cap) P.flags[slot] = rec;
          it.assign[i] = top[0].i >= 0 ? top[0].i : 0;
        }
      }
      if (BATCH && changed && (ga_next >= it.tend || ga_next >= tr.t1)) {
        atomicAdd(&it.ctl->n_changed, (unsigned long long)changed);  // leaving this instance
        changed = 0;
      }
      ga = ga_next;
    }
    if (!ok) {
      abort_s = 1;
      record_timeout<BATCH>(P);
    }
    if (!BATCH && changed) atomicAdd(&P.ctl->n_changed, (unsigned long long)changed);
  }

  tc_fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after_sync();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace

size_t tc_smem_bytes(int nkb, int bn, int stages, int kp, int fp8, int abufs, int fold) {
  const size_t a_slot = (size_t)nkb * BM * ROWB + (fp8 && fold ? (size_t)BM * HROWB : 0);
  return 1024 + (size_t)abufs * a_slot + (size_t)stages * (nkb * bn * ROWB + fold * bn * HROWB) +
         (fold ? (fp8 ? 0 : (size_t)BM * HROWB) : (size_t)kp * 4);
}

// A slots and B stages that fit the shared memory: the most A slots (up to 4,
// so that the next tile pair's A tiles load while a pair is scored) that leave
// at least three B stages; failing that two A slots and at least two stages;
// failing that one slot. Returns the number of B stages (< 2: does not fit).
int tc_pick_buffers(int nkb, int bn, int kp, int fp8, int* abufs, int fold) {
  const size_t budget = 227 * 1024 - 1024, b = (size_t)nkb * bn * ROWB + (size_t)fold * bn * HROWB;
  auto stages_for = [&](int na) -> int {
    const size_t fixed = tc_smem_bytes(nkb, bn, 0, kp, fp8, na, fold);
    return fixed + 2 * b <= budget ? (int)std::min<size_t>(MAX_STAGES, (budget - fixed) / b) : 0;
  };
  for (int na = MAX_ABUF; na >= 3; --na)
    if (stages_for(na) >= 3) {
      *abufs = na;
      return stages_for(na);
    }
  for (int na = 2; na >= 1; --na)
    if (stages_for(na) >= 2) {
      *abufs = na;
      return stages_for(na);
    }
  *abufs = 1;
  return 0;
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
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<0, false, false>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<0, false, true>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<1, false, false>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<1, false, true>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<0, true, false>, optin);
  if (e == cudaSuccess) e = raise_smem(assign_tc_kernel<1, true, false>, optin);
  return e;
}

cudaError_t launch_assign_tc(const Problem& p, const TcLaunch& L, const TcParams& P, cudaStream_t s) {
  const int64_t tiles = (p.n + BM - 1) / BM;
  const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
  const size_t smem = tc_smem_bytes(P.nkb, P.bn, P.stages, P.nchunks * P.bn, L.fp8, P.abufs, P.fold);
  if (L.fp8 && P.fold)
    assign_tc_kernel<1, false, true><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, L.mapH, L.mapXh, P);
  else if (L.fp8)
    assign_tc_kernel<1, false, false><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, L.mapH, L.mapXh, P);
  else if (P.fold)
    assign_tc_kernel<0, false, true><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, L.mapH, L.mapXh, P);
  else
    assign_tc_kernel<0, false, false><<<grid, NTHREADS, smem, s>>>(L.mapX, L.mapC, L.mapH, L.mapXh, P);
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
  P.nchunks = (kp_max + bn - 1) / bn;
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
  P.bcta = W.cta_tile;
  P.nb = W.nb;
  P.sorted = sorted;
  P.ntiles = W.T;
  P.bctls = W.ctls;
  P.bmaps = W.maps;
  P.bmaps_s = W.maps_s;
  P.bh = W.hq;
  P.bsc = W.scq;
  P.bcst = W.cst;
  P.bCq = W.Cq;
  P.bxs = W.xs;
  P.bxs_sorted = W.xs_sorted;
  P.blab_sorted = W.lab_sorted;
  P.bperm = W.perm;
  const int grid = W.cta_grid;
  const size_t smem = tc_smem_bytes(nkb_max, bn, stages, kp_max, fp8, abufs);
  CUtensorMap dummy;
  memset(&dummy, 0, sizeof dummy);
  if (fp8) assign_tc_kernel<1, true, false><<<grid, NTHREADS, smem, s>>>(dummy, dummy, dummy, dummy, P);
  else assign_tc_kernel<0, true, false><<<grid, NTHREADS, smem, s>>>(dummy, dummy, dummy, dummy, P);
  return cudaGetLastError();
}

}  // namespace km
