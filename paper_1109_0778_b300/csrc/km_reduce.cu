// Keyed reduce of the Lloyd step (DeliteReduceElem keyed by cluster, Sec. 2.4)
// and the per-cluster divide avg = sum / length (Sec. 2.1).
//
// The sums are formed by a counting sort of the point indices by cluster
// followed by a segmented sum over the sorted order:
//   count   -- counts_j = |{i : a_i = j}| (shared-memory histogram when k is
//              small enough, else global atomics), exact integers;
//   scan    -- segment starts offs_j = sum_{j' < j} counts_j';
//   scatter -- perm[offs_j + r] = i and slab[offs_j + r] = j for the r-th
//              member found (cursors reserved once per block and cluster for
//              k <= 8192, else warp-aggregated; order within a segment
//              unspecified);
//   segsum  -- each warp walks one contiguous range of sorted positions; the
//              rows are gathered into shared memory with cp.async, one batch
//              ahead of the batch being summed. While the cluster stays the
//              same the warp Kahan-accumulates the rows in FP32 registers, and
//              on every cluster change it flushes its partial into an FP64 sum
//              (one atomic add per coordinate). The objective term
//              ||x_i - c_{a_i}||^2 is formed in the same pass from the
//              centroid held in registers for the segment.
// Error: a Kahan-summed run of m rows carries <= 2u + O(m u^2) of the summed
// magnitudes, and the FP64 combine adds ~2^-53 per partial, so every sum is
// within ~1.2e-7 of sum |x_it| regardless of cluster size or order, far
// inside the 1e-5 centroid tolerance.
//
// Deterministic mode (DET): the same passes, but every coordinate of a row is
// split into three integer parts on the grid of 2^E >= max_i ||x_i||
// (fx_add), summed in 32-bit integers per run (at most 1024 rows, |sum| <=
// 2^30) and added into 64-bit integer accumulators; the objective terms of a
// lane likewise on the grid of (max ||x|| + max ||c||)^2. Integer sums do not
// depend on the order of the additions, so sums, centroids and the objective
// come out bit-identical run after run; the divide forms each FP64 sum from
// its three integers in a fixed order. Dropped per point and coordinate:
// <= 2^(E-63).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "km_gather.cuh"
#include "km_internal.cuh"
#include "km_quant.cuh"
#include "km_scatter.cuh"

namespace km {

namespace {

constexpr int kSmemHistMax = 12288;  // bins held in shared memory by the count stage

__global__ void __launch_bounds__(256)
count_kernel(const int32_t* __restrict__ assign, int64_t n, int k, int32_t* __restrict__ counts,
             const Ctl* ctl) {
  if (halted(ctl)) return;
  extern __shared__ int hist[];
  const bool use_smem = k <= kSmemHistMax;
  if (use_smem) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) hist[j] = 0;
    __syncthreads();
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int j = assign[i];
    if (use_smem) atomicAdd(&hist[j], 1);
    else atomicAdd(&counts[j], 1);
  }
  if (use_smem) {
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (hist[j]) atomicAdd(&counts[j], hist[j]);
  }
}

// Exclusive scan of counts into offs[0..k] and the scatter cursors. One block.
__global__ void __launch_bounds__(1024)
scan_kernel(const int32_t* __restrict__ counts, int k, int32_t* __restrict__ offs,
            int32_t* __restrict__ cursor, const Ctl* ctl) {
  if (halted(ctl)) return;
  __shared__ int warp_tot[32];
  __shared__ int carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < k; base += 1024) {
    const int j = base + threadIdx.x;
    const int v = j < k ? counts[j] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    const int excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
    if (j < k) {
      offs[j] = excl;
      cursor[j] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) offs[k] = carry_s;
}

__global__ void __launch_bounds__(256)
scatter_kernel(const int32_t* __restrict__ assign, int64_t n, int32_t* __restrict__ cursor,
               int32_t* __restrict__ perm, int32_t* __restrict__ slab, const Ctl* ctl) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool valid = i < n;
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const int j = assign[i];
      const unsigned peers = __match_any_sync(active, j);
      const int leader = __ffs(peers) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(&cursor[j], __popc(peers));
      pos = __shfl_sync(peers, pos, leader);
      pos += __popc(peers & ((1u << lane) - 1));
      perm[pos] = (int32_t)i;
      slab[pos] = j;
    }
  }
}

// Scatter with block-level aggregation (k <= kSmemScatterMax): each block takes
// a contiguous chunk of points, ranks them per cluster with shared-memory
// atomics, reserves one range per (block, cluster) in the global cursors, and
// writes its points there.
constexpr int kSmemScatterMax = 8192;
constexpr int kScatterPerThread = 16;

__global__ void __launch_bounds__(256)
scatter_block_kernel(const int32_t* __restrict__ assign, int64_t n, int k, int32_t* __restrict__ cursor,
                     int32_t* __restrict__ perm, int32_t* __restrict__ slab, const Ctl* ctl) {
  if (halted(ctl)) return;
  extern __shared__ int cnt[];  // per-cluster count, then the block's base position
  const int64_t chunk = (int64_t)blockDim.x * kScatterPerThread;
  for (int64_t c0 = blockIdx.x * chunk; c0 < n; c0 += (int64_t)gridDim.x * chunk) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    int lab[kScatterPerThread], rank[kScatterPerThread];
#pragma unroll
    for (int q = 0; q < kScatterPerThread; ++q) {
      const int64_t i = c0 + (int64_t)q * blockDim.x + threadIdx.x;
      lab[q] = i < n ? assign[i] : -1;
      rank[q] = lab[q] >= 0 ? atomicAdd(&cnt[lab[q]], 1) : 0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (cnt[j]) cnt[j] = atomicAdd(&cursor[j], cnt[j]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kScatterPerThread; ++q) {
      const int64_t i = c0 + (int64_t)q * blockDim.x + threadIdx.x;
      if (lab[q] >= 0) {
        perm[cnt[lab[q]] + rank[q]] = (int32_t)i;
        slab[cnt[lab[q]] + rank[q]] = lab[q];
      }
    }
    __syncthreads();
  }
}

// Scatter for k <= kSortedScatterMax: as scatter_block_kernel, but each chunk
// is written out in cluster order (scatter_chunk_sorted: runs of consecutive
// positions instead of one scattered 4-byte write per point and array).
__global__ void __launch_bounds__(256)
scatter_sorted_kernel(const int32_t* __restrict__ assign, int64_t n, int k, int32_t* __restrict__ cursor,
                      int32_t* __restrict__ perm, int32_t* __restrict__ slab, const Ctl* ctl) {
  if (halted(ctl)) return;
  extern __shared__ int ssm[];
  __shared__ int wsum[8];
  for (int64_t c0 = blockIdx.x * (int64_t)kScatterChunk; c0 < n; c0 += (int64_t)gridDim.x * kScatterChunk)
    scatter_chunk_sorted(assign + c0, (int)min((int64_t)kScatterChunk, n - c0), c0, k, cursor, perm, slab, ssm,
                         wsum);
}

// Lane column of slice v: v 32 + lane, or lane V + v when BLK (V contiguous
// columns per lane, V = 2, 4 or 8).
template <int V, bool BLK>
__device__ __forceinline__ int seg_col(int v, int lane) {
  return BLK ? lane * V + v : v * 32 + lane;
}

template <int V, bool BLK = false>
__device__ __forceinline__ void flush_sums(double* __restrict__ sums64, int j, int d, int lane,
                                           float (&s)[V], float (&c)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int t = seg_col<V, BLK>(v, lane);
    if (t < d) atomicAdd(sums64 + (int64_t)j * d + t, (double)s[v] - (double)c[v]);
    s[v] = 0.f;
    c[v] = 0.f;
  }
}

// Deterministic flush: the run's integer parts into the 64-bit accumulators
// facc[l][j d + t] (two's-complement adds through unsigned atomics).
template <int V, bool BLK = false>
__device__ __forceinline__ void flush_fixed(unsigned long long* __restrict__ facc, int64_t kd, int j, int d, int lane,
                                            int (&q)[V][3]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int t = seg_col<V, BLK>(v, lane);
    if (t < d) {
#pragma unroll
      for (int l = 0; l < 3; ++l)
        if (q[v][l]) atomicAdd(facc + l * kd + (int64_t)j * d + t, (unsigned long long)(long long)q[v][l]);
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) q[v][l] = 0;
  }
}

// The warp's objective integer parts (lane sums widened to 64 bits) into oacc[0..2].
__device__ __forceinline__ void flush_objective_fixed(unsigned long long* __restrict__ oacc, int lane, int (&o)[3]) {
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    long long v = o[l];
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0 && v) atomicAdd(oacc + l, (unsigned long long)v);
    o[l] = 0;
  }
}

// Rows of one gathered batch per stage of the segmented sum (two stages of at
// most 4 KB per warp, so that three CTAs of 8 warps share an SM).
template <int V>
__host__ __device__ constexpr int seg_rows() {
  return V == 1 ? 32 : (V == 2 ? 16 : (V <= 4 ? 8 : 4));
}

template <int V>
__host__ __device__ constexpr size_t seg_smem_bytes() {
  return (size_t)8 * 2 * seg_rows<V>() * 32 * V * sizeof(float);  // 8 warps x 2 stages x rows x 32V floats
}

// QM = 1 / 2 / 3: the pass also writes the BF16 / E4M3 / two-part BF16 codes
// of each row it reads at its sorted position p (row stride Kp elements, 2 Kp
// for the two-part codes), using the row scale in xs, and the row statistics
// xs at p; the codes equal those the quantisation stage produces for the same
// point (of the centred row x - mu when mu is given).
template <int V, int QM, bool DET>
__global__ void __launch_bounds__(256, 3)
segsum_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
              const int32_t* __restrict__ perm, const int32_t* __restrict__ slab, double* __restrict__ sums64,
              Ctl* ctl, uint8_t* __restrict__ Xq, const float4* __restrict__ xs, int Kp,
              float4* __restrict__ xs_sorted, int k, unsigned long long* __restrict__ facc,
              unsigned long long* __restrict__ oacc, const unsigned int* __restrict__ xmax, uint4* __restrict__ Xh,
              const float* __restrict__ mu) {
  constexpr int RB = seg_rows<V>();  // rows per batch (lane r < RB holds row r's indices)
  constexpr int RS = 32 * V;         // shared-memory floats per row
  // V = 2, 4, 8: a lane owns V contiguous columns, so a row is one shared-memory
  // vector load and its codes one vector store per lane (not for the two-part
  // codes, whose element-wise stores would then stride the row)
  constexpr bool BLK = (V == 2 || V == 4 || V == 8) && QM != 3;
  extern __shared__ __align__(16) float seg_smem[];
  if (halted(ctl)) return;
  // deterministic mode: grids of the coordinate sums and of the objective terms
  FxScale fxs, fxo;
  int q[DET ? V : 1][3], oq[3] = {0, 0, 0}, run_rows = 0, obj_rows = 0;
  const int64_t kd = (int64_t)k * d;
  if constexpr (DET) {
    const float xm = __uint_as_float(*xmax), cm = __uint_as_float(ctl->cmax_bits);
    fxs = fx_scale(xm);
    const float ob = __fmul_ru(__fadd_ru(xm, cm), __fadd_ru(xm, cm));  // >= every lane's sum of squares
    fxo = fx_scale(__fmul_ru(ob, 1.f + 0x1p-12f));
#pragma unroll
    for (int v = 0; v < V; ++v) q[v][0] = q[v][1] = q[v][2] = 0;
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the lane's slices of the codes' centring vector (0 without one): x - 0 = x exactly
  float muv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int t = seg_col<V, BLK>(v, lane);
    muv[v] = (QM != 0 && mu && t < d) ? __ldg(mu + t) : 0.f;
  }
  float* stage0 = seg_smem + (size_t)wib * 2 * RB * RS;
  float* stage1 = stage0 + RB * RS;
  if (BLK && d < RS) {  // columns [d, RS) of every row slot hold zeros (the gathers write only [0, d))
    for (int e = lane; e < 2 * RB * RS; e += 32)
      if (e % RS >= d) stage0[e] = 0.f;
    __syncwarp();
  }
  const int64_t nw = (int64_t)gridDim.x * 8, gw = (int64_t)blockIdx.x * 8 + wib;
  const int64_t P0 = n * gw / nw, P1 = n * (gw + 1) / nw;  // this warp's sorted positions
  const int64_t nb = (P1 - P0 + RB - 1) / RB;

  // indices of batch b: lane r < RB takes position P0 + b RB + r
  auto meta = [&](int64_t b, int& i, int& j) {
    const int64_t p = P0 + b * RB + lane;
    i = 0;
    j = -1;
    if (lane < RB && p < P1) {
      i = perm[p];
      j = slab[p];
    }
  };
  // gathers the rows of batch b into a stage (one commit group)
  auto gather = [&](int64_t b, float* st, int i_lane) {
    const int rows = (int)min((int64_t)RB, P1 - (P0 + b * RB));
    gather_rows(st, RS, X, d, rows, (int64_t)i_lane * d, lane);
  };

  float s[V], c[V], cj[V];
#pragma unroll
  for (int v = 0; v < V; ++v) { s[v] = 0.f; c[v] = 0.f; cj[v] = 0.f; }
  float objS = 0.f, objC = 0.f;
  int cur = -1;
  int i_c = 0, j_c = -1, i_n = 0, j_n = -1;
  float4 xs_c = make_float4(1.f, 0.f, 0.f, 0.f), xs_n = xs_c;
  if (nb > 0) {
    meta(0, i_c, j_c);
    gather(0, stage0, i_c);
    if (QM != 0 && lane < RB && j_c >= 0) xs_c = __ldg(&xs[i_c]);
    if (nb > 1) meta(1, i_n, j_n);
  }
  for (int64_t b = 0; b < nb; ++b) {
    float* st = (b & 1) ? stage1 : stage0;
    if (b + 1 < nb) {
      gather(b + 1, (b & 1) ? stage0 : stage1, i_n);
      if (QM != 0 && lane < RB && j_n >= 0) xs_n = __ldg(&xs[i_n]);
    }
    int i_nn = 0, j_nn = -1;
    if (b + 2 < nb) meta(b + 2, i_nn, j_nn);
    if (b + 1 < nb) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncwarp();
    const int rows = (int)min((int64_t)RB, P1 - (P0 + b * RB));
    // lane r holds row r's statistics: one coalesced store of the batch's sorted statistics
    if (QM != 0 && lane < rows) {
      xs_sorted[P0 + b * RB + lane] = xs_c;
      if (QM == 2 && Xh) store_row_slice(Xh + 2 * (P0 + b * RB + lane), xs_c.x);  // folded E4M3: 1/s slice
    }
    // rows that start a cluster run (lane r holds row r's label), found once per batch
    const int jprev = __shfl_up_sync(0xffffffffu, j_c, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane < rows && j_c != (lane == 0 ? cur : jprev));
    for (int r = 0; r < rows;) {
      if ((starts >> r) & 1u) {  // the same for every lane
        if constexpr (DET) {
          if (cur >= 0) flush_fixed<V, BLK>(facc, kd, cur, d, lane, q);
          run_rows = 0;
        } else {
          if (cur >= 0) flush_sums<V, BLK>(sums64, cur, d, lane, s, c);
        }
        cur = __shfl_sync(0xffffffffu, j_c, r);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int t = seg_col<V, BLK>(v, lane);
          cj[v] = t < d ? C[(int64_t)cur * d + t] : 0.f;
        }
      }
      const unsigned later = starts & ~((2u << r) - 1u);  // run starts after row r
      const int rend = later ? __ffs(later) - 1 : rows;
      for (; r < rend; ++r) {
        float xr[V], qo = 0.f;
        if constexpr (BLK) {
          const float* xp = st + r * RS + lane * V;
          if constexpr (V == 2) {
            const float2 a = *reinterpret_cast<const float2*>(xp);
            xr[0] = a.x;
            xr[1] = a.y;
          } else {
#pragma unroll
            for (int k4 = 0; k4 < V / 4; ++k4) {
              const float4 a = reinterpret_cast<const float4*>(xp)[k4];
              xr[4 * k4] = a.x;
              xr[4 * k4 + 1] = a.y;
              xr[4 * k4 + 2] = a.z;
              xr[4 * k4 + 3] = a.w;
            }
          }
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int t = v * 32 + lane;
            xr[v] = t < d ? st[r * RS + t] : 0.f;
          }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if constexpr (DET) fx_add(xr[v], fxs, q[v]);
          else kahan_add(s[v], c[v], xr[v]);
          const float df = __fsub_rn(xr[v], cj[v]);
          qo = fmaf(df, df, qo);
        }
        if constexpr (DET) {
          fx_add(qo, fxo, oq);
          if (++run_rows == 1024) {  // keeps every 32-bit run sum within 2^30
            flush_fixed<V, BLK>(facc, kd, cur, d, lane, q);
            run_rows = 0;
          }
          if (++obj_rows == 1024) {
            flush_objective_fixed(oacc, lane, oq);
            obj_rows = 0;
          }
        } else {
          kahan_add(objS, objC, qo);
        }
        if constexpr (QM != 0) {
          const int64_t prow = P0 + b * RB + r;
          // (BLK: a lane's columns past d get the code of 0, which is what the
          // quantisation stage leaves there; 32 V <= Kp for every BLK width)
          if constexpr (QM == 1) {
            __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(Xq) + prow * Kp;
            if constexpr (BLK) {
              uint32_t w[V / 2];
#pragma unroll
              for (int h2 = 0; h2 < V / 2; ++h2) {
                const __nv_bfloat162 pr = __floats2bfloat162_rn(__fsub_rn(xr[2 * h2], muv[2 * h2]),
                                                                __fsub_rn(xr[2 * h2 + 1], muv[2 * h2 + 1]));
                w[h2] = *reinterpret_cast<const uint32_t*>(&pr);
              }
              uint32_t* dst = reinterpret_cast<uint32_t*>(row + lane * V);
              if constexpr (V == 2) dst[0] = w[0];
              else if constexpr (V == 4) *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
              else *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const int t = v * 32 + lane;
                if (t < d) row[t] = __float2bfloat16_rn(__fsub_rn(xr[v], muv[v]));
              }
            }
          } else if constexpr (QM == 3) {
            __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(Xq) + prow * 2 * Kp;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const int t = v * 32 + lane;
              float hi, lo;
              if (t < d) split_bf16(__fsub_rn(xr[v], muv[v]), row + t, row + Kp + t, hi, lo);
            }
          } else {
            const float inv = pow2_inv(__shfl_sync(0xffffffffu, xs_c.x, r));  // 1 / row scale, exact
            uint8_t* row = Xq + prow * Kp;
            if constexpr (BLK) {
              uint8_t b[V];
#pragma unroll
              for (int v = 0; v < V; ++v) b[v] = __nv_fp8_e4m3(__fsub_rn(xr[v], muv[v]) * inv).__x;
              uint8_t* dst = row + lane * V;
              if constexpr (V == 2) {
                *reinterpret_cast<uint16_t*>(dst) = (uint16_t)(b[0] | (b[1] << 8));
              } else if constexpr (V == 4) {
                *reinterpret_cast<uint32_t*>(dst) = (uint32_t)b[0] | ((uint32_t)b[1] << 8) | ((uint32_t)b[2] << 16) |
                                                    ((uint32_t)b[3] << 24);
              } else {
                uint32_t lo4 = 0, hi4 = 0;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                  lo4 |= (uint32_t)b[v] << (8 * v);
                  hi4 |= (uint32_t)b[v + 4] << (8 * v);
                }
                *reinterpret_cast<uint2*>(dst) = make_uint2(lo4, hi4);
              }
            } else {
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const int t = v * 32 + lane;
                if (t < d) row[t] = __nv_fp8_e4m3(__fsub_rn(xr[v], muv[v]) * inv).__x;
              }
            }
          }
        }
      }
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
    i_c = i_n;
    j_c = j_n;
    xs_c = xs_n;
    i_n = i_nn;
    j_n = j_nn;
  }
  if constexpr (DET) {
    if (cur >= 0) flush_fixed<V, BLK>(facc, kd, cur, d, lane, q);
    flush_objective_fixed(oacc, lane, oq);
  } else {
    if (cur >= 0) flush_sums<V, BLK>(sums64, cur, d, lane, s, c);
    double o = (double)objS - (double)objC;
#pragma unroll
    for (int off = 16; off; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
    if (lane == 0 && o != 0.0) atomicAdd(&ctl->objective, o);
  }
}

// Deterministic mode: the grids the segmented sum used (same inputs, same values).
__device__ __forceinline__ void det_scales(const Work& w, const Ctl* ctl, FxScale& fxs, FxScale& fxo) {
  const float xm = __uint_as_float(*w.xmax), cm = __uint_as_float(ctl->cmax_bits);
  fxs = fx_scale(xm);
  const float ob = __fmul_ru(__fadd_ru(xm, cm), __fadd_ru(xm, cm));
  fxo = fx_scale(__fmul_ru(ob, 1.f + 0x1p-12f));
}

// Deterministic mode: the FP64 value of coordinate sum e, its accumulators cleared.
__device__ __forceinline__ double det_take_sum(const Work& w, int64_t kd, int64_t e, const FxScale& fxs) {
  const long long a0 = (long long)w.facc[e], a1 = (long long)w.facc[kd + e], a2 = (long long)w.facc[2 * kd + e];
  w.facc[e] = 0ull;
  w.facc[kd + e] = 0ull;
  w.facc[2 * kd + e] = 0ull;
  return fx_value(a0, a1, a2, fxs);
}

__device__ __forceinline__ double det_take_objective(const Work& w, const FxScale& fxo) {
  const long long a0 = (long long)w.oacc[0], a1 = (long long)w.oacc[1], a2 = (long long)w.oacc[2];
  w.oacc[0] = w.oacc[1] = w.oacc[2] = 0ull;
  return fx_value(a0, a1, a2, fxo);
}

// c_j = sums_j / counts_j in FP64, rounded to FP32 (an empty cluster keeps
// c_j); sums are returned rounded to FP32 and the FP64 accumulators are
// cleared for the next step. The last block to finish records the step's
// statistics and evaluates the stop rule. One warp per centroid. DET: the sums
// and the objective come from the exact integer accumulators.
template <bool DET>
__global__ void __launch_bounds__(256)
divide_kernel(float* __restrict__ C, int k, int d, const int32_t* __restrict__ counts,
              double* __restrict__ sums64, float* __restrict__ sums, Ctl* ctl, Work w, double tol) {
  if (halted(ctl)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int64_t kd = (int64_t)k * d;
  FxScale fxs, fxo;
  if constexpr (DET) det_scales(w, ctl, fxs, fxo);
  for (int j = gw; j < k; j += nw) {
    const int cnt = counts[j];
    double acc = 0.0;
    for (int t = lane; t < d; t += 32) {
      const int64_t e = (int64_t)j * d + t;
      double sv;
      if constexpr (DET) {
        sv = det_take_sum(w, kd, e, fxs);
      } else {
        sv = sums64[e];
        sums64[e] = 0.0;
      }
      sums[e] = (float)sv;
      const float co = C[e];
      const float cn = cnt > 0 ? (float)(sv / (double)cnt) : co;
      C[e] = cn;
      const double df = (double)cn - (double)co;
      acc = fma(df, df, acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      atomic_max_nonneg(&ctl->shift2_bits, acc);
      if (cnt == 0) atomicAdd(&ctl->n_empty, 1);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(&ctl->blocks_done, 1u);
    if (ticket == gridDim.x - 1) {  // last block: every other block's atomics are visible
      __threadfence();
      volatile Ctl* vc = ctl;
      const int it = vc->iters_done;
      const double shift = sqrt(__longlong_as_double((long long)vc->shift2_bits));
      const unsigned long long changed = vc->n_changed;
      if constexpr (DET) vc->objective = det_take_objective(w, fxo);
      w.obj_hist[it] = vc->objective;
      w.shift_hist[it] = shift;
      w.changed_hist[it] = changed;
      w.flagged_hist[it] = vc->n_flagged;
      w.full_hist[it] = vc->n_full;
      w.empty_hist[it] = vc->n_empty;
      w.queued_hist[it] = min(vc->n_fullq, (unsigned long long)w.fq_cap);
      vc->iters_done = it + 1;
      if (tol > 0.0 && (changed == 0 || shift <= tol)) vc->done = 1;
    }
  }
}

// max_i of the per-point norm bounds (FP32 path: xnorm; quantised paths: xs[i].w).
__global__ void __launch_bounds__(256)
xmax_kernel(const float* __restrict__ xnorm, const float4* __restrict__ xs, int64_t n, unsigned int* xmax,
            const Ctl* ctl) {
  if (halted(ctl)) return;
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, xnorm ? xnorm[i] : xs[i].w);
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomic_max_nonneg(xmax, m);
}

// A shard's partials: part[0, kd) already holds the FP64 sums (the segmented sum
// accumulates into it) or, DET, is formed from the integer accumulators;
// part[kd, kd + k) = counts, part[kd + k] = objective, part[kd + k + 1] =
// n_changed. The last block records the step's statistics (as the divide does,
// with shift and empties 0) and counts the step.
template <bool DET>
__global__ void __launch_bounds__(256)
finish_partial_kernel(const int32_t* __restrict__ counts, int k, int d, double* __restrict__ part, Ctl* ctl,
                      Work w) {
  if (halted(ctl)) return;
  const int64_t kd = (int64_t)k * d;
  FxScale fxs, fxo;
  if constexpr (DET) det_scales(w, ctl, fxs, fxo);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kd + k; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < kd) {
      if constexpr (DET) part[e] = det_take_sum(w, kd, e, fxs);
    } else {
      part[e] = (double)counts[e - kd];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(&ctl->blocks_done, 1u);
    if (ticket == gridDim.x - 1) {
      __threadfence();
      volatile Ctl* vc = ctl;
      const int it = vc->iters_done;
      if constexpr (DET) vc->objective = det_take_objective(w, fxo);
      part[kd + k] = vc->objective;
      part[kd + k + 1] = (double)vc->n_changed;
      w.obj_hist[it] = vc->objective;
      w.shift_hist[it] = 0.0;
      w.changed_hist[it] = vc->n_changed;
      w.flagged_hist[it] = vc->n_flagged;
      w.full_hist[it] = vc->n_full;
      w.empty_hist[it] = 0;
      w.queued_hist[it] = min(vc->n_fullq, (unsigned long long)w.fq_cap);
      vc->iters_done = it + 1;
    }
  }
}

// actl[0] = 1 when a count of the reduced buffer is not an integer in [0, 2^31).
__global__ void __launch_bounds__(256)
check_partials_kernel(const double* __restrict__ part, int k, int d, unsigned long long* actl) {
  const int64_t kd = (int64_t)k * d;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
    const double c = part[kd + j];
    if (!(c >= 0.0 && c < 2147483648.0 && c == floor(c))) atomicExch(actl, 1ull);
  }
}

// The divide from a reduced buffer (one warp per centroid): as divide_kernel,
// with actl[1] = max_j ||dc_j||^2 (FP64 bits) and actl[2] = empty clusters.
__global__ void __launch_bounds__(256)
apply_partials_kernel(const double* __restrict__ part, int k, int d, float* __restrict__ C, float* __restrict__ sums,
                      int32_t* __restrict__ counts, unsigned long long* actl) {
  if (*(volatile unsigned long long*)actl) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int64_t kd = (int64_t)k * d;
  for (int j = gw; j < k; j += nw) {
    const int cnt = (int)part[kd + j];
    double acc = 0.0;
    for (int t = lane; t < d; t += 32) {
      const int64_t e = (int64_t)j * d + t;
      const double sv = part[e];
      if (sums) sums[e] = (float)sv;
      const float co = C[e];
      const float cn = cnt > 0 ? (float)(sv / (double)cnt) : co;
      C[e] = cn;
      const double df = (double)cn - (double)co;
      acc = fma(df, df, acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      atomic_max_nonneg(&actl[1], acc);
      if (cnt == 0) atomicAdd(&actl[2], 1ull);
      if (counts) counts[j] = cnt;
    }
  }
}

}  // namespace

cudaError_t launch_count(const Problem& p, const Work& w, cudaStream_t s) {
  const size_t smem = p.k <= kSmemHistMax ? (size_t)p.k * sizeof(int) : 0;
  int64_t blocks = (p.n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 2;
  if (blocks > cap) blocks = cap;
  count_kernel<<<(int)blocks, 256, smem, s>>>(p.assign, p.n, p.k, p.counts, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_scan(const Problem& p, const Work& w, cudaStream_t s) {
  scan_kernel<<<1, 1024, 0, s>>>(p.counts, p.k, w.offs, w.cursor, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const Problem& p, const Work& w, cudaStream_t s) {
  if (p.k <= kSortedScatterMax) {
    int64_t blocks = (p.n + kScatterChunk - 1) / kScatterChunk;
    const int64_t cap = (int64_t)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    const size_t smem = (size_t)sorted_scatter_ints(p.k) * sizeof(int);
    scatter_sorted_kernel<<<(int)blocks, 256, smem, s>>>(p.assign, p.n, p.k, w.cursor, w.perm, w.lab_sorted, w.ctl);
    return cudaGetLastError();
  }
  if (p.k <= kSmemScatterMax) {
    int64_t blocks = (p.n + 256 * kScatterPerThread - 1) / (256 * kScatterPerThread);
    const int64_t cap = (int64_t)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    scatter_block_kernel<<<(int)blocks, 256, (size_t)p.k * sizeof(int), s>>>(p.assign, p.n, p.k, w.cursor, w.perm,
                                                                              w.lab_sorted, w.ctl);
    return cudaGetLastError();
  }
  int64_t blocks = (p.n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  scatter_kernel<<<(int)blocks, 256, 0, s>>>(p.assign, p.n, w.cursor, w.perm, w.lab_sorted, w.ctl);
  return cudaGetLastError();
}

template <int V, int QM, bool DET>
cudaError_t seg_attr() {
  return cudaFuncSetAttribute(segsum_kernel<V, QM, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)seg_smem_bytes<V>());
}

template <int V>
cudaError_t seg_attrs() {
  cudaError_t e = seg_attr<V, 0, false>();
  if (e == cudaSuccess) e = seg_attr<V, 1, false>();
  if (e == cudaSuccess) e = seg_attr<V, 2, false>();
  if (e == cudaSuccess) e = seg_attr<V, 3, false>();
  if (e == cudaSuccess) e = seg_attr<V, 0, true>();
  if (e == cudaSuccess) e = seg_attr<V, 1, true>();
  if (e == cudaSuccess) e = seg_attr<V, 2, true>();
  if (e == cudaSuccess) e = seg_attr<V, 3, true>();
  return e;
}

cudaError_t init_segsum() {
  cudaError_t e = seg_attrs<1>();
  if (e == cudaSuccess) e = seg_attrs<2>();
  if (e == cudaSuccess) e = seg_attrs<3>();
  if (e == cudaSuccess) e = seg_attrs<4>();
  if (e == cudaSuccess) e = seg_attrs<5>();
  if (e == cudaSuccess) e = seg_attrs<6>();
  if (e == cudaSuccess) e = seg_attrs<7>();
  if (e == cudaSuccess) e = seg_attrs<8>();
  return e;
}

template <int V, int QM, bool DET>
void seg_launch(int blocks, const Problem& p, const Work& w, int Kp, cudaStream_t s) {
  segsum_kernel<V, QM, DET><<<blocks, 256, seg_smem_bytes<V>(), s>>>(
      p.X, p.n, p.d, p.C, w.perm, w.lab_sorted, w.sums64, w.ctl, QM ? w.Xq : nullptr, QM ? w.xs : nullptr,
      QM ? Kp : 0, QM ? w.xs_sorted : nullptr, p.k, w.facc, w.oacc, w.xmax,
      QM == 2 ? reinterpret_cast<uint4*>(w.Xh) : nullptr, QM ? w.mu : nullptr);
}

template <int V, bool DET>
void seg_launch_q(int qmode, int blocks, const Problem& p, const Work& w, int Kp, cudaStream_t s) {
  if (qmode == 1) seg_launch<V, 1, DET>(blocks, p, w, Kp, s);
  else if (qmode == 2) seg_launch<V, 2, DET>(blocks, p, w, Kp, s);
  else if (qmode == 3) seg_launch<V, 3, DET>(blocks, p, w, Kp, s);
  else seg_launch<V, 0, DET>(blocks, p, w, Kp, s);
}

template <int V>
void seg_launch_v(int qmode, int det, int blocks, const Problem& p, const Work& w, int Kp, cudaStream_t s) {
  if (det) seg_launch_q<V, true>(qmode, blocks, p, w, Kp, s);
  else seg_launch_q<V, false>(qmode, blocks, p, w, Kp, s);
}

cudaError_t launch_segsum(const Problem& p, const Work& w, cudaStream_t s, int qmode, int Kp, int det) {
  // two CTAs of 8 warps per SM; each warp takes a contiguous range of at least 64 positions
  int64_t blocks = (p.n + 8 * 64 - 1) / (8 * 64);
  if (blocks > 3 * num_sms()) blocks = 3 * num_sms();  // three CTAs of 8 warps per SM
  if (det && (!w.facc || !w.oacc || !w.xmax)) return cudaErrorInvalidValue;
  const int V = (p.d + 31) / 32;
  switch (V) {
    case 1: seg_launch_v<1>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 2: seg_launch_v<2>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 3: seg_launch_v<3>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 4: seg_launch_v<4>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 5: seg_launch_v<5>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 6: seg_launch_v<6>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 7: seg_launch_v<7>(qmode, det, (int)blocks, p, w, Kp, s); break;
    case 8: seg_launch_v<8>(qmode, det, (int)blocks, p, w, Kp, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_divide(const Problem& p, const Work& w, int iter, double tol, cudaStream_t s, int det) {
  (void)iter;
  int blocks = (p.k + 7) / 8;
  const int cap = num_sms() * 4;
  if (blocks > cap) blocks = cap;
  if (det) divide_kernel<true><<<blocks, 256, 0, s>>>(p.C, p.k, p.d, p.counts, w.sums64, p.sums, w.ctl, w, tol);
  else divide_kernel<false><<<blocks, 256, 0, s>>>(p.C, p.k, p.d, p.counts, w.sums64, p.sums, w.ctl, w, tol);
  return cudaGetLastError();
}

cudaError_t launch_xmax(const float* xnorm, const float4* xs, int64_t n, const Work& w, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.xmax, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  xmax_kernel<<<(int)blocks, 256, 0, s>>>(xnorm, xs, n, w.xmax, w.ctl);
  return cudaGetLastError();
}

cudaError_t launch_finish_partial(const Problem& p, const Work& w, double* part, int det, cudaStream_t s) {
  const int64_t kd = (int64_t)p.k * p.d;
  int64_t blocks = (kd + p.k + 255) / 256;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  if (det) finish_partial_kernel<true><<<(int)blocks, 256, 0, s>>>(p.counts, p.k, p.d, part, w.ctl, w);
  else finish_partial_kernel<false><<<(int)blocks, 256, 0, s>>>(p.counts, p.k, p.d, part, w.ctl, w);
  return cudaGetLastError();
}

cudaError_t launch_apply_partials(const double* part, int k, int d, float* C, float* sums, int32_t* counts,
                                  unsigned long long* actl, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(actl, 0, 4 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int blocks = (k + 255) / 256;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  check_partials_kernel<<<blocks, 256, 0, s>>>(part, k, d, actl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  blocks = (k + 7) / 8;
  if (blocks > num_sms() * 4) blocks = num_sms() * 4;
  apply_partials_kernel<<<blocks, 256, 0, s>>>(part, k, d, C, sums, counts, actl);
  return cudaGetLastError();
}

}  // namespace km
