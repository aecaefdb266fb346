// Counting-sort scatter of one chunk of points by cluster (the reduce stage of
// km_reduce.cu and km_batched.cu).
#pragma once

#include "km_internal.cuh"

namespace km {

constexpr int kScatterChunk = 4096;      // points per chunk: 16 per thread of a 256-thread block
constexpr int kSortedScatterMax = 1536;  // clusters of the sorted-write scatter (2 k + 2 chunk ints < 48 KB)

// Shared-memory ints the sorted-write scatter of a chunk needs for k clusters.
__host__ __device__ constexpr int sorted_scatter_ints(int k) { return 2 * k + 2 * kScatterChunk; }

// Scatters points i0 + r (r < n <= kScatterChunk) with labels a[r] in [0, k):
// ranks them per cluster with shared-memory atomics, takes the exclusive
// prefix of the counts (the local sorted order), reserves one range per
// cluster in the global cursors, places the points in shared memory in
// cluster order and writes them out with consecutive threads on consecutive
// positions of perm (point index) and slab (label). One 256-thread block;
// sm holds sorted_scatter_ints(k) ints, wsum 8. Ends with a block barrier.
__device__ __forceinline__ void scatter_chunk_sorted(const int32_t* __restrict__ a, int n, int64_t i0, int k,
                                                     int32_t* __restrict__ cursor, int32_t* __restrict__ perm,
                                                     int32_t* __restrict__ slab, int* sm, int* wsum) {
  constexpr int kPer = kScatterChunk / 256;
  int* cnt = sm;                   // [k] per-cluster count, then the cluster's global base
  int* lst = sm + k;               // [k] the cluster's first local sorted index
  int* sidx = sm + 2 * k;          // [kScatterChunk] point offsets in local sorted order
  int* slabs = sidx + kScatterChunk;  // [kScatterChunk] their labels
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int j = tid; j < k; j += 256) cnt[j] = 0;
  __syncthreads();
  int lab[kPer], rank[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int r = q * 256 + tid;
    lab[q] = r < n ? __ldg(a + r) : -1;
    rank[q] = lab[q] >= 0 ? atomicAdd(&cnt[lab[q]], 1) : 0;
  }
  __syncthreads();
  // exclusive prefix of the counts: thread tid takes entries [tid per, tid per + per)
  const int per = (k + 255) / 256;
  const int j0 = tid * per;
  int loc = 0;
  for (int u = 0; u < per; ++u)
    if (j0 + u < k) loc += cnt[j0 + u];
  int x = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < 8 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < 8) wsum[lane] = w;
  }
  __syncthreads();
  int base = (wid ? wsum[wid - 1] : 0) + x - loc;
  for (int u = 0; u < per; ++u)
    if (j0 + u < k) {
      lst[j0 + u] = base;
      base += cnt[j0 + u];
    }
  __syncthreads();
  for (int j = tid; j < k; j += 256)
    if (cnt[j]) cnt[j] = atomicAdd(&cursor[j], cnt[j]);
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (lab[q] >= 0) {
      const int ls = lst[lab[q]] + rank[q];
      sidx[ls] = q * 256 + tid;
      slabs[ls] = lab[q];
    }
  __syncthreads();
  for (int e = tid; e < n; e += 256) {  // every point of the chunk was placed
    const int j = slabs[e];
    perm[cnt[j] + (e - lst[j])] = (int32_t)(i0 + sidx[e]);
    slab[cnt[j] + (e - lst[j])] = j;
  }
  __syncthreads();
}

}  // namespace km
