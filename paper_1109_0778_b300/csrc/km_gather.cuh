// Row gathers into shared memory with cp.async (the segmented sums of
// km_reduce.cu and km_batched.cu).
#pragma once

#include "km_internal.cuh"

namespace km {

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies rows 0..bn-1 (bn <= 32) of a batch into st, row r at st + r * rs.
// Lane r < bn holds row r's element offset off into X; every row has d
// elements. The warp's lanes split into groups of L (a power of two covering a
// row's 16-byte pieces, at most 32), one row per group, so a warp instruction
// moves 32 / L rows. 16-byte pieces when rows start on 16-byte boundaries
// (d a multiple of 4 and X itself 16-byte aligned), else 4-byte ones. Commits
// one group (unless commit is false: the caller commits several gathers as one).
__device__ __forceinline__ void gather_rows(float* st, int rs, const float* X, int d, int bn, int64_t off, int lane,
                                            bool commit = true) {
  const bool v4 = (d & 3) == 0 && ((uintptr_t)X & 15) == 0;
  const int cpr = v4 ? d >> 2 : d;  // pieces per row
  int lg = 0;
  while ((1 << lg) < cpr && lg < 5) ++lg;
  const int L = 1 << lg, rpi = 32 >> lg;  // lanes per row, rows per instruction
  const int sub = lane >> lg, o0 = lane & (L - 1);
  for (int r0 = 0; r0 < bn; r0 += rpi) {
    const int r = r0 + sub;
    const int64_t ro = __shfl_sync(0xffffffffu, off, r < bn ? r : 0);
    if (r < bn) {
      const float* x = X + ro;
      float* dst = st + r * rs;
      if (v4) {
        for (int o = o0; o < cpr; o += L) cp_async16(dst + 4 * o, x + 4 * o);
      } else {
        for (int o = o0; o < cpr; o += L) cp_async4(dst + o, x + o);
      }
    }
  }
  if (commit) cp_async_commit();
}

}  // namespace km
