// flat.cuh -- block-flat traversal of the arcs of 256 consecutive rows.
//
// A block loads the rows [r0, r0 + 256), takes an exclusive prefix sum of their lengths in
// shared memory and lets all its threads walk the flat index space of their arcs; the owning row
// of flat index f is found by binary search.  Consecutive lanes get consecutive f, so within a
// warp the owners are non-decreasing -- warp_seg_scan relies on that.
#pragma once

#include "common.cuh"

namespace lv {

struct FlatRows {
  int64_t excl[kBlock + 1];
  int64_t beg[kBlock];
};

// Fills fr for rows [r0, r0 + kBlock) of (rbeg, rend) with n rows; returns the arc total.
__device__ __forceinline__ int64_t flat_load(FlatRows& fr, int64_t r0, int64_t n, const int64_t* rbeg,
                                             const int64_t* rend) {
  const int64_t r = r0 + threadIdx.x;
  int64_t len = 0, b = 0;
  if (r < n) { b = rbeg[r]; len = rend[r] - b; }
  fr.beg[threadIdx.x] = b;
  fr.excl[threadIdx.x + 1] = len;
  if (threadIdx.x == 0) fr.excl[0] = 0;
  __syncthreads();
  for (int o = 1; o < kBlock; o <<= 1) {
    const int64_t v = (int)threadIdx.x + 1 > o ? fr.excl[threadIdx.x + 1 - o] : 0;
    __syncthreads();
    fr.excl[threadIdx.x + 1] += v;
    __syncthreads();
  }
  return fr.excl[kBlock];
}

// Row (0..kBlock-1) owning flat index f < total.
__device__ __forceinline__ int flat_row(const FlatRows& fr, int64_t f) {
  int lo = 0, hi = kBlock - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr.excl[mid] <= f) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Segmented inclusive sum across a warp whose keys are non-decreasing by lane; is_tail marks the
// last lane of each run of equal keys.
template <class T>
__device__ __forceinline__ T warp_seg_scan(int key, T v, bool& is_tail) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, v, o);
    const int k2 = __shfl_up_sync(0xffffffffu, key, o);
    if (lane >= o && k2 == key) v += y;
  }
  const int kn = __shfl_down_sync(0xffffffffu, key, 1);
  is_tail = lane == 31 || kn != key;
  return v;
}

}  // namespace lv
