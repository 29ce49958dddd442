// common.cuh -- shared device definitions of the GB300 Louvain kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "louvain.h"

namespace lv {

constexpr int32_t kEmpty = -1;     // empty hash-table key
constexpr int kBlock = 256;        // threads per block of the vertex-parallel kernels
constexpr int kNumBuckets = 7;     // degree buckets of the per-vertex kernels
constexpr int64_t kInFlightPerSm = 1024;  // vertices a local-moving launch holds per SM (4-lane groups)

// Degree buckets: upper bound of the row length (arcs, self-loop included) handled by each.
//   0: 1..4       groups of 4 lanes, 8-slot shared-memory table
//   1: 5..16      groups of 8 lanes, 32 slots
//   2: 17..128    one warp, 256 slots
//   3: 129..512   one warp, 1024 slots (8 KB per warp, 64 KB of dynamic shared memory per block)
//   4: 513..2048  one 256-thread block, 4096 slots (32 KB)
//   5: 2049..4096 one 256-thread block, 8192 slots (64 KB, dynamic shared memory)
//   6: > 4096     giant: arc chunks and table slices over the whole GPU (giant.cu)
__host__ __device__ inline int degree_bucket(int64_t deg) {
  if (deg <= 0) return -1;
  if (deg <= 4) return 0;
  if (deg <= 16) return 1;
  if (deg <= 128) return 2;
  if (deg <= 512) return 3;
  if (deg <= 2048) return 4;
  if (deg <= 4096) return 5;
  return 6;
}

// Device control block: per-iteration accumulators and convergence state.
struct Ctrl {
  unsigned long long sum_lo, sum_hi;  // integer mode: sum of performed-move scores N (128-bit)
  double sum_f;                       // fp mode: same in fp64
  unsigned long long moves;           // moves in the current iteration
  unsigned long long moves_pass;      // moves in the current pass
  int32_t done;                       // local-moving phase finished
  int32_t iterations;                 // l_i of the current pass
  int32_t max_iterations;
  int32_t error;                      // bit set by kernels on an internal failure
  long long two_m_i;                  // 2m, integer mode
  double two_m_f;                     // 2m, fp mode
  double tau;                         // current tolerance
  unsigned long long cnt[8];          // general counters (colouring rounds, maxima, reductions)
  long long acc_i[4];                 // general integer accumulators
  double acc_f[4];                    // general fp accumulators
  double q;                           // last modularity
  unsigned long long gslots;          // table slots the giant rows of a bucket sort need
  // algorithmic-traffic counters, summed over a run (reset by the host before each run)
  unsigned long long lm_stat[kNumBuckets][6];  // local move: list entries, vertices processed, arcs
                                                // scanned, candidates scored, moves, neighbour marks
  unsigned long long mg_stat[kNumBuckets][4];  // merge: communities, members, arcs scanned, arcs written
  unsigned long long hub_arcs, all_arcs;        // arcs in rows over 512 arcs, all arcs (hub_share)
};

// Adds K per-thread counters of a whole block to dst[0..K) (one atomic per counter per block).
// Every thread of the block must call it; the block has at most W warps (the merge kernels keep
// W = 32: their smaller footprint let more blocks share an SM's L1 and measured slower).
template <int K, int W = 32>
__device__ __forceinline__ void block_add_counters(unsigned long long* dst, unsigned long long (&v)[K]) {
  __shared__ unsigned long long part[K][W];
#pragma unroll
  for (int k = 0; k < K; k++) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < K; k++) part[k][threadIdx.x >> 5] = v[k];
  __syncthreads();
  if (threadIdx.x < K) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[threadIdx.x][w];
    if (t) atomicAdd(&dst[threadIdx.x], t);
  }
}

enum CtrlErr : int32_t { kErrTableFull = 1, kErrTimeout = 2, kErrRange = 4 };

// Per-graph control of a batched run (louvain_run_batch): the graphs of a batch are disjoint
// vertex ranges of one union graph, and everything the method keeps per graph -- 2m, the
// per-iteration sum of N, the tolerance test, l_i, the pass decisions -- lives here.
struct GraphCtl {
  unsigned long long sum_lo, sum_hi;  // integer mode: sum of performed-move scores N (128-bit)
  double sum_f;                       // fp mode
  long long two_m_i;                  // 2m of the graph
  double two_m_f;
  long long vbase;                    // first vertex of the graph at the current level
  long long nlev;                     // vertices of the graph at the current level
  long long nbase;                    // first vertex at the next level (continuing graphs)
  long long comm_base;                // occupied community ids before the graph (renumbering)
  long long n_comm;                   // communities after the current pass
  long long sig_in_i, sq_i;           // final modularity sums, integer mode
  double sig_in_f, sq_f;              // final modularity sums, fp mode
  double q;                           // final modularity
  int32_t active;                     // in the pass loop at the current level
  int32_t done;                       // local-moving phase of the current pass finished
  int32_t iterations;                 // l_i of the current pass
  int32_t cont;                       // continues to the next pass
  int32_t passes;                     // passes run
  int32_t total_iterations;           // sum of l_i
};

// Vertex segmentation of a batched run: vg[v] = graph of vertex v at the current level (null for
// a single graph).  The colouring priority and the random classes hash the id LOCAL to the graph,
// so a graph is treated identically alone and inside a batch.
struct Segs {
  const int32_t* vg = nullptr;
  const GraphCtl* gc = nullptr;
};
__device__ __forceinline__ uint64_t local_id(const Segs& s, int32_t v) {
  return s.vg ? (uint64_t)((long long)v - s.gc[s.vg[v]].vbase) : (uint64_t)v;
}

// ------------------------------------------------------------------ mode traits
struct IntMode {
  typedef int32_t w_t;             // stored arc weight
  typedef uint32_t h_t;            // per-vertex community sum (< 2m < 2^31)
  typedef long long a_t;           // K, Sigma, 2m
  typedef long long s_t;           // move score N
  static constexpr bool is_fp = false;
  static __device__ __forceinline__ s_t score(h_t kic, h_t kid, a_t ki, a_t sc, a_t sd, a_t two_m) {
    // Eq. 2 times 2m^2: 2m (K_i->c - K_i->d) - K_i (Sigma_c - Sigma_d + K_i), exact in int64
    return two_m * ((long long)kic - (long long)kid) - ki * (sc - sd + ki);
  }
  static __device__ __forceinline__ s_t lowest() { return (long long)0x8000000000000000ULL; }
};

struct FpMode {
  typedef float w_t;
  typedef float h_t;               // fp32 accumulation of K_i->c
  typedef double a_t;              // fp64 K, Sigma, 2m
  typedef double s_t;
  static constexpr bool is_fp = true;
  static __device__ __forceinline__ s_t score(h_t kic, h_t kid, a_t ki, a_t sc, a_t sd, a_t two_m) {
    return two_m * ((double)kic - (double)kid) - ki * (sc - sd + ki);
  }
  static __device__ __forceinline__ s_t lowest() { return -1.0e300; }
};

// ------------------------------------------------------------------ atomics on the accumulator types
__device__ __forceinline__ void atomic_add_a(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void atomic_add_a(double* p, double v) { atomicAdd(p, v); }

// ------------------------------------------------------------------ counter hash (colouring priority)
// SplitMix64 output function (Steele, Lea and Flood 2014); hash3 chains it over three words:
// x = mix(a + g); x = mix(x + b + 2g); return mix(x + c + 3g), g = 0x9e3779b97f4a7c15.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t hash3(uint64_t a, uint64_t b, uint64_t c) {
  const uint64_t g = 0x9e3779b97f4a7c15ULL;
  uint64_t x = mix64(a + g);
  x = mix64(x + b + 2 * g);
  return mix64(x + c + 3 * g);
}
// Strict priority order of the colouring: u before v iff (prio(u), u) > (prio(v), v).
__device__ __forceinline__ bool higher(uint64_t pu, int32_t u, uint64_t pv, int32_t v) {
  return pu > pv || (pu == pv && u > v);
}

// ------------------------------------------------------------------ 128-bit exact sums
// Adds a 128-bit (hi, lo) value to a global pair with carry propagation.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lo_p, unsigned long long* hi_p,
                                                unsigned long long lo, unsigned long long hi) {
  if (lo) {
    unsigned long long old = atomicAdd(lo_p, lo);
    if (old + lo < old) hi += 1;
  }
  if (hi) atomicAdd(hi_p, hi);
}

// Round-to-nearest-even conversion of the unsigned 128-bit value (hi, lo) to double.  Keeps the
// top 64 significant bits with a sticky bit for everything below, then one hardware u64->f64
// rounding (the 64-bit value has >= 11 bits beyond the 53-bit mantissa, so the sticky bit makes
// the single rounding exact), then an exact power-of-two scaling.
__device__ __forceinline__ double u128_to_double_rn(unsigned long long hi, unsigned long long lo) {
  if (hi == 0) return __ull2double_rn(lo);
  int lz = __clzll(hi);                 // 0..63
  int sh = 64 - lz;                     // bits to drop from the bottom
  unsigned long long top = (hi << lz) | (lz ? (lo >> (64 - lz)) : 0ULL);
  unsigned long long dropped_mask = (sh >= 64) ? ~0ULL : ((1ULL << sh) - 1ULL);
  unsigned long long sticky = (lo & dropped_mask) != 0ULL ? 1ULL : 0ULL;
  top |= sticky;
  return ldexp(__ull2double_rn(top), sh);
}

// ------------------------------------------------------------------ groups of G threads
// G <= 32: an aligned sub-warp tile; G > 32: the whole block (blockDim.x == G).
template <int G>
struct Grp {
  static __device__ __forceinline__ unsigned lane() { return G <= 32 ? (threadIdx.x & (G - 1)) : threadIdx.x; }
  static __device__ __forceinline__ unsigned mask() {
    if constexpr (G >= 32) return 0xffffffffu;
    else return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  }
  static __device__ __forceinline__ void sync() {
    if constexpr (G <= 32) __syncwarp(mask());
    else __syncthreads();
  }
};

// Sum over a group.  Block groups use `scratch` (>= G / 32 elements of T) in shared memory.
template <int G, class T>
__device__ __forceinline__ T group_sum(T v, T* scratch) {
  if (G <= 32) {
    unsigned m = Grp<G>::mask();
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
  } else {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = T(0);
    for (int w = 0; w < G / 32; w++) t += scratch[w];
    __syncthreads();
    return t;
  }
}

// (score, community) argmax over a group: larger score wins, ties to the smaller community id.
template <class S>
__device__ __forceinline__ bool better(S s1, int32_t c1, S s2, int32_t c2) {
  return s1 > s2 || (s1 == s2 && (unsigned)c1 < (unsigned)c2);
}

template <int G, class S>
__device__ __forceinline__ void group_argmax(S& s, int32_t& c, S* ss, int32_t* sc) {
  if (G <= 32) {
    unsigned m = Grp<G>::mask();
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) {
      S s2 = __shfl_xor_sync(m, s, o);
      int32_t c2 = __shfl_xor_sync(m, c, o);
      if (better(s2, c2, s, c)) { s = s2; c = c2; }
    }
  } else {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      S s2 = __shfl_xor_sync(0xffffffffu, s, o);
      int32_t c2 = __shfl_xor_sync(0xffffffffu, c, o);
      if (better(s2, c2, s, c)) { s = s2; c = c2; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { ss[threadIdx.x >> 5] = s; sc[threadIdx.x >> 5] = c; }
    __syncthreads();
    s = ss[0]; c = sc[0];
    for (int w = 1; w < G / 32; w++)
      if (better(ss[w], sc[w], s, c)) { s = ss[w]; c = sc[w]; }
    __syncthreads();
  }
}

// OR of a predicate over the group (uniform result; for a block it is also a barrier).
template <int G>
__device__ __forceinline__ bool group_any(bool p) {
  if constexpr (G <= 32) return __any_sync(Grp<G>::mask(), p);
  else return __syncthreads_or(p ? 1 : 0) != 0;
}

// Broadcast lane 0's value to the group.
template <int G, class T>
__device__ __forceinline__ T group_bcast(T v, T* scratch) {
  if (G <= 32) {
    return __shfl_sync(Grp<G>::mask(), v, 0, G);
  } else {
    __syncthreads();
    if (threadIdx.x == 0) scratch[0] = v;
    __syncthreads();
    T r = scratch[0];
    __syncthreads();
    return r;
  }
}

// ------------------------------------------------------------------ open-addressing table
// Keys are community ids (kEmpty = free), linear probing from a multiplicative hash.  A table
// of `size` (power of two) slots is only used for at most size/2 distinct keys, so an insert
// always finds a slot; the probe loop is bounded anyway and reports failure.
__device__ __forceinline__ unsigned tbl_home(int32_t key, int shift) {
  return ((unsigned)key * 2654435769u) >> shift;
}

template <class V>
__device__ __forceinline__ bool tbl_add(int32_t* keys, V* vals, unsigned size, int shift, int32_t key, V w) {
  unsigned s = tbl_home(key, shift);
  for (unsigned p = 0; p < size; p++) {
    int32_t k = *((volatile int32_t*)&keys[s]);
    if (k == key) { atomicAdd(&vals[s], w); return true; }
    if (k == kEmpty) {
      int32_t old = atomicCAS(&keys[s], kEmpty, key);
      if (old == kEmpty || old == key) { atomicAdd(&vals[s], w); return true; }
    }
    s = (s + 1) & (size - 1);
  }
  return false;
}

// tbl_add that also reports a new key: 0 = table full, 1 = added to an existing key, 2 = this call
// claimed the key's slot (*slot = its index).
template <class V>
__device__ __forceinline__ int tbl_add_claim(int32_t* keys, V* vals, unsigned size, int shift, int32_t key, V w,
                                             unsigned* slot) {
  unsigned s = tbl_home(key, shift);
  for (unsigned p = 0; p < size; p++) {
    int32_t k = *((volatile int32_t*)&keys[s]);
    if (k == key) { atomicAdd(&vals[s], w); return 1; }
    if (k == kEmpty) {
      int32_t old = atomicCAS(&keys[s], kEmpty, key);
      if (old == kEmpty) { atomicAdd(&vals[s], w); *slot = s; return 2; }
      if (old == key) { atomicAdd(&vals[s], w); return 1; }
    }
    s = (s + 1) & (size - 1);
  }
  return 0;
}

// Tables of {key, value} pairs (the giant-row pool): slot s is kv[2s] (key) and kv[2s + 1] (value
// bits of an h_t, a uint32_t or float), so one 8-byte access reads or clears a slot; empty =
// {kEmpty, 0}.
template <class V>
__device__ __forceinline__ uint32_t val_bits(V w);
template <>
__device__ __forceinline__ uint32_t val_bits<uint32_t>(uint32_t w) { return w; }
template <>
__device__ __forceinline__ uint32_t val_bits<float>(float w) { return __float_as_uint(w); }
template <class H>
__device__ __forceinline__ H int_as_h(int32_t x);
template <>
__device__ __forceinline__ uint32_t int_as_h<uint32_t>(int32_t x) { return (uint32_t)x; }
template <>
__device__ __forceinline__ float int_as_h<float>(int32_t x) { return __int_as_float(x); }
constexpr unsigned long long kEmptyPair = 0xFFFFFFFFull;  // {kEmpty, 0} as one little-endian word

// log2 of the table size for `distinct_bound` keys: the smallest power of two >= 2*bound, at
// least `min_size`, at most `max_size` (callers guarantee 2*bound <= max_size).
__host__ __device__ __forceinline__ int tbl_log2(int64_t distinct_bound, int min_log2, int max_log2) {
  int l = min_log2;
  while (l < max_log2 && ((int64_t)1 << l) < 2 * distinct_bound) l++;
  return l;
}

// The same with f table slots per key of the bound (f = 1, 2 or 4: tables up to full, half full or
// a quarter full); tbl_log2 is f = 2.
__host__ __device__ __forceinline__ int tbl_log2f(int64_t distinct_bound, int f, int min_log2, int max_log2) {
  int l = min_log2;
  while (l < max_log2 && ((int64_t)1 << l) < (int64_t)f * distinct_bound) l++;
  return l;
}

// tbl_log2f by counting leading zeros (device code; f * bound below 2^31).
__device__ __forceinline__ int tbl_log2f_fast(int64_t distinct_bound, int f, int min_log2, int max_log2) {
  const unsigned need = (unsigned)f * (unsigned)distinct_bound;  // slots wanted
  const int l = need <= 1u ? 0 : 32 - __clz(need - 1u);           // smallest l with 2^l >= need
  return l < min_log2 ? min_log2 : (l > max_log2 ? max_log2 : l);
}

// Warp-level (or sub-warp) lane mask of the lanes below this one within the warp.
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

}  // namespace lv
