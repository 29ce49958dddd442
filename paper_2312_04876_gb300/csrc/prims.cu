// prims.cu -- exclusive scan, counting sort into degree / colour buckets, renumbering helpers.
//
// Scan (Algorithm 3's exclusiveScan, also used for renumbering in Algorithm 1): three launches,
// tile sums -> scan of the tile sums in one block -> per-tile scan with the tile prefix.  Tiles of
// 4096 elements; each warp of a tile owns 512 consecutive elements and scans them 32 at a time
// with shuffles (coalesced loads and stores).  No inter-block waiting, so nothing can spin.
#include "internal.cuh"

namespace lv {

constexpr int kScanTile = 4096;
constexpr int kScanWarpSpan = kScanTile / (kBlock / 32);  // 512

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <class T>
__device__ __forceinline__ long long warp_chunk_sum(const T* in, int64_t beg, int64_t n) {
  long long s = 0;
  int lane = threadIdx.x & 31;
  for (int r = 0; r < kScanWarpSpan / 32; r++) {
    int64_t i = beg + r * 32 + lane;
    if (i < n) s += (long long)in[i];
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

template <class T>
__global__ void __launch_bounds__(kBlock) scan_tile_sums(const T* in, int64_t n, long long* tsum) {
  __shared__ long long ws[kBlock / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (threadIdx.x >> 5) * kScanWarpSpan;
  long long s = warp_chunk_sum(in, base, n);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kBlock / 32; w++) t += ws[w];
    tsum[blockIdx.x] = t;
  }
}

// Exclusive scan of tsum[0, m) in place by one block of 1024 threads; *total = sum.
__global__ void __launch_bounds__(1024) scan_tile_prefix(long long* tsum, int64_t m, long long* total) {
  __shared__ long long part[1024];
  int64_t per = (m + 1023) / 1024;
  int64_t b = (int64_t)threadIdx.x * per, e = b + per < m ? b + per : m;
  long long s = 0;
  for (int64_t i = b; i < e; i++) s += tsum[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan of the 1024 partials
    long long v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t i = b; i < e; i++) { long long v = tsum[i]; tsum[i] = run; run += v; }
  if (threadIdx.x == 1023) *total = part[1023];
}

template <class T>
__global__ void __launch_bounds__(kBlock) scan_tiles(const T* in, long long* out, int64_t n, const long long* tsum) {
  __shared__ long long ws[kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t base = (int64_t)blockIdx.x * kScanTile + warp * kScanWarpSpan;
  long long s = warp_chunk_sum(in, base, n);
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  long long run = tsum[blockIdx.x];
  for (int w = 0; w < warp; w++) run += ws[w];
  for (int r = 0; r < kScanWarpSpan / 32; r++) {
    int64_t i = base + r * 32 + lane;
    long long v = i < n ? (long long)in[i] : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (i < n) out[i] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
}

template <class T>
static void scan_exclusive(Ctx& c, const T* in, int64_t* out, int64_t n, int64_t* tile_tmp) {
  long long* o = reinterpret_cast<long long*>(out);
  long long* t = reinterpret_cast<long long*>(tile_tmp);
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), c.s);
    return;
  }
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  scan_tile_sums<T><<<(unsigned)tiles, kBlock, 0, c.s>>>(in, n, t);
  scan_tile_prefix<<<1, 1024, 0, c.s>>>(t, tiles, o + n);
  scan_tiles<T><<<(unsigned)tiles, kBlock, 0, c.s>>>(in, o, n, t);
  c.launches += 3;
}

void scan_exclusive_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* tile_tmp) {
  scan_exclusive<long long>(c, reinterpret_cast<const long long*>(in), out, n, tile_tmp);
}
void scan_exclusive_i32(Ctx& c, const int32_t* in, int64_t* out, int64_t n, int64_t* tile_tmp) {
  scan_exclusive<int32_t>(c, in, out, n, tile_tmp);
}

// ---------------------------------------------------------------- fills
__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_iota_i32(int32_t* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}
void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n) {
  if (n <= 0) return;
  k_fill_i32<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(p, v, n);
  c.launches++;
}
void iota_i32(Ctx& c, int32_t* p, int64_t n) {
  if (n <= 0) return;
  k_iota_i32<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(p, n);
  c.launches++;
}

// ---------------------------------------------------------------- counting sort by key
// Degree bucket with the run's giant threshold: rows of 2049..4096 arcs go to the 8192-slot block
// kernel, or to the giant path when the threshold is lower.
__device__ __forceinline__ int bucket_of(int64_t deg, int64_t giant_min) {
  int b = degree_bucket(deg);
  if (b == kNumBuckets - 2 && deg > giant_min) b = kNumBuckets - 1;
  return b;
}

__device__ __forceinline__ int sort_key(KeyDesc kd, int64_t i, const int64_t* rbeg, const int64_t* rend,
                                        const int32_t* colour, const int64_t* deg64) {
  if (kd.kind == 2) return bucket_of(deg64[i], kd.giant_min);
  int b = bucket_of(rend[i] - rbeg[i], kd.giant_min);
  if (kd.kind == 0 || b < 0) return b;
  if (kd.kind == 3) {  // hash class of the fast schedule; giant rows optionally all in one class
    const uint64_t h = kd.giant_class >= 0 && b == kNumBuckets - 1
                           ? (uint64_t)kd.giant_class
                           : hash3(kd.seed, (uint64_t)kd.pass, local_id(kd.seg, (int32_t)i));
    return b * kd.classes + (int)(h % (uint64_t)kd.classes);  // bucket-major: classes contiguous per bucket
  }
  return colour[i] * kNumBuckets + b;
}

constexpr int kSmemKeys = 4096;

// Histogram of keys; block-local shared histograms when the key space is small.
__global__ void __launch_bounds__(kBlock) k_key_hist(KeyDesc kind, int64_t n, const int64_t* rbeg, const int64_t* rend,
                                                     const int32_t* colour, const int64_t* deg64, int64_t nkeys,
                                                     int64_t* hist, unsigned long long* max_deg,
                                                     unsigned long long* giant_slots, int64_t n_bound) {
  unsigned long long gs = 0;
  __shared__ int32_t sh[kSmemKeys];
  const bool local = nkeys <= kSmemKeys;
  if (local) {
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) sh[k] = 0;
    __syncthreads();
  }
  long long mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const long long dg = kind.kind == 2 ? deg64[i] : rend[i] - rbeg[i];
    mx = dg > mx ? dg : mx;
    if (giant_slots && bucket_of(dg, kind.giant_min) == kNumBuckets - 1)
      gs += 1ULL << tbl_log2f(dg < n_bound ? dg : n_bound, kind.table_factor, 6, 31);
    int k = sort_key(kind, i, rbeg, rend, colour, deg64);
    if (k < 0) continue;
    if (local) atomicAdd(&sh[k], 1);
    else atomicAdd(reinterpret_cast<unsigned long long*>(&hist[k]), 1ULL);
  }
  if (giant_slots) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
    if ((threadIdx.x & 31) == 0 && gs) atomicAdd(giant_slots, gs);
  }
  if (max_deg) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      long long y = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(max_deg, (unsigned long long)mx);
  }
  if (local) {
    __syncthreads();
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x)
      if (sh[k]) atomicAdd(reinterpret_cast<unsigned long long*>(&hist[k]), (unsigned long long)sh[k]);
  }
}

// Scatter: each block reserves a range per key (one global atomic per key per block), then
// ranks its own elements inside it.  Small key spaces only; large ones use one atomic per element.
__global__ void __launch_bounds__(kBlock) k_key_scatter(KeyDesc kind, int64_t n, const int64_t* rbeg, const int64_t* rend,
                                                        const int32_t* colour, const int64_t* deg64, int64_t nkeys,
                                                        const int64_t* offsets, int32_t* cursor, int32_t* perm) {
  __shared__ int32_t cnt[kSmemKeys];
  __shared__ int64_t basep[kSmemKeys];
  const bool local = nkeys <= kSmemKeys;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // each block processes a contiguous range so the two sweeps below see the same elements
  int64_t per_block = (n + gridDim.x - 1) / gridDim.x;
  int64_t b0 = (int64_t)blockIdx.x * per_block, b1 = b0 + per_block < n ? b0 + per_block : n;
  (void)stride;
  if (!local) {
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      int k = sort_key(kind, i, rbeg, rend, colour, deg64);
      if (k < 0) continue;
      int32_t r = atomicAdd(&cursor[k], 1);
      perm[offsets[k] + r] = (int32_t)i;
    }
    return;
  }
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    int k = sort_key(kind, i, rbeg, rend, colour, deg64);
    if (k >= 0) atomicAdd(&cnt[k], 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nkeys; k += blockDim.x) {
    int32_t m = cnt[k];
    basep[k] = m ? offsets[k] + atomicAdd(&cursor[k], m) : 0;
    cnt[k] = 0;
  }
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    int k = sort_key(kind, i, rbeg, rend, colour, deg64);
    if (k < 0) continue;
    int32_t r = atomicAdd(&cnt[k], 1);
    perm[basep[k] + r] = (int32_t)i;
  }
}

void bucket_sort(Ctx& c, KeyDesc key_kind, int64_t n, const int64_t* rbeg, const int64_t* rend, const int32_t* colour,
                 const int64_t* deg64, int64_t nkeys, int32_t* perm, int64_t* offsets, int32_t* cursor,
                 int64_t* tile_tmp, unsigned long long* max_deg, unsigned long long* giant_slots,
                 int64_t n_bound) {
  key_kind.giant_min = c.giant_min;
  key_kind.table_factor = c.table_factor;
  cudaMemsetAsync(offsets, 0, (size_t)(nkeys + 1) * sizeof(int64_t), c.s);
  cudaMemsetAsync(cursor, 0, (size_t)nkeys * sizeof(int32_t), c.s);
  if (n <= 0) return;
  int grid = grid_for(n, kBlock * 16, c.num_sms * 4);
  k_key_hist<<<grid, kBlock, 0, c.s>>>(key_kind, n, rbeg, rend, colour, deg64, nkeys, offsets, max_deg, giant_slots,
                                       n_bound);
  scan_exclusive_i64(c, offsets, offsets, nkeys, tile_tmp);
  k_key_scatter<<<grid, kBlock, 0, c.s>>>(key_kind, n, rbeg, rend, colour, deg64, nkeys, offsets, cursor, perm);
  c.launches += 2;
}

// ---------------------------------------------------------------- renumbering
__global__ void k_mark(const int32_t* ids, int64_t m, int32_t* occ) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    occ[ids[i]] = 1;
}
void mark_occupied(Ctx& c, const int32_t* ids, int64_t m, int32_t* occ, int64_t n) {
  cudaMemsetAsync(occ, 0, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), c.s);
  if (m <= 0) return;
  k_mark<<<grid_for(m, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(ids, m, occ);
  c.launches++;
}

__global__ void k_relabel(int32_t* ids, int64_t m, const int64_t* newid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    ids[i] = (int32_t)newid[ids[i]];
}
void relabel(Ctx& c, int32_t* ids, int64_t m, const int64_t* newid) {
  if (m <= 0) return;
  k_relabel<<<grid_for(m, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(ids, m, newid);
  c.launches++;
}

__global__ void k_lookup(int32_t* C, int64_t n0, const int32_t* Cp) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x)
    C[v] = Cp[C[v]];
}
void dendrogram_lookup(Ctx& c, int32_t* C, int64_t n0, const int32_t* Cp) {
  if (n0 <= 0) return;
  k_lookup<<<grid_for(n0, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(C, n0, Cp);
  c.launches++;
}

template <class A>
__global__ void k_gather_totals(const A* sig, const int32_t* occ, const int64_t* newid, int64_t n_old, A* k_next) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_old; i += (int64_t)gridDim.x * blockDim.x)
    if (occ[i]) k_next[newid[i]] = sig[i];
}
template <class A>
void gather_totals(Ctx& c, const A* sig, const int32_t* occ, const int64_t* newid, int64_t n_old, A* k_next) {
  if (n_old <= 0) return;
  k_gather_totals<A><<<grid_for(n_old, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(sig, occ, newid, n_old, k_next);
  c.launches++;
}
template void gather_totals<long long>(Ctx&, const long long*, const int32_t*, const int64_t*, int64_t, long long*);
template void gather_totals<double>(Ctx&, const double*, const int32_t*, const int64_t*, int64_t, double*);

__global__ void k_max_i64(const int64_t* p, int64_t n, unsigned long long* out) {
  long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = p[i] > m ? p[i] : m;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, (unsigned long long)m);
}
void max_i64(Ctx& c, const int64_t* p, int64_t n, unsigned long long* out) {
  if (n <= 0) return;
  k_max_i64<<<grid_for(n, kBlock * 8, c.num_sms * 4), kBlock, 0, c.s>>>(p, n, out);
  c.launches++;
}

}  // namespace lv
