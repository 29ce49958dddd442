// dynamic.cu -- dynamic graphs: a batch of edge deletions and insertions applied to a symmetric
// CSR, and the state of a first pass that starts from a given membership (a warm start).
// Within a row of the updated graph the surviving arcs come first, then the inserted ones; the
// order inside each group is unspecified (no step of the method depends on the order of a row).
//
// The paper keeps the first pass's graph in whatever format suits dynamic batch updates
// (Section 4.2) and hands every later pass an initial community membership (Figure 2); its
// Conclusion names updating the memberships of dynamic graphs as the next step.  Here the update
// builds a new CSR in one scan (counts, prefix sum, fill) and the warm start replaces the
// singleton initialisation of pass 0 with the caller's membership.
#include "internal.cuh"

namespace lv {

namespace {

constexpr unsigned long long kNoPair = ~0ull;

__device__ __forceinline__ unsigned long long pair_key(int32_t u, int32_t v) {
  const uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
  return ((unsigned long long)a << 32) | b;
}

__device__ __forceinline__ unsigned pair_home(unsigned long long k, unsigned mask) {
  unsigned long long z = k * 0x9E3779B97F4A7C15ull;
  return (unsigned)(z >> 32) & mask;
}

// Deleted pairs {min, max} into an open-addressing set of `mask + 1` slots (all kNoPair).
__global__ void k_del_insert(const int32_t* du, const int32_t* dv, int64_t n_del, int64_t n_new,
                             unsigned long long* set, unsigned mask, Ctrl* ctrl) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_del; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = du[k], v = dv[k];
    if (u < 0 || u >= n_new || v < 0 || v >= n_new) { atomicAdd(&ctrl->cnt[5], 1ull); continue; }
    const unsigned long long key = pair_key(u, v);
    unsigned s = pair_home(key, mask);
    for (unsigned p = 0; p <= mask; p++) {
      const unsigned long long old = atomicCAS(&set[s], kNoPair, key);
      if (old == kNoPair || old == key) break;
      s = (s + 1) & mask;
    }
  }
}

__device__ __forceinline__ bool is_deleted(const unsigned long long* set, unsigned mask, int32_t u, int32_t v) {
  const unsigned long long key = pair_key(u, v);
  unsigned s = pair_home(key, mask);
  for (unsigned p = 0; p <= mask; p++) {
    const unsigned long long k = set[s];
    if (k == key) return true;
    if (k == kNoPair) return false;
    s = (s + 1) & mask;
  }
  return false;
}

// Row of arc e in [lo, hi] (off[lo] <= e < off[hi + 1]): the last row whose offset is <= e.
__device__ __forceinline__ int64_t row_of(const int64_t* off, int64_t e, int64_t lo, int64_t hi) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Row of arc e given a row lo with off[lo] <= e: gallop forward (rows are mostly short or empty
// runs), then binary search the last bracket.
__device__ __forceinline__ int64_t row_from(const int64_t* off, int64_t e, int64_t lo, int64_t n_old) {
  int64_t step = 1;
  while (lo + step < n_old && off[lo + step] <= e) {
    lo += step;
    step <<= 1;
  }
  const int64_t hi = lo + step - 1 < n_old - 1 ? lo + step - 1 : n_old - 1;
  return row_of(off, e, lo, hi);
}

constexpr int kTileSteps = 16;  // 32-arc steps per warp tile (one binary search per tile)

// Arc-parallel over the old arcs: a warp takes tiles of 16 x 32 consecutive arcs, finds the tile's
// first row by binary search and every later row by galloping from the step's first row; each lane
// tests its arc's pair against the deleted set, and the lanes of one row combine into one atomic --
// a survivor count (FILL = false) or a block of slots taken from the row's cursor (FILL = true), so
// hub rows spread over the whole grid.
template <bool FILL>
__global__ void __launch_bounds__(kBlock) k_arcs(int64_t n_old, int64_t n_arcs, const int64_t* off, const int32_t* tg,
                                                 const uint32_t* w, const unsigned long long* set, unsigned mask,
                                                 bool any_del, unsigned long long* cnt, const int64_t* out_off,
                                                 int32_t* otg, uint32_t* ow) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  constexpr int64_t kTile = 32 * kTileSteps;
  for (int64_t tile = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kTile; tile < n_arcs;
       tile += warps * kTile) {
    int64_t rcur = 0;
    if (lane == 0) rcur = row_of(off, tile, 0, n_old - 1);
    rcur = __shfl_sync(0xffffffffu, rcur, 0);
    for (int k = 0; k < kTileSteps; k++) {
      const int64_t base = tile + (int64_t)k * 32;
      if (base >= n_arcs) break;
      if (k > 0) {
        int64_t r0 = 0;
        if (lane == 0) r0 = row_from(off, base, rcur, n_old);
        rcur = __shfl_sync(0xffffffffu, r0, 0);
      }
      const int64_t e = base + lane;
      int64_t r = -1;
      bool keep = false;
      int32_t t = 0;
      if (e < n_arcs) {
        r = row_from(off, e, rcur, n_old);
        t = tg[e];
        keep = !any_del || !is_deleted(set, mask, (int32_t)r, t);
      }
      const unsigned keepers = __ballot_sync(0xffffffffu, keep);
      const unsigned peers = __match_any_sync(0xffffffffu, keep ? r : (int64_t)-1) & keepers;
      if (keep) {
        const int leader = __ffs(peers) - 1;
        const unsigned below = peers & ((1u << lane) - 1u);
        unsigned long long slot0 = 0;
        if (lane == leader) slot0 = atomicAdd(&cnt[r], (unsigned long long)__popc(peers));
        if (FILL) {
          slot0 = __shfl_sync(peers, slot0, leader);
          const int64_t pos = out_off[r] + (int64_t)slot0 + __popc(below);
          otg[pos] = t;
          ow[pos] = w[e];
        }
      }
    }
  }
}

// Inserted arcs: per edge (u, v, w) the arc u->v and, for u != v, v->u.
template <bool FILL>
__global__ void k_ins(const int32_t* iu, const int32_t* iv, const uint32_t* iw, int64_t n_ins, int64_t n_new,
                      unsigned long long* cnt, const int64_t* out_off, int32_t* otg, uint32_t* ow, Ctrl* ctrl) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_ins; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = iu[k], v = iv[k];
    if (u < 0 || u >= n_new || v < 0 || v >= n_new) {
      if (!FILL) atomicAdd(&ctrl->cnt[5], 1ull);
      continue;
    }
    for (int side = 0; side < (u != v ? 2 : 1); side++) {
      const int32_t a = side ? v : u, b = side ? u : v;
      const unsigned long long slot = atomicAdd(&cnt[a], 1ull);
      if (FILL) {
        const int64_t pos = out_off[a] + (int64_t)slot;
        otg[pos] = b;
        ow[pos] = iw[k];
      }
    }
  }
}

template <class A>
__global__ void k_warm_clear(A* Sig, int32_t* csize, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Sig[i] = A(0);
    csize[i] = 0;
  }
}

template <class A>
__global__ void k_warm_set(const int32_t* init, const A* K, A* Sig, int32_t* Cp, int32_t* csize, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = init[i];
    Cp[i] = c;
    atomic_add_a(&Sig[c], K[i]);
    atomicAdd(&csize[c], 1);
  }
}

}  // namespace

int64_t update_scratch_words(int64_t n_new, int64_t n_del) {
  int64_t slots = 1;
  while (slots < 2 * n_del + 2) slots <<= 1;
  return slots + n_new + 1;
}

int update_count(Ctx& c, int64_t n_old, int64_t arcs_of, const int64_t* off, const int32_t* tg, int64_t n_new,
                 const int32_t* du,
                 const int32_t* dv, int64_t n_del, const int32_t* iu, const int32_t* iv, const void* iw,
                 int64_t n_ins, unsigned long long* scratch, int64_t* out_off, int64_t* tile_tmp, Ctrl* ctrl) {
  unsigned slots = 1;
  while (slots < 2 * n_del + 2) slots <<= 1;
  unsigned long long* set = scratch;
  int64_t* cnt = reinterpret_cast<int64_t*>(scratch + slots);
  cudaMemsetAsync(set, 0xff, (size_t)slots * sizeof(unsigned long long), c.s);
  cudaMemsetAsync(cnt, 0, (size_t)(n_new + 1) * sizeof(int64_t), c.s);
  const int cap = c.num_sms * 8;
  if (n_del > 0) {
    k_del_insert<<<grid_for(n_del, kBlock, cap), kBlock, 0, c.s>>>(du, dv, n_del, n_new, set, slots - 1, ctrl);
    c.launches++;
  }
  const int64_t n_arcs = n_old > 0 ? arcs_of : 0;
  if (n_arcs > 0) {
    k_arcs<false><<<grid_for(n_arcs, kBlock * kTileSteps, cap * 2), kBlock, 0, c.s>>>(
        n_old, n_arcs, off, tg, nullptr, set, slots - 1, n_del > 0, reinterpret_cast<unsigned long long*>(cnt),
        nullptr, nullptr, nullptr);
    c.launches++;
  }
  if (n_ins > 0) {
    k_ins<false><<<grid_for(n_ins, kBlock, cap), kBlock, 0, c.s>>>(
        iu, iv, reinterpret_cast<const uint32_t*>(iw), n_ins, n_new, reinterpret_cast<unsigned long long*>(cnt),
        nullptr, nullptr, nullptr, ctrl);
    c.launches++;
  }
  scan_exclusive_i64(c, cnt, out_off, n_new, tile_tmp);
  return (int)slots;
}

void update_fill(Ctx& c, int64_t n_old, int64_t arcs_of, const int64_t* off, const int32_t* tg, const void* w,
                 int64_t n_new,
                 int64_t n_del, const int32_t* iu, const int32_t* iv, const void* iw, int64_t n_ins,
                 unsigned long long* scratch, unsigned slots, const int64_t* out_off, int32_t* otg, void* ow,
                 Ctrl* ctrl) {
  int64_t* cnt = reinterpret_cast<int64_t*>(scratch + slots);
  cudaMemsetAsync(cnt, 0, (size_t)(n_new + 1) * sizeof(int64_t), c.s);
  const int cap = c.num_sms * 8;
  const int64_t n_arcs = n_old > 0 ? arcs_of : 0;
  if (n_arcs > 0) {
    k_arcs<true><<<grid_for(n_arcs, kBlock * kTileSteps, cap * 2), kBlock, 0, c.s>>>(
        n_old, n_arcs, off, tg, reinterpret_cast<const uint32_t*>(w), scratch, slots - 1, n_del > 0,
        reinterpret_cast<unsigned long long*>(cnt), out_off, otg, reinterpret_cast<uint32_t*>(ow));
    c.launches++;
  }
  if (n_ins > 0) {
    k_ins<true><<<grid_for(n_ins, kBlock, cap), kBlock, 0, c.s>>>(
        iu, iv, reinterpret_cast<const uint32_t*>(iw), n_ins, n_new, reinterpret_cast<unsigned long long*>(cnt),
        out_off, otg, reinterpret_cast<uint32_t*>(ow), ctrl);
    c.launches++;
  }
}

template <class M>
void warm_init(Ctx& c, const PassState<M>& st, const int32_t* init, int64_t n) {
  if (n <= 0) return;
  const int grid = grid_for(n, kBlock, c.num_sms * 8);
  k_warm_clear<typename M::a_t><<<grid, kBlock, 0, c.s>>>(st.Sig, st.csize, n);
  k_warm_set<typename M::a_t><<<grid, kBlock, 0, c.s>>>(init, st.K, st.Sig, st.Cp, st.csize, n);
  c.launches += 2;
}

template void warm_init<IntMode>(Ctx&, const PassState<IntMode>&, const int32_t*, int64_t);
template void warm_init<FpMode>(Ctx&, const PassState<FpMode>&, const int32_t*, int64_t);

}  // namespace lv
