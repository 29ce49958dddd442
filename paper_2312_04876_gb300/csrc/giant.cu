// giant.cu -- the multi-block path for giant rows (the last degree bucket: rows longer than the giant threshold, 4096 arcs by default).
//
// A hub vertex (R-MAT hubs reach 10^5 arcs) or a giant community (10^6-10^7 member arcs after a
// pass) handled by one block serialises a whole launch on one SM.  Here the work of a giant is cut
// into arc chunks and table slices that every SM shares:
//   plan    per giant its chunk count, table size (a power of two >= 2 x its distinct-key bound)
//           and slice count; a one-block scan gives each giant its chunk / slot / slice range in a
//           shared pool of global-memory tables; owner arrays map every chunk and slice back to its
//           giant (binary search, fully parallel).  The local-moving plan covers every giant of a
//           pass at once (the giants listed class by class), so it is built once per pass; each
//           iteration of a class only decides which of its giants are active (pruning flags);
//   insert  grid-stride over chunks of 512 arcs (local move) or 2048 arcs (merge): K_i->c into the
//           giant's global table with L2 atomics, K_i->d in registers (scanCommunities).  The
//           local-moving steps of a pass run one after another and each leaves its tables empty,
//           so every step lays its giants' tables out from the start of the pool: a step of one
//           class touches a few tens of MB that stay in L2 from step to step, not a fresh region
//           of a pool sized for the whole pass;
//   scan    one warp per range of 1024 table slots, one word of the pool's occupancy bitmap per
//           lane (an insert that claims a slot sets its bit), so only occupied slots are read:
//           local move scores every candidate with the Eq. 2 numerator and keeps the range's best;
//           merge emits the range's (community, weight) pairs into the holey row of the community.
//           Every occupied slot and bit is cleared, so the pool is all-empty between uses;
//   decide  (local move) per giant: best over its ranges, then the move exactly as the per-vertex
//           kernels make it;
//   mark    (local move, pruning) grid-stride over chunks of the giants that moved.
// Merges cut the concatenated member rows of each giant community (community-vertex CSR order)
// into chunks taken community after community, so a community's arcs spread over the GPU however
// its members are shaped, while the blocks in flight touch the tables of only a few communities.
#include "internal.cuh"

namespace lv {

constexpr int kChunk = 2048;    // arcs per chunk (merge, modularity, compaction)
constexpr int kLmChunk = 512;   // arcs per chunk of the local-moving phase (2 per thread)
constexpr int kSliceLog = 10;   // merge: 1024 table slots (32 bitmap words) per slice
constexpr int kRangeLog = 10;   // local move: 1024 table slots (32 bitmap words) per warp range
constexpr int kLocLog = 12;     // shared pre-aggregation table: 4096 slots >= 2 x kChunk keys

// ---------------------------------------------------------------- plan
// kind 0: local move, item = vertex list[k]: table for min(deg, n_bound) keys, chunks over its row;
// kind 1: merge, item = community list[k]: table for min(cdeg, n_bound) keys, chunks over the
//         concatenated rows of its members; gix[c] = k;
// kind 2: chunks only, item = vertex list[k] whose community Cp[i] >= 0 is giant (gix >= 0);
// kind 3: chunks only, every listed row.
__global__ void k_gplan_counts(int kind, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                               const int64_t* cdeg, int64_t n_bound, const int32_t* Cp, int32_t* gix, int slice_log,
                               GiantPlan p, int tf) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[k];
    int64_t nch = 0, ts = 0;
    if (kind == 1) {
      const int64_t bound = cdeg[v] < n_bound ? cdeg[v] : n_bound;
      ts = (int64_t)1 << tbl_log2f(bound, tf, 6, 31);
      nch = (cdeg[v] + kChunk - 1) / kChunk;
      gix[v] = (int32_t)k;
    } else {
      const int64_t deg = rend[v] - rbeg[v];
      const bool used = kind != 2 || (Cp[v] >= 0 && gix[Cp[v]] >= 0);
      if (used) {
        const int64_t ch = kind == 0 ? kLmChunk : kChunk;
        nch = (deg + ch - 1) / ch;
        if (kind == 0) ts = (int64_t)1 << tbl_log2f(deg < n_bound ? deg : n_bound, tf, 6, 31);
      }
    }
    p.chunk_off[k] = nch;
    p.tab_off[k] = ts;
    p.slice_off[k] = (ts + ((int64_t)1 << slice_log) - 1) >> slice_log;
    reinterpret_cast<uint32_t*>(p.kid)[k] = 0u;  // 0u is also 0.0f
    p.moved[k] = 0;
    p.active[k] = 0;
  }
}

// Exclusive scans of the three counts (one block); totals at [m].  A plan that does not fit the
// capacities runs nothing (chunk and slice totals read 0) and reports the error.
__global__ void __launch_bounds__(1024) k_gplan_scan(int64_t m, GiantPlan p, Ctrl* ctrl) {
  __shared__ int64_t part[3][1024];
  const int t = threadIdx.x;
  const int64_t per = (m + 1023) / 1024;
  const int64_t b = t * per, e = b + per < m ? b + per : m;
  int64_t sc = 0, st = 0, ss = 0;
  for (int64_t k = b; k < e; k++) { sc += p.chunk_off[k]; st += p.tab_off[k]; ss += p.slice_off[k]; }
  part[0][t] = sc; part[1][t] = st; part[2][t] = ss;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int64_t v0 = t >= o ? part[0][t - o] : 0, v1 = t >= o ? part[1][t - o] : 0, v2 = t >= o ? part[2][t - o] : 0;
    __syncthreads();
    part[0][t] += v0; part[1][t] += v1; part[2][t] += v2;
    __syncthreads();
  }
  const int64_t tot_c = part[0][1023], tot_t = part[1][1023], tot_s = part[2][1023];
  const bool fits = tot_c <= p.chunk_cap && tot_s <= p.slice_cap && tot_t <= p.pool_slots;
  int64_t rc = t ? part[0][t - 1] : 0, rt = t ? part[1][t - 1] : 0, rs = t ? part[2][t - 1] : 0;
  for (int64_t k = b; k < e; k++) {
    const int64_t nch = p.chunk_off[k], ts = p.tab_off[k], ns = p.slice_off[k];
    // an over-full plan gets empty ranges everywhere, so no kernel touches a chunk or slice
    p.chunk_off[k] = fits ? rc : 0; p.tab_off[k] = rt; p.slice_off[k] = fits ? rs : 0;
    rc += nch; rt += ts; rs += ns;
  }
  if (t == 1023) {
    p.chunk_off[m] = fits ? tot_c : 0;
    p.tab_off[m] = tot_t;
    p.slice_off[m] = fits ? tot_s : 0;
    if (!fits) atomicOr(&ctrl->error, kErrTableFull);
  }
}

// Largest k in [0, m) with off[k] <= q (the item whose range holds q).
__device__ __forceinline__ int32_t owner_of(const int64_t* off, int64_t m, int64_t q) {
  int64_t lo = 0, hi = m;  // off[lo] <= q < off[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= q) lo = mid; else hi = mid;
  }
  return (int32_t)lo;
}

__global__ void k_gplan_owners(int64_t m, GiantPlan p) {
  const int64_t nc = p.chunk_off[m], ns = p.slice_off[m];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += stride)
    p.cowner[q] = owner_of(p.chunk_off, m, q);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += stride)
    p.sowner[q] = owner_of(p.slice_off, m, q);
}

void giant_plan(Ctx& c, int kind, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                const int64_t* cdeg, int64_t n_bound, const int32_t* Cp, int32_t* gix, int slice_log,
                const GiantPlan& p, Ctrl* ctrl) {
  const int cap = c.num_sms * 8;
  k_gplan_counts<<<grid_for(m, kBlock, cap), kBlock, 0, c.s>>>(kind, list, m, rbeg, rend, cdeg, n_bound, Cp, gix,
                                                              slice_log, p, c.table_factor);
  k_gplan_scan<<<1, 1024, 0, c.s>>>(m, p, ctrl);
  k_gplan_owners<<<cap, kBlock, 0, c.s>>>(m, p);
  c.launches += 3;
}

// Pool slots: slot s of a table at pool offset `base` is the pair {key, value} at kv[2s], kv[2s + 1]
// (kv = pool + 2 base), so a probe, its claim and its add touch one 32-byte sector.
__global__ void k_pool_init(int2* kv, int64_t n) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    kv[s] = make_int2(kEmpty, 0);  // value 0 is 0u and 0.0f
}
void pool_init(Ctx& c, int32_t* slots, int64_t n) {
  if (n <= 0) return;
  k_pool_init<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(reinterpret_cast<int2*>(slots), n);
  c.launches++;
}

template <class V>
__device__ __forceinline__ V* slot_val(int32_t* kv, unsigned s) {
  return reinterpret_cast<V*>(&kv[2 * (size_t)s + 1]);
}

// tbl_add for a giant's table (kv, at pool offset `base`) that also sets the slot's bit in the
// pool's occupancy bitmap when it claims the slot, so the scan visits only occupied slots.
// Probing starts at slot s (the key's home) whose key was already read as k0.
// An empty slot is claimed together with its first value by one 64-bit compare-and-swap of the
// pair ({kEmpty, 0} -> {key, w}); a slot that holds the key gets an add.
template <class V>
__device__ __forceinline__ bool tbl_add_mark_at(int32_t* kv, unsigned size, int32_t key, V w, unsigned* bits,
                                                int64_t base, unsigned s, int32_t k0) {
  const unsigned long long mine = ((unsigned long long)val_bits<V>(w) << 32) | (uint32_t)key;
  for (unsigned p = 0; p < size; p++) {
    const int32_t k = p == 0 ? k0 : *((volatile int32_t*)&kv[2 * (size_t)s]);
    if (k == key) { atomicAdd(slot_val<V>(kv, s), w); return true; }
    if (k == kEmpty) {
      const unsigned long long old =
          atomicCAS(reinterpret_cast<unsigned long long*>(&kv[2 * (size_t)s]), kEmptyPair, mine);
      if (old == kEmptyPair) {
        atomicOr(&bits[(base + s) >> 5], 1u << ((base + s) & 31));
        return true;
      }
      if ((int32_t)(uint32_t)old == key) { atomicAdd(slot_val<V>(kv, s), w); return true; }
    }
    s = (s + 1) & (size - 1);
  }
  return false;
}

template <class V>
__device__ __forceinline__ bool tbl_add_mark(int32_t* kv, unsigned size, int shift, int32_t key, V w, unsigned* bits,
                                             int64_t base) {
  const unsigned s = tbl_home(key, shift);
  return tbl_add_mark_at(kv, size, key, w, bits, base, s, *((volatile int32_t*)&kv[2 * (size_t)s]));
}

// ---------------------------------------------------------------- shared pre-aggregation
// Sums a chunk's (key, weight) pairs in the block's shared table, then flushes each distinct key
// once into the global table (kv, size 2^lg).  Every thread of the block must call both.
template <class H>
struct LocalAgg {
  int32_t keys[1 << kLocLog];
  H vals[1 << kLocLog];
};

template <class H>
__device__ __forceinline__ void local_clear(LocalAgg<H>& la) {
  for (int s = threadIdx.x; s < (1 << kLocLog); s += kBlock) { la.keys[s] = kEmpty; la.vals[s] = H(0); }
}

template <class H>
__device__ __forceinline__ bool local_flush(LocalAgg<H>& la, int32_t* kv, unsigned size, int lg, unsigned* bits,
                                            int64_t base) {
  bool ok = true;
  __syncthreads();
  // V slots per thread per round: the home-slot reads of the V keys are issued together
  constexpr int V = 4;
  for (int s0 = threadIdx.x; s0 < (1 << kLocLog); s0 += kBlock * V) {
    int32_t key[V], seen[V];
    H val[V];
    unsigned home[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
      const int s = s0 + v * kBlock;
      key[v] = la.keys[s];
      val[v] = la.vals[s];
      if (key[v] != kEmpty) {
        la.keys[s] = kEmpty;
        la.vals[s] = H(0);
      }
    }
#pragma unroll
    for (int v = 0; v < V; v++) {
      home[v] = tbl_home(key[v], 32 - lg);
      seen[v] = key[v];
      if (key[v] != kEmpty) seen[v] = *((volatile int32_t*)&kv[2 * (size_t)home[v]]);
    }
#pragma unroll
    for (int v = 0; v < V; v++)
      if (key[v] != kEmpty) ok &= tbl_add_mark_at(kv, size, key[v], val[v], bits, base, home[v], seen[v]);
  }
  __syncthreads();
  return ok;
}

// A captured iteration passes its giant range (list offset, k0, k1) in device memory; eager
// launches pass it as arguments (krng null).
__device__ __forceinline__ void giant_range(const int64_t* krng, const int32_t*& list, int64_t& k0, int64_t& k1) {
  if (krng) {
    list += krng[0];
    k0 = krng[1];
    k1 = krng[2];
  }
}

// ---------------------------------------------------------------- local move: activation
// Giants [k0, k1) of the class: active iff their graph has not converged and (pruning) their flag
// is set, which is then cleared (processed).  Also resets K_i->d and the moved marks, and counts
// list entries / processed vertices / arcs.
template <class W>
__global__ void k_glm_activate(GraphView<W> g, const int32_t* list, int64_t k0, int64_t k1, uint8_t* flags,
                               int pruning, const GraphCtl* gc, const int32_t* vg, GiantPlan p, Ctrl* ctrl,
                               const int64_t* krng) {
  if (*(volatile int32_t*)&ctrl->done) return;
  giant_range(krng, list, k0, k1);
  unsigned long long act = 0, arcs = 0;
  for (int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < k1; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = list[k];
    bool a = !(gc && gc[vg[v]].done);
    if (a && pruning) {
      a = flags[v] != 0;
      if (a) flags[v] = 0;
    }
    p.active[k] = a ? 1 : 0;
    p.moved[k] = 0;
    reinterpret_cast<uint32_t*>(p.kid)[k] = 0u;
    if (a) { act++; arcs += (unsigned long long)(g.rend[v] - g.rbeg[v]); }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    act += __shfl_xor_sync(0xffffffffu, act, o);
    arcs += __shfl_xor_sync(0xffffffffu, arcs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][0], (unsigned long long)(k1 - k0));
    if (act) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][1], act);
    if (arcs) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][2], arcs);
  }
}

// Where a giant's activity comes from: fast mode snapshots it in k_glm_activate (a neighbour in the
// same random class may re-mark the giant while its step runs); the deterministic mode reads it
// from the flags directly in every kernel of the step -- a colour class is an independent set, so
// nothing marks one of its giants during the step -- and its decide kernel then does what the
// activation did (clears the flag, resets K_i->d, sets the moved mark, counts), one launch fewer.
struct GiantAct {
  int snap = 1;                  // 1: p.active (fast); 0: read below (deterministic)
  int pruning = 0;
  const uint8_t* flags = nullptr;
  const GraphCtl* gc = nullptr;
  const int32_t* vg = nullptr;
};
__device__ __forceinline__ bool giant_active(const GiantAct& ga, const GiantPlan& p, int64_t k, int32_t v) {
  if (ga.snap) return p.active[k] != 0;
  if (ga.gc && *(const volatile int32_t*)&ga.gc[ga.vg[v]].done) return false;
  return !ga.pruning || ga.flags[v] != 0;
}

// ---------------------------------------------------------------- local move: insert

// One block per chunk of an active giant; each thread loads its U arcs before their C'[j] gathers
// and table updates (U memory requests in flight per thread).
template <class M>
__global__ void __launch_bounds__(kBlock) k_glm_insert(GraphView<typename M::w_t> g, const int32_t* list, int64_t k0,
                                                       int64_t k1, const int32_t* Cp, GiantPlan p, Ctrl* ctrl,
                                                       const int64_t* krng, GiantAct ga) {
  typedef typename M::h_t H;
  constexpr int U = kLmChunk / kBlock;  // 2
  __shared__ H red[32];
  if (*(volatile int32_t*)&ctrl->done) return;
  giant_range(krng, list, k0, k1);
  const int64_t q0 = p.chunk_off[k0], q1 = p.chunk_off[k1];
  bool ok = true;
  for (int64_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    const int32_t i = list[k];
    if (!giant_active(ga, p, k, i)) continue;  // uniform over the block
    const int32_t d = Cp[i];
    const int64_t ts = p.tab_off[k + 1] - p.tab_off[k];
    const int64_t off = p.tab_off[k] - p.tab_off[k0];  // the step's tables from the pool's start
    int lg = 0;
    while (((int64_t)1 << lg) < ts) lg++;
    int32_t* kv = p.slots + 2 * off;
    const int64_t e0 = g.rbeg[i] + (q - p.chunk_off[k]) * kLmChunk;
    const int64_t e1 = e0 + kLmChunk < g.rend[i] ? e0 + kLmChunk : g.rend[i];
    int32_t jj[U];
    H ww[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t e = e0 + threadIdx.x + (int64_t)u * kBlock;
      jj[u] = e < e1 ? g.tg[e] : i;
      ww[u] = e < e1 ? (H)g.w[e] : H(0);
    }
    int32_t cc[U];
#pragma unroll
    for (int u = 0; u < U; u++) cc[u] = jj[u] != i ? Cp[jj[u]] : kEmpty;
    H kid = H(0);
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (jj[u] == i) continue;
      if (cc[u] == d) kid += ww[u];
      else ok &= tbl_add_mark(kv, (unsigned)ts, 32 - lg, cc[u], ww[u], p.bits, off);
    }
    kid = group_sum<kBlock>(kid, red);
    if (threadIdx.x == 0 && kid != H(0)) atomicAdd(reinterpret_cast<H*>(p.kid) + k, kid);
  }
  if (!ok) atomicOr(&ctrl->error, kErrTableFull);
}

// ---------------------------------------------------------------- local move: range scan
// One warp per range of 1024 slots of an active giant's table: each lane reads one word of the
// occupancy bitmap and visits only its occupied slots (key, value and Sigma loads of up to four
// slots issued together), clearing slots and bits.  Writes the range's best to part_s/c.
template <class M>
__global__ void __launch_bounds__(kBlock) k_glm_scan(const int32_t* list, int64_t k0, int64_t k1, const int32_t* Cp,
                                                     const typename M::a_t* K, const typename M::a_t* Sig,
                                                     GiantPlan p, Ctrl* ctrl, const GraphCtl* gc, const int32_t* vg,
                                                     const int64_t* krng, GiantAct ga) {
  typedef typename M::h_t H;
  typedef typename M::a_t A;
  typedef typename M::s_t S;
  if (*(volatile int32_t*)&ctrl->done) return;
  giant_range(krng, list, k0, k1);
  const int64_t r0 = p.slice_off[k0], r1 = p.slice_off[k1];
  const A two_m_all = M::is_fp ? (A)ctrl->two_m_f : (A)ctrl->two_m_i;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  unsigned long long cand = 0;
  for (int64_t q = r0 + (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); q < r1; q += nwarps) {
    const int64_t k = p.sowner[q];
    const int32_t i = list[k];
    if (!giant_active(ga, p, k, i)) continue;  // uniform over the warp
    const int32_t d = Cp[i];
    const int64_t ts = p.tab_off[k + 1] - p.tab_off[k];
    const int64_t off = p.tab_off[k] - p.tab_off[k0];  // as the insert placed them
    const H kid = reinterpret_cast<const H*>(p.kid)[k];
    const A ki = K[i], sd = Sig[d];
    const A two_m = gc ? (M::is_fp ? (A)gc[vg[i]].two_m_f : (A)gc[vg[i]].two_m_i) : two_m_all;
    int2* kv = reinterpret_cast<int2*>(p.slots) + off;
    // the range's bitmap words, one per lane (tables are >= 64 slots and 64-slot aligned)
    const int64_t sb = (q - p.slice_off[k]) << kRangeLog;
    const int64_t se = sb + (1 << kRangeLog) < ts ? sb + (1 << kRangeLog) : ts;
    const int nwords = (int)((se - sb) >> 5);
    unsigned* wp = p.bits + ((off + sb) >> 5) + lane;
    unsigned word = lane < nwords ? *wp : 0u;
    if (word) *wp = 0u;
    S best = M::lowest();
    int32_t bc = 0x7fffffff;
    const int64_t s0 = sb + 32 * lane;
    while (word) {
      // up to 4 occupied slots at a time: their key, value and Sigma loads are issued together
      int64_t ss[4];
      int nb = 0;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        ss[u] = -1;
        if (word) {
          ss[u] = s0 + (__ffs(word) - 1);
          word &= word - 1;
          nb++;
        }
      }
      int32_t ks[4];
      H vv[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int2 e = ss[u] >= 0 ? kv[ss[u]] : make_int2(kEmpty, 0);  // key and value: one 8-byte load
        ks[u] = e.x;
        vv[u] = int_as_h<H>(e.y);
      }
      A sg[4];
#pragma unroll
      for (int u = 0; u < 4; u++) sg[u] = ks[u] != kEmpty ? Sig[ks[u]] : A(0);
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (ss[u] < 0) continue;
        kv[ss[u]] = make_int2(kEmpty, 0);
        cand++;
        const S sc = M::score(vv[u], kid, ki, sg[u], sd, two_m);
        if (better(sc, ks[u], best, bc)) { best = sc; bc = ks[u]; }
      }
      (void)nb;
    }
    group_argmax<32>(best, bc, (S*)nullptr, (int32_t*)nullptr);
    if (lane == 0) {
      reinterpret_cast<S*>(p.part_s)[q] = best;
      p.part_c[q] = bc;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, o);
  if ((threadIdx.x & 31) == 0 && cand) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][3], cand);
}

// ---------------------------------------------------------------- local move: decide (+ apply)
template <class M>
__global__ void __launch_bounds__(kBlock) k_glm_decide(GraphView<typename M::w_t> g, const int32_t* list, int64_t k0,
                                                       int64_t k1, PassState<M> st, GiantPlan p, int fast,
                                                       const int64_t* krng, GiantAct ga) {
  typedef typename M::a_t A;
  typedef typename M::s_t S;
  Ctrl* ctrl = st.ctrl;
  if (*(volatile int32_t*)&ctrl->done) return;
  giant_range(krng, list, k0, k1);
  unsigned long long acc_lo = 0, acc_hi = 0, acc_mv = 0;
  double acc_f = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
  unsigned long long n_act = 0, n_arcs = 0;  // deterministic mode: the activation's counts
  for (int64_t k = k0 + (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); k < k1; k += nw) {
    const int32_t iv = list[k];
    // lane 0's reading for the whole warp, taken before lane 0 clears the flag below
    const bool act = __shfl_sync(0xffffffffu, giant_active(ga, p, k, iv) ? 1 : 0, 0) != 0;
    if (!ga.snap && lane == 0) {
      // what k_glm_activate does in fast mode, now that every kernel of the step has read the flag
      p.moved[k] = 0;
      reinterpret_cast<uint32_t*>(p.kid)[k] = 0u;  // (scan has read it) for the next use of the plan
      if (act) {
        if (ga.pruning) st.flags[iv] = 0;
        n_act++;
        n_arcs += (unsigned long long)(g.rend[iv] - g.rbeg[iv]);
      }
    }
    if (!act) continue;
    const int64_t q0 = p.slice_off[k], q1 = p.slice_off[k + 1];
    S best = M::lowest();
    int32_t bc = 0x7fffffff;
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const S s = reinterpret_cast<const S*>(p.part_s)[q];
      const int32_t c = p.part_c[q];
      if (better(s, c, best, bc)) { best = s; bc = c; }
    }
    group_argmax<32>(best, bc, (S*)nullptr, (int32_t*)nullptr);
    if (lane != 0) continue;
    const int32_t i = list[k];
    const int32_t d = st.Cp[i];
    if (bc == 0x7fffffff || !(best > S(0))) continue;
    if (fast && st.csize[d] == 1 && st.csize[bc] == 1 && bc > d) continue;
    const A ki = st.K[i];
    if (fast) {
      atomic_add_a(&st.Sig[d], -ki);
      atomic_add_a(&st.Sig[bc], ki);
      atomicSub(&st.csize[d], 1);
      atomicAdd(&st.csize[bc], 1);
    } else {
      st.mv_from[i] = d;
      st.mv_to[i] = bc;
    }
    st.Cp[i] = bc;
    p.moved[k] = 1;
    if (st.gc) {
      GraphCtl* gcv = st.gc + st.vg[i];
      if (M::is_fp) atomicAdd(&gcv->sum_f, (double)best);
      else atomic_add_u128(&gcv->sum_lo, &gcv->sum_hi, (unsigned long long)best, 0ULL);
    } else if (M::is_fp) {
      acc_f += (double)best;
    } else {
      const unsigned long long b = (unsigned long long)best;
      acc_lo += b;
      if (acc_lo < b) acc_hi++;
    }
    acc_mv++;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, acc_lo, o), hi2 = __shfl_xor_sync(0xffffffffu, acc_hi, o);
    unsigned long long s = acc_lo + lo2;
    acc_hi += hi2 + (s < acc_lo ? 1ULL : 0ULL);
    acc_lo = s;
    acc_mv += __shfl_xor_sync(0xffffffffu, acc_mv, o);
    if (M::is_fp) acc_f += __shfl_xor_sync(0xffffffffu, acc_f, o);
  }
  if (lane == 0 && acc_mv) {
    atomicAdd(&ctrl->moves, acc_mv);
    atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][4], acc_mv);
    if (M::is_fp) atomicAdd(&ctrl->sum_f, acc_f);
    else atomic_add_u128(&ctrl->sum_lo, &ctrl->sum_hi, acc_lo, acc_hi);
  }
  if (!ga.snap) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      n_act += __shfl_xor_sync(0xffffffffu, n_act, o);
      n_arcs += __shfl_xor_sync(0xffffffffu, n_arcs, o);
    }
    if (lane == 0) {
      if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][0], (unsigned long long)(k1 - k0));
      if (n_act) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][1], n_act);
      if (n_arcs) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][2], n_arcs);
    }
  }
}

// ---------------------------------------------------------------- local move: mark neighbours
template <class W>
__global__ void __launch_bounds__(kBlock) k_glm_mark(GraphView<W> g, const int32_t* list, int64_t k0, int64_t k1,
                                                     uint8_t* flags, GiantPlan p, Ctrl* ctrl, const int64_t* krng) {
  constexpr int U = kLmChunk / kBlock;
  if (*(volatile int32_t*)&ctrl->done) return;
  giant_range(krng, list, k0, k1);
  const int64_t q0 = p.chunk_off[k0], q1 = p.chunk_off[k1];
  unsigned long long marks = 0;
  for (int64_t q = q0 + blockIdx.x; q < q1; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    if (!p.moved[k]) continue;
    const int32_t i = list[k];
    const int64_t e0 = g.rbeg[i] + (q - p.chunk_off[k]) * kLmChunk;
    const int64_t e1 = e0 + kLmChunk < g.rend[i] ? e0 + kLmChunk : g.rend[i];
    int32_t jj[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t e = e0 + threadIdx.x + (int64_t)u * kBlock;
      jj[u] = e < e1 ? g.tg[e] : i;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (jj[u] != i) { flags[jj[u]] = 1; marks++; }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) marks += __shfl_xor_sync(0xffffffffu, marks, o);
  if ((threadIdx.x & 31) == 0 && marks) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][5], marks);
}

template <class M>
void giant_move_plan(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* list, int64_t m, const GiantPlan& p,
                     Ctrl* ctrl) {
  if (m <= 0) return;
  giant_plan(c, 0, list, m, g.rbeg, g.rend, nullptr, g.n, nullptr, nullptr, kRangeLog, p, ctrl);
}

template <class M>
void giant_move(Ctx& c, const GraphView<typename M::w_t>& g, const PassState<M>& st, const int32_t* list, int64_t k0,
                int64_t k1, const GiantPlan& p, bool fast, bool pruning, const int64_t* krng) {
  if (k1 <= k0 && !krng) return;
  const int grid = c.num_sms * (c.lm_blocks_per_sm < 8 ? c.lm_blocks_per_sm : 8);
  // a device-resident range has no host count: the per-giant kernels take their cap
  const int ga = krng ? c.num_sms * 2 : grid_for(k1 - k0, kBlock, c.num_sms * 2);
  const int gd = krng ? c.num_sms * 2 : grid_for(k1 - k0, kBlock / 32, c.num_sms * 2);
  GiantAct act;
  act.snap = fast ? 1 : 0;
  act.pruning = pruning ? 1 : 0;
  act.flags = st.flags;
  act.gc = st.gc;
  act.vg = st.vg;
  if (fast) {
    k_glm_activate<typename M::w_t><<<ga, kBlock, 0, c.s>>>(g, list, k0, k1, st.flags, pruning ? 1 : 0, st.gc, st.vg,
                                                            p, st.ctrl, krng);
    c.launches++;
  }
  k_glm_insert<M><<<grid, kBlock, 0, c.s>>>(g, list, k0, k1, st.Cp, p, st.ctrl, krng, act);
  k_glm_scan<M><<<grid, kBlock, 0, c.s>>>(list, k0, k1, st.Cp, st.K, st.Sig, p, st.ctrl, st.gc, st.vg, krng, act);
  k_glm_decide<M><<<gd, kBlock, 0, c.s>>>(g, list, k0, k1, st, p, fast ? 1 : 0, krng, act);
  c.launches += 3;
  if (pruning) {
    k_glm_mark<typename M::w_t><<<grid, kBlock, 0, c.s>>>(g, list, k0, k1, st.flags, p, st.ctrl, krng);
    c.launches++;
  }
}

// ---------------------------------------------------------------- merge of giant communities
// The member rows of a giant community, concatenated in community-vertex CSR order, form one arc
// range [memoff[coff[c]], memoff[coff[c+1]]) (memoff = exclusive scan of the member degrees in
// cverts order).  A block takes chunks of kChunk arcs of that range in community order, so the
// blocks in flight share the tables of a few communities, which stay in L2; each chunk is summed
// in the block's shared table and flushed once per distinct key.
constexpr int kMemWin = 1024;  // members of a chunk staged in shared memory at a time

// deg[j] = degree of member cverts[j] for the coff[nc] listed members (vertices of graphs that left
// the pass loop are not listed), 0 for j in [coff[nc], n).
__global__ void k_member_degrees(const int32_t* cverts, const int64_t* coff, int64_t nc, int64_t n,
                                 const int64_t* rbeg, const int64_t* rend, int64_t* deg) {
  const int64_t listed = coff[nc];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = 0;
    if (j < listed) {
      const int32_t i = cverts[j];
      d = rend[i] - rbeg[i];
    }
    deg[j] = d;
  }
}

template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_mg_comm_chunks(GraphView<typename M::w_t> g, const int32_t* clist,
                                                                 int64_t m, const int64_t* coff, const int32_t* cverts,
                                                                 const int64_t* memoff, const int32_t* Cp, GiantPlan p,
                                                                 Ctrl* ctrl) {
  typedef typename M::h_t H;
  __shared__ LocalAgg<H> la;
  __shared__ int32_t s_off[kMemWin + 1];  // memoff of the staged members relative to the chunk start,
                                          // clamped to +-2^30 (compared against [0, kChunk) only)
  __shared__ int64_t s_rb[kMemWin];       // row start - (memoff - chunk start): arc of position r
  __shared__ int64_t s_j0;
  if (p.slice_off[m] == 0) return;        // no (or an over-full) plan
  const int64_t nchunks = p.chunk_off[m];
  local_clear(la);
  bool ok = true;
  unsigned long long n_comm = 0, n_mem = 0, n_arcs = 0;  // traffic counters (thread 0)
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int32_t k = p.cowner[q];
    const int32_t c = clist[k];
    const int64_t jb = coff[c], je = coff[c + 1];
    const int64_t a0 = memoff[jb] + (q - p.chunk_off[k]) * kChunk;
    const int64_t a1 = a0 + kChunk < memoff[je] ? a0 + kChunk : memoff[je];
    if (threadIdx.x == 0) {  // the member holding arc a0: largest j in [jb, je) with memoff[j] <= a0
      n_arcs += (unsigned long long)(a1 - a0);
      if (q == p.chunk_off[k]) {
        n_comm++;
        n_mem += (unsigned long long)(je - jb);
      }
      int64_t lo = jb, hi = je;
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (memoff[mid] <= a0) lo = mid; else hi = mid;
      }
      s_j0 = lo;
    }
    __syncthreads();
    int64_t jw = s_j0;
    while (true) {
      const int nm = (int)(je - jw < kMemWin ? je - jw : kMemWin);
      for (int t = threadIdx.x; t <= nm; t += kBlock) {
        const int64_t r = memoff[jw + t] - a0;
        s_off[t] = (int32_t)(r < (1 << 30) ? (r > -(1 << 30) ? r : -(1 << 30)) : (1 << 30));
        if (t < nm) s_rb[t] = g.rbeg[cverts[jw + t]] - r;
      }
      __syncthreads();
      const int32_t lo = s_off[0] > 0 ? s_off[0] : 0;
      const int32_t span = (int32_t)(a1 - a0);
      const int32_t hi = s_off[nm] < span ? s_off[nm] : span;
      int kk = 0;
      constexpr int U = 4;  // arcs per thread per round: U independent load chains in flight
      for (int32_t r0 = lo + (int32_t)threadIdx.x; r0 < hi; r0 += kBlock * U) {
        int64_t ee[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int32_t r = r0 + u * kBlock;
          ee[u] = -1;
          if (r < hi) {
            int kh = nm;  // largest kk in [kk, nm) with s_off[kk] <= r (r only grows)
            while (kh - kk > 1) {
              const int mid = (kk + kh) >> 1;
              if (s_off[mid] <= r) kk = mid; else kh = mid;
            }
            ee[u] = s_rb[kk] + r;
          }
        }
        int32_t jj[U];
        H ww[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          jj[u] = ee[u] >= 0 ? g.tg[ee[u]] : 0;
          ww[u] = ee[u] >= 0 ? (H)g.w[ee[u]] : H(0);
        }
        int32_t cc[U];
#pragma unroll
        for (int u = 0; u < U; u++) cc[u] = ee[u] >= 0 ? Cp[jj[u]] : kEmpty;
#pragma unroll
        for (int u = 0; u < U; u++)
          if (ee[u] >= 0) ok &= tbl_add(la.keys, la.vals, 1u << kLocLog, 32 - kLocLog, cc[u], ww[u]);
      }
      const bool more = s_off[nm] < span && jw + nm < je;
      __syncthreads();  // s_off / s_rb are restaged
      if (!more) break;
      jw += nm;
    }
    const int64_t off = p.tab_off[k];
    const unsigned ts = (unsigned)(p.tab_off[k + 1] - off);
    int lg = 0;
    while ((1u << lg) < ts) lg++;
    ok &= local_flush(la, p.slots + 2 * off, ts, lg, p.bits, off);
  }
  if (!ok) atomicOr(&ctrl->error, kErrTableFull);
  if (threadIdx.x == 0 && n_arcs) {
    unsigned long long* st = ctrl->mg_stat[kNumBuckets - 1];
    atomicAdd(&st[0], n_comm);
    atomicAdd(&st[1], n_mem);
    atomicAdd(&st[2], n_arcs);
  }
}

// Emits the occupied slots of every slice into the holey row of its community: one warp per slice
// of 1024 slots, one occupancy-bitmap word per lane, a warp prefix of the words' populations and
// one atomic per warp on hend[c] (hend starts at hoff[c]).  Slots and bits are cleared.
template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_mg_emit(const int32_t* list, int64_t m, int64_t* hend,
                                                          int32_t* otg, typename M::w_t* ow, GiantPlan p, Ctrl* ctrl) {
  typedef typename M::h_t H;
  const int64_t nslices = p.slice_off[m];
  const int lane = threadIdx.x & 31;
  unsigned long long written = 0;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  for (int64_t q = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); q < nslices; q += nwarps) {
    const int64_t k = p.sowner[q];
    const int32_t c = list[k];
    const int64_t off = p.tab_off[k], ts = p.tab_off[k + 1] - off;
    int2* kv = reinterpret_cast<int2*>(p.slots) + off;
    const int64_t sb = (q - p.slice_off[k]) << kSliceLog;
    const int64_t se = sb + (1 << kSliceLog) < ts ? sb + (1 << kSliceLog) : ts;
    const int nwords = (int)((se - sb) >> 5);
    unsigned* wp = p.bits + ((off + sb) >> 5) + lane;
    unsigned word = lane < nwords ? *wp : 0u;
    const int cnt = __popc(word);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
    if (wtot == 0) continue;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(reinterpret_cast<unsigned long long*>(&hend[c]), (unsigned long long)wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    int64_t pos = (int64_t)base + incl - cnt;
    if (word) *wp = 0u;
    const int64_t s0 = sb + 32 * lane;
    while (word) {
      const int64_t s = s0 + (__ffs(word) - 1);
      word &= word - 1;
      const int2 e = kv[s];
      otg[pos] = e.x;
      ow[pos] = (typename M::w_t)int_as_h<H>(e.y);
      kv[s] = make_int2(kEmpty, 0);
      pos++;
    }
    written += (unsigned long long)cnt;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) written += __shfl_xor_sync(0xffffffffu, written, o);
  if (lane == 0 && written) atomicAdd(&ctrl->mg_stat[kNumBuckets - 1][3], written);
}

template <class M>
void giant_merge(Ctx& c, const MergeArgs<M>& a, const int32_t* clist, int64_t m, int32_t* gix, const GiantPlan& p,
                 int64_t* deg_tmp, int64_t* memoff, int64_t* tile_tmp) {
  if (m <= 0) return;
  const int grid = c.num_sms * 8;
  // tables and member-arc chunks of the giant communities; gix = -1 for every other community
  cudaMemsetAsync(gix, 0xFF, (size_t)a.nc * sizeof(int32_t), c.s);
  giant_plan(c, 1, clist, m, nullptr, nullptr, a.cdeg, a.nc, nullptr, gix, kSliceLog, p, a.ctrl);
  const int64_t n = a.g.n;
  k_member_degrees<<<grid_for(n, kBlock, grid), kBlock, 0, c.s>>>(a.cverts, a.coff, a.nc, n, a.g.rbeg, a.g.rend,
                                                                    deg_tmp);
  scan_exclusive_i64(c, deg_tmp, memoff, n, tile_tmp);
  k_giant_mg_comm_chunks<M><<<c.num_sms * 4, kBlock, 0, c.s>>>(a.g, clist, m, a.coff, a.cverts, memoff, a.Cp, p,
                                                               a.ctrl);
  k_giant_mg_emit<M><<<grid, kBlock, 0, c.s>>>(clist, m, a.hend, a.otg, a.ow, p, a.ctrl);
  c.launches += 3;
}

// ---------------------------------------------------------------- chunk-only plans (rows of list[k])
void giant_chunk_plan(Ctx& c, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                      const GiantPlan& p, Ctrl* ctrl) {
  if (m <= 0) return;
  giant_plan(c, 3, list, m, rbeg, rend, nullptr, 0, nullptr, nullptr, kSliceLog, p, ctrl);
}

// Eq. 1 terms of giant rows: each chunk adds its part of K_i to Sigma_{C_i} and its intra-community
// arc weight to sigma.
template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_mod_chunks(GraphView<typename M::w_t> g, const int32_t* list,
                                                             int64_t m, const int32_t* C, typename M::a_t* tot,
                                                             GiantPlan p, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  const int64_t nchunks = p.chunk_off[m];
  A sig_all = A(0), k_all = A(0);
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    const int32_t i = list[k];
    const int32_t ci = C[i];
    const int64_t e0 = g.rbeg[i] + (q - p.chunk_off[k]) * kChunk;
    const int64_t e1 = e0 + kChunk < g.rend[i] ? e0 + kChunk : g.rend[i];
    A ks = A(0), ss = A(0);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
      const A w = (A)g.w[e];
      ks += w;
      if (C[g.tg[e]] == ci) ss += w;
    }
    ks = group_sum<kBlock>(ks, red);
    if (threadIdx.x == 0 && ks != A(0)) atomic_add_a(&tot[ci], ks);
    sig_all += ss;
    k_all += ks;  // the block total, identical in every thread; thread 0's copy is used
  }
  sig_all = group_sum<kBlock>(sig_all, red);
  if (threadIdx.x == 0) {
    if (M::is_fp) { atomicAdd(&ctrl->acc_f[0], (double)sig_all); atomicAdd(&ctrl->acc_f[1], (double)k_all); }
    else { atomic_add_a(&ctrl->acc_i[0], (long long)sig_all); atomic_add_a(&ctrl->acc_i[1], (long long)k_all); }
  }
}

template <class M>
void giant_modularity(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* list, int64_t m, const int32_t* C,
                      typename M::a_t* tot, const GiantPlan& p, Ctrl* ctrl) {
  if (m <= 0) return;
  giant_chunk_plan(c, list, m, g.rbeg, g.rend, p, ctrl);
  k_giant_mod_chunks<M><<<c.num_sms * 4, kBlock, 0, c.s>>>(g, list, m, C, tot, p, ctrl);
  c.launches++;
}

// Copies the chunks of giant holey rows list[k] (rows [hbeg, hend)) to their dense offsets doff.
template <class W>
__global__ void __launch_bounds__(kBlock) k_giant_copy_chunks(const int32_t* list, int64_t m, const int64_t* hbeg,
                                                              const int64_t* doff, const int32_t* itg, const W* iw,
                                                              int32_t* otg, W* ow, GiantPlan p, const int64_t* hend) {
  const int64_t nchunks = p.chunk_off[m];
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    const int32_t r = list[k];
    const int64_t o = (q - p.chunk_off[k]) * kChunk;
    const int64_t e0 = hbeg[r] + o;
    const int64_t e1 = e0 + kChunk < hend[r] ? e0 + kChunk : hend[r];
    const int64_t d0 = doff[r] + o;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
      otg[d0 + (e - e0)] = itg[e];
      ow[d0 + (e - e0)] = iw[e];
    }
  }
}

template <class W>
void giant_compact(Ctx& c, const int32_t* list, int64_t m, const int64_t* hbeg, const int64_t* hend,
                   const int64_t* doff, const int32_t* itg, const W* iw, int32_t* otg, W* ow, const GiantPlan& p,
                   Ctrl* ctrl) {
  if (m <= 0) return;
  giant_chunk_plan(c, list, m, hbeg, hend, p, ctrl);
  k_giant_copy_chunks<W><<<c.num_sms * 4, kBlock, 0, c.s>>>(list, m, hbeg, doff, itg, iw, otg, ow, p, hend);
  c.launches++;
}

template void giant_modularity<IntMode>(Ctx&, const GraphView<int32_t>&, const int32_t*, int64_t, const int32_t*,
                                        long long*, const GiantPlan&, Ctrl*);
template void giant_modularity<FpMode>(Ctx&, const GraphView<float>&, const int32_t*, int64_t, const int32_t*, double*,
                                       const GiantPlan&, Ctrl*);
template void giant_compact<int32_t>(Ctx&, const int32_t*, int64_t, const int64_t*, const int64_t*, const int64_t*,
                                     const int32_t*, const int32_t*, int32_t*, int32_t*, const GiantPlan&, Ctrl*);
template void giant_compact<float>(Ctx&, const int32_t*, int64_t, const int64_t*, const int64_t*, const int64_t*,
                                   const int32_t*, const float*, int32_t*, float*, const GiantPlan&, Ctrl*);
template void giant_move<IntMode>(Ctx&, const GraphView<int32_t>&, const PassState<IntMode>&, const int32_t*, int64_t,
                                  int64_t, const GiantPlan&, bool, bool, const int64_t*);
template void giant_move<FpMode>(Ctx&, const GraphView<float>&, const PassState<FpMode>&, const int32_t*, int64_t,
                                 int64_t, const GiantPlan&, bool, bool, const int64_t*);
template void giant_move_plan<IntMode>(Ctx&, const GraphView<int32_t>&, const int32_t*, int64_t, const GiantPlan&,
                                       Ctrl*);
template void giant_move_plan<FpMode>(Ctx&, const GraphView<float>&, const int32_t*, int64_t, const GiantPlan&, Ctrl*);
template void giant_merge<IntMode>(Ctx&, const MergeArgs<IntMode>&, const int32_t*, int64_t, int32_t*,
                                   const GiantPlan&, int64_t*, int64_t*, int64_t*);
template void giant_merge<FpMode>(Ctx&, const MergeArgs<FpMode>&, const int32_t*, int64_t, int32_t*,
                                  const GiantPlan&, int64_t*, int64_t*, int64_t*);

}  // namespace lv
