// giant.cu -- the multi-block path for giant rows (degree bucket 4, > 2048 arcs).
//
// A hub vertex (R-MAT hubs reach 10^5 arcs) or a giant community (10^6-10^7 member arcs after a
// pass) handled by one block serialises a whole launch on one SM.  Here the work of a giant is cut
// into arc chunks and table slices that every SM shares:
//   plan    one block: per giant its chunk count, table size (a power of two >= 2 x its distinct-key
//           bound) and slice count; exclusive scans give each giant its chunk / slot / slice range
//           in a shared pool of global-memory tables, and owner arrays map every chunk and slice
//           back to its giant in one load;
//   insert  grid-stride over chunks of 2048 arcs: a block first sums its chunk per key in a
//           shared-memory table (K_i->c, scanCommunities), then adds each distinct key once to the
//           giant's global table with L2 atomics;
//   scan    grid-stride over slices of 8192 slots (16-byte key loads): local move scores every
//           candidate with the Eq. 2 numerator and keeps the slice's best; merge emits the slice's
//           (community, weight) pairs into the holey row of the community.  Every occupied slot
//           is cleared, so the pool is all-empty between uses;
//   decide  (local move) per giant: best over its slices, then the move exactly as the per-vertex
//           kernels make it;
//   mark    (local move, pruning) grid-stride over chunks of the giants that moved.
// Merges insert member rows vertex by vertex (members of giant communities, by their own degree
// bucket), so a giant community's arcs spread over the GPU however its members are shaped.
#include "internal.cuh"

namespace lv {

constexpr int kChunk = 2048;   // arcs per chunk
constexpr int kSlice = 128;    // table slots per slice: one warp, one 16-byte key load per lane
constexpr int kLocLog = 12;    // shared pre-aggregation table: 4096 slots >= 2 x kChunk keys

// ---------------------------------------------------------------- plan (one block)
// kind 0: local move, item = vertex list[k], bound = min(deg, n_bound), chunks over its row; a
//          pruned vertex gets nothing, an active one has its flag cleared (marked processed).
// kind 1: merge, item = community list[k], bound = min(cdeg, n_bound), no chunks (rows are inserted
//          member-wise); gix[c] = k.
// kind 2: chunks only, item = vertex list[k] if its community Cp[i] is giant (gix >= 0).
// kind 3: chunks only, every listed row.
__global__ void __launch_bounds__(1024) k_giant_plan(int kind, const int32_t* list, int64_t m, const int64_t* rbeg,
                                                     const int64_t* rend, const int64_t* cdeg, int64_t n_bound,
                                                     uint8_t* flags, int pruning, const int32_t* Cp, int32_t* gix,
                                                     GiantPlan p, Ctrl* ctrl, const GraphCtl* gc = nullptr,
                                                     const int32_t* vg = nullptr) {
  __shared__ int64_t part[3][1024];
  if (kind == 0 && *(volatile int32_t*)&ctrl->done) return;
  const int t = threadIdx.x;
  const int64_t per = (m + 1023) / 1024;
  const int64_t b = t * per, e = b + per < m ? b + per : m;
  int64_t sc = 0, st = 0, ss = 0;
  for (int64_t k = b; k < e; k++) {
    const int32_t v = list[k];
    int64_t nch = 0, ts = 0;
    if (kind == 1) {
      const int64_t bound = cdeg[v] < n_bound ? cdeg[v] : n_bound;
      ts = (int64_t)1 << tbl_log2(bound, 6, 31);
    } else {
      const int64_t deg = rend[v] - rbeg[v];
      bool active = true;
      if (kind == 0 && gc && gc[vg[v]].done) active = false;  // batched: graph converged
      if (kind == 0 && pruning && active) {
        active = flags[v] != 0;
        if (active) flags[v] = 0;
      }
      if (kind == 2) active = Cp[v] >= 0 && gix[Cp[v]] >= 0;  // batched: Cp < 0 = graph left
      if (active) {
        nch = (deg + kChunk - 1) / kChunk;
        if (kind == 0) ts = (int64_t)1 << tbl_log2(deg < n_bound ? deg : n_bound, 6, 31);
      }
    }
    p.chunk_off[k] = nch;
    p.tab_off[k] = ts;
    p.slice_off[k] = ts ? (ts + kSlice - 1) / kSlice : 0;
    sc += nch; st += ts; ss += p.slice_off[k];
  }
  part[0][t] = sc; part[1][t] = st; part[2][t] = ss;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t v0 = t >= o ? part[0][t - o] : 0, v1 = t >= o ? part[1][t - o] : 0, v2 = t >= o ? part[2][t - o] : 0;
    __syncthreads();
    part[0][t] += v0; part[1][t] += v1; part[2][t] += v2;
    __syncthreads();
  }
  const int64_t tot_c = part[0][1023], tot_t = part[1][1023], tot_s = part[2][1023];
  const bool fits = tot_c <= p.chunk_cap && tot_s <= p.slice_cap && tot_t <= p.pool_slots;
  int64_t rc = t ? part[0][t - 1] : 0, rt = t ? part[1][t - 1] : 0, rs = t ? part[2][t - 1] : 0;
  for (int64_t k = b; k < e; k++) {
    const int64_t nch = p.chunk_off[k], ts = p.tab_off[k], ns = p.slice_off[k];
    p.chunk_off[k] = rc; p.tab_off[k] = rt; p.slice_off[k] = rs;
    if (fits) {
      for (int64_t q = 0; q < nch; q++) p.cowner[rc + q] = (int32_t)k;
      for (int64_t q = 0; q < ns; q++) p.sowner[rs + q] = (int32_t)k;
    }
    if (kind == 1) gix[list[k]] = (int32_t)k;
    reinterpret_cast<uint32_t*>(p.kid)[k] = 0u;  // 0u is also 0.0f
    p.moved[k] = 0;
    rc += nch; rt += ts; rs += ns;
  }
  if (t == 1023) {
    // an over-full plan runs nothing (chunk and slice totals read 0) and reports the error
    p.chunk_off[m] = fits ? tot_c : 0;
    p.tab_off[m] = tot_t;
    p.slice_off[m] = fits ? tot_s : 0;
    if (!fits) atomicOr(&ctrl->error, kErrTableFull);
  }
}

// ---------------------------------------------------------------- shared pre-aggregation
// Sums a chunk's (key, weight) pairs in the block's shared table, then flushes each distinct key
// once into the global table (tk, tv, size 2^lg).  Every thread of the block must call both.
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
__device__ __forceinline__ bool local_flush(LocalAgg<H>& la, int32_t* tk, H* tv, unsigned size, int lg) {
  bool ok = true;
  __syncthreads();
  for (int s = threadIdx.x; s < (1 << kLocLog); s += kBlock) {
    const int32_t key = la.keys[s];
    if (key != kEmpty) {
      ok &= tbl_add(tk, tv, size, 32 - lg, key, la.vals[s]);
      la.keys[s] = kEmpty;
      la.vals[s] = H(0);
    }
  }
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------- local move: insert
template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_lm_insert(GraphView<typename M::w_t> g, const int32_t* list, int64_t m,
                                                            const int32_t* Cp, GiantPlan p, Ctrl* ctrl) {
  typedef typename M::h_t H;
  __shared__ H red[32];
  if (*(volatile int32_t*)&ctrl->done) return;
  const int64_t nchunks = p.chunk_off[m];
  bool ok = true;
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    const int32_t i = list[k];
    const int32_t d = Cp[i];
    const int64_t off = p.tab_off[k], ts = p.tab_off[k + 1] - off;
    int lg = 0;
    while (((int64_t)1 << lg) < ts) lg++;
    int32_t* tk = p.keys + off;
    H* tv = reinterpret_cast<H*>(p.vals) + off;
    const int64_t e0 = g.rbeg[i] + (q - p.chunk_off[k]) * kChunk;
    const int64_t e1 = e0 + kChunk < g.rend[i] ? e0 + kChunk : g.rend[i];
    H kid = H(0);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
      const int32_t j = g.tg[e];
      if (j == i) continue;
      const H wv = (H)g.w[e];
      const int32_t cj = Cp[j];
      if (cj == d) kid += wv;
      else ok &= tbl_add(tk, tv, (unsigned)ts, 32 - lg, cj, wv);
    }
    kid = group_sum<kBlock>(kid, red);
    if (threadIdx.x == 0 && kid != H(0)) atomicAdd(reinterpret_cast<H*>(p.kid) + k, kid);
  }
  if (!ok) atomicOr(&ctrl->error, kErrTableFull);
}

// ---------------------------------------------------------------- local move: slice scan
template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_lm_scan(const int32_t* list, int64_t m, const int32_t* Cp,
                                                          const typename M::a_t* K, const typename M::a_t* Sig,
                                                          GiantPlan p, Ctrl* ctrl, const GraphCtl* gc,
                                                          const int32_t* vg) {
  typedef typename M::h_t H;
  typedef typename M::a_t A;
  typedef typename M::s_t S;
  if (*(volatile int32_t*)&ctrl->done) return;
  const int64_t nslices = p.slice_off[m];
  const A two_m_all = M::is_fp ? (A)ctrl->two_m_f : (A)ctrl->two_m_i;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (kBlock / 32);
  unsigned long long cand = 0;
  // one warp per slice of 128 slots, one 16-byte key load per lane (tables are >= 64 slots and
  // 64-slot aligned, so a slice never straddles two tables and every load is aligned)
  for (int64_t q = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); q < nslices; q += nwarps) {
    const int64_t k = p.sowner[q];
    const int64_t off = p.tab_off[k], ts = p.tab_off[k + 1] - off;
    const int64_t s = (q - p.slice_off[k]) * kSlice + 4 * lane;
    S best = M::lowest();
    int32_t bc = 0x7fffffff;
    if (s < ts) {
      int32_t* tk = p.keys + off;
      H* tv = reinterpret_cast<H*>(p.vals) + off;
      const int4 kk = *reinterpret_cast<const int4*>(tk + s);
      const int32_t ks[4] = {kk.x, kk.y, kk.z, kk.w};
      if ((kk.x & kk.y & kk.z & kk.w) != kEmpty) {  // some slot occupied
        const int32_t i = list[k];
        const int32_t d = Cp[i];
        const H kid = reinterpret_cast<const H*>(p.kid)[k];
        const A ki = K[i], sd = Sig[d];
        const GraphCtl* gcv = gc ? gc + vg[i] : nullptr;
        const A two_m = gcv ? (M::is_fp ? (A)gcv->two_m_f : (A)gcv->two_m_i) : two_m_all;
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int32_t c = ks[u];
          if (c == kEmpty) continue;
          const H v = tv[s + u];
          tk[s + u] = kEmpty;
          tv[s + u] = H(0);
          cand++;
          const S sc = M::score(v, kid, ki, Sig[c], sd, two_m);
          if (better(sc, c, best, bc)) { best = sc; bc = c; }
        }
      }
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
__global__ void __launch_bounds__(kBlock) k_giant_lm_decide(const int32_t* list, int64_t m, PassState<M> st,
                                                            GiantPlan p, int fast) {
  typedef typename M::a_t A;
  typedef typename M::s_t S;
  Ctrl* ctrl = st.ctrl;
  if (*(volatile int32_t*)&ctrl->done || p.slice_off[m] == 0) return;
  unsigned long long acc_lo = 0, acc_hi = 0, acc_mv = 0;
  double acc_f = 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
  for (int64_t k = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); k < m; k += nw) {
    const int64_t q0 = p.slice_off[k], q1 = p.slice_off[k + 1];
    if (q0 == q1) continue;  // pruned
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
}

// ---------------------------------------------------------------- local move: mark neighbours
template <class W>
__global__ void __launch_bounds__(kBlock) k_giant_lm_mark(GraphView<W> g, const int32_t* list, int64_t m,
                                                          uint8_t* flags, GiantPlan p, Ctrl* ctrl) {
  if (*(volatile int32_t*)&ctrl->done) return;
  const int64_t nchunks = p.chunk_off[m];
  unsigned long long marks = 0;
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int64_t k = p.cowner[q];
    if (!p.moved[k]) continue;
    const int32_t i = list[k];
    const int64_t e0 = g.rbeg[i] + (q - p.chunk_off[k]) * kChunk;
    const int64_t e1 = e0 + kChunk < g.rend[i] ? e0 + kChunk : g.rend[i];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock) {
      const int32_t j = g.tg[e];
      if (j != i) { flags[j] = 1; marks++; }
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) marks += __shfl_xor_sync(0xffffffffu, marks, o);
  if ((threadIdx.x & 31) == 0 && marks) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][5], marks);
}

// list / processed / arcs counters of the giant bucket (after the plan)
__global__ void k_giant_lm_count(GraphView<int32_t> gs, const int32_t* list, int64_t m, GiantPlan p, Ctrl* ctrl) {
  if (*(volatile int32_t*)&ctrl->done) return;
  unsigned long long act = 0, arcs = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    if (p.slice_off[k + 1] > p.slice_off[k]) { act++; arcs += (unsigned long long)(gs.rend[list[k]] - gs.rbeg[list[k]]); }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    act += __shfl_xor_sync(0xffffffffu, act, o);
    arcs += __shfl_xor_sync(0xffffffffu, arcs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][0], (unsigned long long)m);
    if (act) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][1], act);
    if (arcs) atomicAdd(&ctrl->lm_stat[kNumBuckets - 1][2], arcs);
  }
}

template <class M>
void giant_move(Ctx& c, const GraphView<typename M::w_t>& g, const PassState<M>& st, const int32_t* list, int64_t m,
                const GiantPlan& p, bool fast, bool pruning) {
  if (m <= 0) return;
  const int grid = c.num_sms * 8;
  k_giant_plan<<<1, 1024, 0, c.s>>>(0, list, m, g.rbeg, g.rend, nullptr, g.n, st.flags, pruning ? 1 : 0, nullptr,
                                    nullptr, p, st.ctrl, st.gc, st.vg);
  GraphView<int32_t> gs{g.n, g.rbeg, g.rend, g.tg, nullptr};
  k_giant_lm_count<<<grid_for(m, kBlock, c.num_sms), kBlock, 0, c.s>>>(gs, list, m, p, st.ctrl);
  k_giant_lm_insert<M><<<grid, kBlock, 0, c.s>>>(g, list, m, st.Cp, p, st.ctrl);
  k_giant_lm_scan<M><<<grid, kBlock, 0, c.s>>>(list, m, st.Cp, st.K, st.Sig, p, st.ctrl, st.gc, st.vg);
  k_giant_lm_decide<M><<<grid_for(m, kBlock / 32, c.num_sms * 2), kBlock, 0, c.s>>>(list, m, st, p, fast ? 1 : 0);
  c.launches += 5;
  if (pruning) {
    k_giant_lm_mark<typename M::w_t><<<grid, kBlock, 0, c.s>>>(g, list, m, st.flags, p, st.ctrl);
    c.launches++;
  }
}

// ---------------------------------------------------------------- merge of giant communities
// Member rows of giant communities go into their community's table: one group per member (the
// member's degree bucket), giant members by arc chunks.
template <class M, int G>
__global__ void __launch_bounds__(kBlock) k_giant_mg_insert(GraphView<typename M::w_t> g, const int32_t* list,
                                                            int64_t count, const int32_t* Cp, const int32_t* gix,
                                                            GiantPlan p, int64_t mc, Ctrl* ctrl) {
  typedef typename M::h_t H;
  if (p.slice_off[mc] == 0) return;  // no (or an over-full) plan
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  bool ok = true;
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t i = list[idx];
    const int32_t ci = Cp[i];
    if (ci < 0) continue;  // batched: the graph of i left the pass loop
    const int32_t k = gix[ci];
    if (k < 0) continue;
    const int64_t off = p.tab_off[k];
    const unsigned ts = (unsigned)(p.tab_off[k + 1] - off);
    int lg = 0;
    while ((1u << lg) < ts) lg++;
    int32_t* tk = p.keys + off;
    H* tv = reinterpret_cast<H*>(p.vals) + off;
    for (int64_t e = g.rbeg[i] + lane; e < g.rend[i]; e += G) ok &= tbl_add(tk, tv, ts, 32 - lg, Cp[g.tg[e]], (H)g.w[e]);
  }
  if (!ok) atomicOr(&ctrl->error, kErrTableFull);
}

template <class M>
__global__ void __launch_bounds__(kBlock) k_giant_mg_insert_chunks(GraphView<typename M::w_t> g, const int32_t* list,
                                                                   int64_t m, const int32_t* Cp, const int32_t* gix,
                                                                   GiantPlan pv, GiantPlan p, int64_t mc, Ctrl* ctrl) {
  typedef typename M::h_t H;
  __shared__ LocalAgg<H> la;
  if (p.slice_off[mc] == 0) return;
  const int64_t nchunks = pv.chunk_off[m];
  if (nchunks == 0) return;
  local_clear(la);
  bool ok = true;
  for (int64_t q = blockIdx.x; q < nchunks; q += gridDim.x) {
    const int64_t kv = pv.cowner[q];
    const int32_t i = list[kv];
    const int32_t k = gix[Cp[i]];
    const int64_t off = p.tab_off[k];
    const unsigned ts = (unsigned)(p.tab_off[k + 1] - off);
    const int64_t e0 = g.rbeg[i] + (q - pv.chunk_off[kv]) * kChunk;
    const int64_t e1 = e0 + kChunk < g.rend[i] ? e0 + kChunk : g.rend[i];
    __syncthreads();
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kBlock)
      ok &= tbl_add(la.keys, la.vals, 1u << kLocLog, 32 - kLocLog, Cp[g.tg[e]], (H)g.w[e]);
    int lg = 0;
    while ((1u << lg) < ts) lg++;
    ok &= local_flush(la, p.keys + off, reinterpret_cast<H*>(p.vals) + off, ts, lg);
  }
  if (!ok) atomicOr(&ctrl->error, kErrTableFull);
}

// Emits the occupied slots of every slice into the holey row of its community; hend[c] starts at
// hoff[c] and is advanced atomically (one atomic per warp and 16-byte key group).
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
    int32_t* tk = p.keys + off;
    H* tv = reinterpret_cast<H*>(p.vals) + off;
    {  // one warp per 128-slot slice, one 16-byte key load per lane
      const int64_t s = (q - p.slice_off[k]) * kSlice + 4 * lane;
      int4 kk = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
      if (s < ts) kk = *reinterpret_cast<const int4*>(tk + s);
      const int32_t ks[4] = {kk.x, kk.y, kk.z, kk.w};
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < 4; u++) cnt += ks[u] != kEmpty;
      // warp prefix of the per-lane counts, one atomic per warp
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
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (ks[u] == kEmpty) continue;
        otg[pos] = ks[u];
        ow[pos] = (typename M::w_t)tv[s + u];
        tk[s + u] = kEmpty;
        tv[s + u] = H(0);
        pos++;
      }
      written += (unsigned long long)cnt;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) written += __shfl_xor_sync(0xffffffffu, written, o);
  if (lane == 0 && written) atomicAdd(&ctrl->mg_stat[kNumBuckets - 1][3], written);
}

template <class M>
void giant_merge(Ctx& c, const MergeArgs<M>& a, const int32_t* clist, int64_t m, const int32_t* dperm,
                 const int64_t* hb, int32_t* gix, const GiantPlan& p, const GiantPlan& pv) {
  if (m <= 0) return;
  const int grid = c.num_sms * 8;
  // tables of the giant communities; gix = -1 for every other community
  cudaMemsetAsync(gix, 0xFF, (size_t)a.nc * sizeof(int32_t), c.s);
  k_giant_plan<<<1, 1024, 0, c.s>>>(1, clist, m, nullptr, nullptr, a.cdeg, a.nc, nullptr, 0, nullptr, gix, p, a.ctrl);
  c.launches++;
  // member rows, by the member's degree bucket
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    const int64_t cnt = hb[b + 1] - hb[b];
    if (cnt <= 0) continue;
    const int32_t* l = dperm + hb[b];
    switch (b) {
      case 0: k_giant_mg_insert<M, 4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(a.g, l, cnt, a.Cp, gix, p, m, a.ctrl); break;
      case 1: k_giant_mg_insert<M, 8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(a.g, l, cnt, a.Cp, gix, p, m, a.ctrl); break;
      case 2: k_giant_mg_insert<M, 32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(a.g, l, cnt, a.Cp, gix, p, m, a.ctrl); break;
      case 3:
      case 4: k_giant_mg_insert<M, 256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(a.g, l, cnt, a.Cp, gix, p, m, a.ctrl); break;
      default:
        // giant members: chunk plan over their rows (members of giant communities only)
        k_giant_plan<<<1, 1024, 0, c.s>>>(2, l, cnt, a.g.rbeg, a.g.rend, nullptr, a.g.n, nullptr, 0, a.Cp, gix, pv,
                                          a.ctrl);
        k_giant_mg_insert_chunks<M><<<grid, kBlock, 0, c.s>>>(a.g, l, cnt, a.Cp, gix, pv, p, m, a.ctrl);
        c.launches++;
        break;
    }
    c.launches++;
  }
  k_giant_mg_emit<M><<<grid, kBlock, 0, c.s>>>(clist, m, a.hend, a.otg, a.ow, p, a.ctrl);
  c.launches++;
}

// ---------------------------------------------------------------- chunk-only plans (rows of list[k])
void giant_chunk_plan(Ctx& c, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                      const GiantPlan& p, Ctrl* ctrl) {
  if (m <= 0) return;
  k_giant_plan<<<1, 1024, 0, c.s>>>(3, list, m, rbeg, rend, nullptr, 0, nullptr, 0, nullptr, nullptr, p, ctrl);
  c.launches++;
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
                                  const GiantPlan&, bool, bool);
template void giant_move<FpMode>(Ctx&, const GraphView<float>&, const PassState<FpMode>&, const int32_t*, int64_t,
                                 const GiantPlan&, bool, bool);
template void giant_merge<IntMode>(Ctx&, const MergeArgs<IntMode>&, const int32_t*, int64_t, const int32_t*,
                                   const int64_t*, int32_t*, const GiantPlan&, const GiantPlan&);
template void giant_merge<FpMode>(Ctx&, const MergeArgs<FpMode>&, const int32_t*, int64_t, const int32_t*,
                                  const int64_t*, int32_t*, const GiantPlan&, const GiantPlan&);

}  // namespace lv
