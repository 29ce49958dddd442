// batch.cu -- the per-graph bookkeeping of louvain_run_batch.
//
// A batch of independent graphs runs as ONE union graph: graph g owns the vertex range
// [vbase_g, vbase_g + nlev_g) of every level, so each launch of the local-moving and aggregation
// kernels covers every graph at once.  What Algorithm 1 and Algorithm 2 keep per graph lives in
// GraphCtl: 2m, the exact per-iteration sum of N and the tolerance test, l_i, the pass tests
// (l_i <= 1, |Gamma| / |V'| > tau_agg), and the renumbering.  A graph leaves the union when its
// pass loop stops: its membership is final (graph-local canonical ids) and the next level holds
// only the graphs that continue.  The colouring priorities and random classes hash graph-local
// ids (Segs), so every graph takes exactly the steps it takes alone.
#include "internal.cuh"

namespace lv {

// ---------------------------------------------------------------- setup
// vg[v] = the graph whose vertex range [vo[g], vo[g+1]) holds v (empty graphs skipped).
__global__ void k_batch_vg0(const int64_t* vo, int32_t G, int64_t n, int32_t* vg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = G;  // vo[lo] <= v < vo[hi]
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (vo[mid] <= v) lo = mid; else hi = mid;
    }
    vg[v] = lo;
  }
}

// ao[g] = offsets[vo[g]]: the arc range of every graph.
__global__ void k_batch_arc_offs(const int64_t* vo, int32_t G, const int64_t* offs, int64_t* ao) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x)
    ao[g] = offs[vo[g]];
}

// Graph-local targets -> union ids; a target outside its graph counts in ctrl->cnt[1].
__global__ void k_batch_targets(const int64_t* vo, const int64_t* ao, int32_t G, int64_t n_arcs, const int32_t* tg,
                                int32_t* out, Ctrl* ctrl) {
  unsigned long long bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_arcs; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = G;  // ao[lo] <= e < ao[hi]
    while (hi - lo > 1) {
      const int32_t mid = (lo + hi) >> 1;
      if (ao[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t base = vo[lo], ng = vo[lo + 1] - base;
    const int32_t t = tg[e];
    if (t < 0 || t >= ng) {
      bad++;
      out[e] = (int32_t)base;  // keeps every id in range; the call fails on the count
    } else {
      out[e] = (int32_t)(base + t);
    }
  }
  if (bad) atomicAdd(&ctrl->cnt[1], bad);
}

__global__ void k_batch_init(GraphCtl* gc, const int64_t* vo, int32_t G) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    GraphCtl c = {};
    c.vbase = vo[g];
    c.nlev = vo[g + 1] - vo[g];
    c.active = c.nlev > 0 ? 1 : 0;
    c.done = 1;
    gc[g] = c;
  }
}

// 2m of every graph = sum of K over its vertex range (one block per graph).
// Integer mode needs 2m < 2^31 per graph: ctrl->cnt[6] counts the graphs that exceed it.
template <class M>
__global__ void __launch_bounds__(kBlock) k_batch_two_m(GraphCtl* gc, int32_t G, const typename M::a_t* K, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    const int64_t b = gc[g].vbase, n = gc[g].nlev;
    A s = A(0);
    for (int64_t v = threadIdx.x; v < n; v += kBlock) s += K[b + v];
    s = group_sum<kBlock>(s, red);
    if (threadIdx.x == 0) {
      if (M::is_fp) {
        gc[g].two_m_f = (double)s;
      } else {
        gc[g].two_m_i = (long long)s;
        if ((long long)s >= (1LL << 31)) atomicAdd(&ctrl->cnt[6], 1ULL);
      }
    }
  }
}

// ---------------------------------------------------------------- local-moving phase
__global__ void k_batch_move_setup(GraphCtl* gc, int32_t G, int max_iterations) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    GraphCtl& c = gc[g];
    c.done = (!c.active || max_iterations <= 0) ? 1 : 0;
    c.iterations = 0;
    c.sum_lo = c.sum_hi = 0;
    c.sum_f = 0.0;
  }
}

// Algorithm 2's tolerance test per graph (the same arithmetic as the single-graph test); the
// union's phase ends when every graph has converged or reached MAX_IT.
template <bool FP>
__global__ void __launch_bounds__(1024) k_batch_finish(Ctrl* ctrl, GraphCtl* gc, int32_t G) {
  __shared__ int left_s;
  if (*(volatile int32_t*)&ctrl->done) return;
  if (threadIdx.x == 0) left_s = 0;
  __syncthreads();
  const double tau = ctrl->tau;
  const int max_it = ctrl->max_iterations;
  int left = 0;
  for (int64_t g = threadIdx.x; g < G; g += blockDim.x) {
    GraphCtl& c = gc[g];
    if (c.done) continue;
    const int it = c.iterations + 1;
    c.iterations = it;
    bool conv;
    if (FP) {
      conv = __dmul_rn(2.0, c.sum_f) <= __dmul_rn(tau, __dmul_rn(c.two_m_f, c.two_m_f));
    } else {
      const unsigned long long hi = (c.sum_hi << 1) | (c.sum_lo >> 63), lo = c.sum_lo << 1;
      const double t = __ll2double_rn(c.two_m_i);
      conv = u128_to_double_rn(hi, lo) <= __dmul_rn(tau, __dmul_rn(t, t));
    }
    c.sum_lo = c.sum_hi = 0;
    c.sum_f = 0.0;
    if (conv || it >= max_it) c.done = 1;
    else left++;
  }
  if (left) atomicAdd(&left_s, left);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctrl->iterations += 1;
    ctrl->moves_pass += ctrl->moves;
    ctrl->moves = 0;
    if (left_s == 0) ctrl->done = 1;
  }
}

// ---------------------------------------------------------------- pass end
// Per active graph: communities after the pass (from the union renumbering scan), the pass tests
// of Algorithm 1, and the next level's vertex base of the continuing graphs (block scan).
// ctrl->acc_i[3] receives the next level's vertex count.
__global__ void __launch_bounds__(1024) k_batch_pass_end(GraphCtl* gc, int32_t G, const int64_t* newid,
                                                         double tau_agg, int last, Ctrl* ctrl) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int64_t per = ((int64_t)G + 1023) / 1024;
  const int64_t b = t * per, e = b + per < G ? b + per : G;
  long long sum = 0;
  for (int64_t g = b; g < e; g++) {
    GraphCtl& c = gc[g];
    c.cont = 0;
    if (!c.active) continue;
    c.comm_base = newid[c.vbase];
    c.n_comm = newid[c.vbase + c.nlev] - c.comm_base;
    c.passes += 1;
    c.total_iterations += c.iterations;
    const bool stop = c.iterations <= 1 || __ddiv_rn((double)c.n_comm, (double)c.nlev) > tau_agg || last;
    c.cont = stop ? 0 : 1;
    if (c.cont) sum += c.n_comm;
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = t ? part[t - 1] : 0;
  for (int64_t g = b; g < e; g++) {
    GraphCtl& c = gc[g];
    if (c.cont) { c.nbase = run; run += c.n_comm; }
  }
  if (t == 1023) ctrl->acc_i[3] = part[1023];
}

// Renumbering (rank among the graph's occupied ids): continuing graphs get next-level union ids,
// graphs that stop get -1 - (local id) so that the lookup can finish them and the aggregation
// kernels skip them.
__global__ void k_batch_relabel(int32_t* Cp, int64_t n, const int64_t* newid, const int32_t* vg, const GraphCtl* gc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const GraphCtl& c = gc[vg[i]];
    const long long r = newid[Cp[i]] - c.comm_base;
    Cp[i] = c.cont ? (int32_t)(c.nbase + r) : (int32_t)(-1 - r);
  }
}

// Dendrogram lookup C[v] = C'[C[v]] for the original vertices of the graphs at this level.
__global__ void k_batch_lookup(int32_t* C, int64_t n0, const int32_t* vg0, const GraphCtl* gc, const int32_t* Cp) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    if (!gc[vg0[v]].active) continue;
    const int32_t x = Cp[C[v]];
    C[v] = x >= 0 ? x : -1 - x;
  }
}

// K of the next level = Sigma of each occupied community of a continuing graph; vg of the next level.
template <class A>
__global__ void k_batch_next_level(const A* sig, const int32_t* occ, const int64_t* newid, const int32_t* vg,
                                   const GraphCtl* gc, int64_t n_old, A* k_next, const int32_t* Cp, int32_t* vg_next) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_old; c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = vg[c];
    const GraphCtl& gg = gc[g];
    if (!gg.cont) continue;
    if (occ[c]) k_next[gg.nbase + (newid[c] - gg.comm_base)] = sig[c];
    const int32_t x = Cp[c];  // vertex c's new community (>= 0 for a continuing graph)
    vg_next[x] = g;
  }
}

__global__ void k_batch_advance(GraphCtl* gc, int32_t G) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    GraphCtl& c = gc[g];
    if (!c.active) continue;
    c.active = c.cont;
    if (c.cont) { c.vbase = c.nbase; c.nlev = c.n_comm; }
  }
}

// Graphs still open when the pass loop ends (only with max_passes = 0): every vertex is its own
// community, with graph-local ids.
__global__ void k_batch_close(int32_t* C, int64_t n0, const int32_t* vg0, GraphCtl* gc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    const GraphCtl& c = gc[vg0[v]];
    if (c.active) C[v] = (int32_t)(C[v] - c.vbase);
  }
}
__global__ void k_batch_close_ctl(GraphCtl* gc, int32_t G) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
    GraphCtl& c = gc[g];
    if (c.active) { c.n_comm = c.nlev; c.active = 0; }
  }
}

// ---------------------------------------------------------------- final modularity (Eq. 1 per graph)
// comm_base = exclusive scan of the graphs' final community counts (one block).
__global__ void __launch_bounds__(1024) k_batch_comm_base(GraphCtl* gc, int32_t G) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int64_t per = ((int64_t)G + 1023) / 1024;
  const int64_t b = t * per, e = b + per < G ? b + per : G;
  long long sum = 0;
  for (int64_t g = b; g < e; g++) sum += gc[g].n_comm;
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = t ? part[t - 1] : 0;
  for (int64_t g = b; g < e; g++) { gc[g].comm_base = run; run += gc[g].n_comm; }
}

// Per vertex (one group of G lanes): intra-community weight into intra[v], K_v into the union
// community total tot[comm_base + C[v]] (C holds graph-local ids).
template <class M, int G>
__global__ void __launch_bounds__(kBlock) k_bmod_group(GraphView<typename M::w_t> g, const int32_t* list, int64_t count,
                                                       const int32_t* C, const int32_t* vg0, const GraphCtl* gc,
                                                       typename M::a_t* intra, typename M::a_t* tot) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t i = list[idx];
    const int32_t ci = C[i];
    A k = A(0), s = A(0);
    for (int64_t e = g.rbeg[i] + lane; e < g.rend[i]; e += G) {
      const A w = (A)g.w[e];
      k += w;
      if (C[g.tg[e]] == ci) s += w;
    }
    k = group_sum<G>(k, red);
    s = group_sum<G>(s, red);
    if (lane == 0) {
      intra[i] = s;
      atomic_add_a(&tot[gc[vg0[i]].comm_base + ci], k);
    }
  }
}

// Block per graph: sigma = sum of intra over its vertices, sum of squared totals over its
// communities, Q as in the single-graph kernel (exact in integer mode).
template <class M>
__global__ void __launch_bounds__(kBlock) k_bmod_final(GraphCtl* gc, int32_t G, const int64_t* vo,
                                                       const typename M::a_t* intra, const typename M::a_t* tot) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
    A s = A(0), q = A(0);
    for (int64_t v = vo[g] + threadIdx.x; v < vo[g + 1]; v += kBlock) s += intra[v];
    const int64_t cb = gc[g].comm_base, nc = gc[g].n_comm;
    for (int64_t c = threadIdx.x; c < nc; c += kBlock) { const A t = tot[cb + c]; q += t * t; }
    s = group_sum<kBlock>(s, red);
    q = group_sum<kBlock>(q, red);
    if (threadIdx.x == 0) {
      GraphCtl& c = gc[g];
      if (M::is_fp) {
        const double tm = c.two_m_f;
        c.sig_in_f = (double)s; c.sq_f = (double)q;
        c.q = tm == 0.0 ? 0.0 : __dsub_rn(__ddiv_rn((double)s, tm), __ddiv_rn((double)q, __dmul_rn(tm, tm)));
      } else {
        const long long tm = c.two_m_i;
        c.sig_in_i = (long long)s; c.sq_i = (long long)q;
        c.q = tm == 0 ? 0.0 : __ddiv_rn(__ll2double_rn(tm * (long long)s - (long long)q), __ll2double_rn(tm * tm));
      }
    }
  }
}

// ---------------------------------------------------------------- host launchers
void batch_setup(Ctx& c, const int64_t* vo, int32_t G, int64_t n, const int64_t* offs, int64_t n_arcs,
                 const int32_t* tg_local, int32_t* tg_union, int64_t* ao, int32_t* vg0, GraphCtl* gc, Ctrl* ctrl) {
  const int cap = c.num_sms * 8;
  k_batch_vg0<<<grid_for(n, kBlock, cap), kBlock, 0, c.s>>>(vo, G, n, vg0);
  k_batch_arc_offs<<<grid_for(G + 1, kBlock, cap), kBlock, 0, c.s>>>(vo, G, offs, ao);
  k_batch_init<<<grid_for(G, kBlock, cap), kBlock, 0, c.s>>>(gc, vo, G);
  c.launches += 3;
  if (n_arcs > 0) {
    k_batch_targets<<<grid_for(n_arcs, kBlock, cap), kBlock, 0, c.s>>>(vo, ao, G, n_arcs, tg_local, tg_union, ctrl);
    c.launches++;
  }
}

template <class M>
void batch_two_m(Ctx& c, GraphCtl* gc, int32_t G, const typename M::a_t* K, Ctrl* ctrl) {
  k_batch_two_m<M><<<grid_for(G, 1, c.num_sms * 16), kBlock, 0, c.s>>>(gc, G, K, ctrl);
  c.launches++;
}

void batch_move_setup(Ctx& c, GraphCtl* gc, int32_t G, int max_iterations) {
  k_batch_move_setup<<<grid_for(G, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(gc, G, max_iterations);
  c.launches++;
}

template <class M>
void batch_finish(Ctx& c, Ctrl* ctrl, GraphCtl* gc, int32_t G) {
  k_batch_finish<M::is_fp><<<1, 1024, 0, c.s>>>(ctrl, gc, G);
  c.launches++;
}

void batch_pass_end(Ctx& c, GraphCtl* gc, int32_t G, const int64_t* newid, double tau_agg, bool last, Ctrl* ctrl) {
  k_batch_pass_end<<<1, 1024, 0, c.s>>>(gc, G, newid, tau_agg, last ? 1 : 0, ctrl);
  c.launches++;
}

template <class A>
void batch_next_level(Ctx& c, int32_t* Cp, int64_t n_cur, const int64_t* newid, const int32_t* vg, GraphCtl* gc,
                      int32_t G, int32_t* C, int64_t n0, const int32_t* vg0, const A* sig, const int32_t* occ,
                      A* k_next, int32_t* vg_next) {
  const int cap = c.num_sms * 8;
  k_batch_relabel<<<grid_for(n_cur, kBlock, cap), kBlock, 0, c.s>>>(Cp, n_cur, newid, vg, gc);
  k_batch_lookup<<<grid_for(n0, kBlock, cap), kBlock, 0, c.s>>>(C, n0, vg0, gc, Cp);
  k_batch_next_level<A><<<grid_for(n_cur, kBlock, cap), kBlock, 0, c.s>>>(sig, occ, newid, vg, gc, n_cur, k_next, Cp,
                                                                           vg_next);
  k_batch_advance<<<grid_for(G, kBlock, cap), kBlock, 0, c.s>>>(gc, G);
  c.launches += 4;
}

void batch_close(Ctx& c, int32_t* C, int64_t n0, const int32_t* vg0, GraphCtl* gc, int32_t G) {
  const int cap = c.num_sms * 8;
  if (n0 > 0) k_batch_close<<<grid_for(n0, kBlock, cap), kBlock, 0, c.s>>>(C, n0, vg0, gc);
  k_batch_close_ctl<<<grid_for(G, kBlock, cap), kBlock, 0, c.s>>>(gc, G);
  c.launches += 2;
}

template <class M>
void batch_modularity(Ctx& c, const GraphView<typename M::w_t>& g0, const int32_t* C, const int32_t* vg0, GraphCtl* gc,
                      int32_t G, const int64_t* vo, const int32_t* dperm, const int64_t* hb, typename M::a_t* intra,
                      typename M::a_t* tot, int64_t n_comm_total) {
  typedef typename M::a_t A;
  k_batch_comm_base<<<1, 1024, 0, c.s>>>(gc, G);
  c.launches++;
  if (n_comm_total > 0) cudaMemsetAsync(tot, 0, (size_t)n_comm_total * sizeof(A), c.s);
  if (g0.n > 0) cudaMemsetAsync(intra, 0, (size_t)g0.n * sizeof(A), c.s);  // isolated vertices stay 0
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    const int64_t cnt = hb[b + 1] - hb[b];
    if (cnt <= 0) continue;
    const int32_t* l = dperm + hb[b];
    switch (b) {
      case 0: k_bmod_group<M, 4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(g0, l, cnt, C, vg0, gc, intra, tot); break;
      case 1: k_bmod_group<M, 8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(g0, l, cnt, C, vg0, gc, intra, tot); break;
      case 2:
      case 3: k_bmod_group<M, 32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(g0, l, cnt, C, vg0, gc, intra, tot); break;
      default: k_bmod_group<M, 256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(g0, l, cnt, C, vg0, gc, intra, tot); break;
    }
    c.launches++;
  }
  k_bmod_final<M><<<grid_for(G, 1, c.num_sms * 16), kBlock, 0, c.s>>>(gc, G, vo, intra, tot);
  c.launches++;
}

#define LV_BATCH_INST(M)                                                                                           \
  template void batch_two_m<M>(Ctx&, GraphCtl*, int32_t, const M::a_t*, Ctrl*);                                          \
  template void batch_finish<M>(Ctx&, Ctrl*, GraphCtl*, int32_t);                                                 \
  template void batch_next_level<M::a_t>(Ctx&, int32_t*, int64_t, const int64_t*, const int32_t*, GraphCtl*,       \
                                         int32_t, int32_t*, int64_t, const int32_t*, const M::a_t*, const int32_t*, \
                                         M::a_t*, int32_t*);                                                       \
  template void batch_modularity<M>(Ctx&, const GraphView<M::w_t>&, const int32_t*, const int32_t*, GraphCtl*,     \
                                    int32_t, const int64_t*, const int32_t*, const int64_t*, M::a_t*, M::a_t*,      \
                                    int64_t);
LV_BATCH_INST(IntMode)
LV_BATCH_INST(FpMode)

}  // namespace lv
