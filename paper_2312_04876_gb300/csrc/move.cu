// move.cu -- the local-moving phase of Algorithm 2 on the GPU.
//
// One group of G threads handles one vertex i (G by degree bucket: 4, 8, 32 lanes or a whole
// block; rows above 4096 arcs take the multi-block path of giant.cu, whose tables live in global
// memory).  The group streams i's arcs (scanCommunities with self = false), accumulates
// K_i->c for every neighbouring community c != C'[i] in an open-addressing table in shared
// memory and K_i->d in registers, then scores
// every candidate with the Eq. 2 numerator
//     N(c) = 2m (K_i->c - K_i->d) - K_i (Sigma_c - Sigma_d + K_i)
// (exact int64 for int32 weights), takes the best with ties to the smallest id and moves iff
// N > 0.  Deterministic mode records the move and defers the Sigma update to move_apply (the
// colour class decides against class-start totals); fast mode applies it at once with atomics.
// A moved vertex re-marks its neighbours for processing (vertex pruning, Section 4.1.6).  The
// sum of the performed N is accumulated exactly (128-bit) and move_finish applies the
// per-iteration tolerance test of Algorithm 2 on the device, so iterations need no host sync.
#include <atomic>
#include <type_traits>

#include "internal.cuh"

namespace lv {

template <class M>
struct LmArgs {
  GraphView<typename M::w_t> g;
  PassState<M> st;
  const int32_t* list;
  int64_t count;
  int fast;
  int pruning;
  int bucket;
  const int64_t* rng;  // device {start, count} of the list (a captured iteration), or null
  int tf;              // table slots per key of the row's distinct-key bound
};

// Block-wide reduction of the per-thread move accumulators into the control block.
template <bool FP>
__device__ __forceinline__ void flush_move_acc(Ctrl* ctrl, unsigned long long lo, unsigned long long hi,
                                               unsigned long long mv, double f, unsigned long long* s_lo,
                                               unsigned long long* s_hi, unsigned long long* s_mv, double* s_f) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
    unsigned long long hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    unsigned long long s = lo + lo2;
    hi += hi2 + (s < lo ? 1ULL : 0ULL);
    lo = s;
    mv += __shfl_xor_sync(0xffffffffu, mv, o);
    if (FP) f += __shfl_xor_sync(0xffffffffu, f, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; s_mv[threadIdx.x >> 5] = mv; s_f[threadIdx.x >> 5] = f;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tl = 0, th = 0, tm = 0;
    double tf = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      unsigned long long s = tl + s_lo[w];
      th += s_hi[w] + (s < tl ? 1ULL : 0ULL);
      tl = s;
      tm += s_mv[w];
      tf += s_f[w];
    }
    if (tm) {
      atomicAdd(&ctrl->moves, tm);
      if (FP) atomicAdd(&ctrl->sum_f, tf);
      else atomic_add_u128(&ctrl->sum_lo, &ctrl->sum_hi, tl, th);
    }
  }
}

// Threads per block: warps with 1024-slot tables run in two-warp blocks, so a block (and its
// shared memory) retires after two vertices instead of waiting for the slowest of eight.
template <int G, int LOG>
__host__ __device__ constexpr int lm_block() {
  return (G == 32 && LOG >= 10) ? 64 : kBlock;
}

// Blocks per SM the register budget is set for: two-warp blocks are held to 12 per SM by their
// 16 KB of tables and lists anyway, so they may use up to 85 registers a thread.
template <int G, int LOG>
__host__ __device__ constexpr int lm_min_blocks() {
  return lm_block<G, LOG>() == 64 ? 12 : (G <= 32 ? 4 : 3);
}

template <class M, int G, int LOG>
__global__ void __launch_bounds__(lm_block<G, LOG>(), (lm_min_blocks<G, LOG>())) lm_kernel(LmArgs<M> a) {
  typedef typename M::h_t H;
  typedef typename M::a_t A;
  typedef typename M::s_t S;
  Ctrl* ctrl = a.st.ctrl;
  if (*(volatile int32_t*)&ctrl->done) return;
  constexpr int BS = lm_block<G, LOG>();
  constexpr int GPB = G <= 32 ? BS / G : 1;
  // a captured iteration reads its list range from device memory (32-bit: counts and offsets are
  // below 2^31); the graph's arrays stay kernel parameters
  int32_t lo = 0, hi = (int32_t)a.count;  // list[lo, hi)
  if (a.rng) {
    lo = (int32_t)a.rng[0];
    hi = lo + (int32_t)a.rng[1];
  }
  if (lo + (int)blockIdx.x * GPB >= hi) return;  // a fixed grid larger than this range
  const GraphView<typename M::w_t>& g = a.g;
  constexpr int SL = 1 << LOG;
  constexpr int U = G >= 32 ? 4 : 2;  // arcs (and table slots) per lane per step
  extern __shared__ __align__(16) unsigned char lm_dyn[];  // GPB tables of SL (key, value) slots
  int32_t* skeys = reinterpret_cast<int32_t*>(lm_dyn);
  H* svals = reinterpret_cast<H*>(lm_dyn + sizeof(int32_t) * GPB * SL);
  // warp and block groups: the slots each vertex claimed, in claim order (a row has at most SL / 2
  // distinct neighbouring communities, since tables hold at least twice the row's arcs), so the
  // scoring visits and clears only occupied slots
  constexpr bool kList = G >= 32;
  constexpr int LMAX = kList ? SL / 2 : 1;
  uint16_t* slist = reinterpret_cast<uint16_t*>(lm_dyn + (sizeof(int32_t) + sizeof(H)) * GPB * SL);
  __shared__ int s_ncl;  // block groups: entries of the claimed-slot list
  // per-warp reduction scratch, sized by the block's warps: static shared memory counts against
  // the blocks an SM holds (13 instead of 11 two-warp blocks of 1024-slot tables)
  constexpr int NW = BS / 32;
  static_assert(BS % 32 == 0 && BS <= kBlock, "whole warps, at most kBlock threads");
  __shared__ S red_s[NW];
  __shared__ int32_t red_c[NW];
  __shared__ H red_h[NW];
  __shared__ int32_t red_i[NW];
  __shared__ unsigned long long r_lo[NW], r_hi[NW], r_mv[NW];
  __shared__ double r_f[NW];

  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int t = threadIdx.x; t < GPB * SL; t += BS) { skeys[t] = kEmpty; svals[t] = H(0); }
  if (threadIdx.x == 0) s_ncl = 0;
  __syncthreads();
  int32_t* tk = skeys + gib * SL;  // this group's table
  H* tv = svals + gib * SL;
  uint16_t* cl = slist + gib * LMAX;  // this group's claimed-slot list
  const A two_m_all = M::is_fp ? (A)ctrl->two_m_f : (A)ctrl->two_m_i;
  GraphCtl* const gcs = a.st.gc;
  unsigned long long acc_lo = 0, acc_hi = 0, acc_mv = 0;
  double acc_f = 0.0;
  unsigned long long ctr[6] = {0, 0, 0, 0, 0, 0};  // list, processed, arcs, candidates, moves, marks

  const int64_t ngroups = (int64_t)gridDim.x * GPB;
  for (int32_t idx = lo + (int32_t)blockIdx.x * GPB + gib; idx < hi; idx += (int32_t)ngroups) {
    const int32_t i = a.list[idx];
    if (lane == 0) ctr[0]++;
    // batched run: the graph of i, skipped once its local-moving phase has converged
    GraphCtl* gcv = nullptr;
    if (gcs) {
      gcv = gcs + a.st.vg[i];
      if (*(volatile int32_t*)&gcv->done) continue;
    }
    const A two_m = gcv ? (M::is_fp ? (A)gcv->two_m_f : (A)gcv->two_m_i) : two_m_all;
    // row bounds, C'[i] and the flag are loaded together (the loads overlap)
    const int64_t beg = g.rbeg[i], end = g.rend[i];
    const int32_t d = a.st.Cp[i];
    if (a.pruning) {
      // every lane reads the flag and the group takes the OR, so the decision is uniform even if a
      // neighbour re-marks i meanwhile; then i is marked as processed
      const int f = a.st.flags[i];
      if (!group_any<G>(f != 0)) continue;
      if (lane == 0) a.st.flags[i] = 0;
    }
    const int64_t deg = end - beg;
    if (lane == 0) { ctr[1]++; ctr[2] += (unsigned long long)deg; }
    // K_i and Sigma_d are needed only for scoring; loaded here they overlap the arc loads (in the
    // deterministic schedule Sigma does not change during a class; the fast schedule reads live values)
    const A ki = a.st.K[i];
    const A sd = a.st.Sig[d];
    const int lg = G > 32 ? tbl_log2f(deg, a.tf, 1, LOG) : tbl_log2f_fast(deg, a.tf, 1, LOG);
    const unsigned size = 1u << lg;
    const int shift = 32 - lg;

    // scanCommunities(i, self = false): K_i->c into the table, K_i->d in registers.  U arcs per
    // lane are loaded before their C'[j] gathers and the table updates, so each lane keeps U
    // independent memory requests in flight.
    H kid = H(0);
    bool ok = true;
    unsigned ncl = 0;  // warp groups: entries of the claimed-slot list (uniform over the warp)
    // every lane of a warp takes the same number of steps (the claim ballots need the whole warp)
    // Warp and sub-warp groups index a row's arcs from its start in 32 bits (a row holds fewer than
    // 2^31 arcs; fewer instructions per arc); the one-block kernels keep absolute 64-bit indices,
    // which measured faster there.
    typedef typename std::conditional<(G > 32), int64_t, int32_t>::type X;
    const int32_t* const rtg = G > 32 ? g.tg : g.tg + beg;
    const typename M::w_t* const rw = G > 32 ? g.w : g.w + beg;
    const X rlo = G > 32 ? (X)beg : X(0), rhi = G > 32 ? (X)end : (X)deg;
    for (X b0 = rlo; b0 < rhi; b0 += (X)(G * U)) {
      const X e0 = b0 + (X)lane;
      int32_t jj[U];
      H ww[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const X e = e0 + (X)(u * G);
        jj[u] = e < rhi ? rtg[e] : i;
        ww[u] = e < rhi ? (H)rw[e] : H(0);
      }
      int32_t cc[U];
#pragma unroll
      for (int u = 0; u < U; u++) cc[u] = jj[u] != i ? a.st.Cp[jj[u]] : kEmpty;
#pragma unroll
      for (int u = 0; u < U; u++) {
        const bool other = jj[u] != i && cc[u] != d;  // padding and i's self-loop are neither
        if (jj[u] != i && cc[u] == d) kid += ww[u];
        if constexpr (kList) {
          // the new keys of this step are appended warp by warp to the claimed-slot list
          int r = 1;
          unsigned sl = 0;
          if (other) r = tbl_add_claim(tk, tv, size, shift, cc[u], ww[u], &sl);
          ok &= r != 0;
          const unsigned b = __ballot_sync(0xffffffffu, r == 2);
          if (b != 0u) {
            unsigned base;
            if constexpr (G == 32) {
              base = ncl;
              ncl += __popc(b);
            } else {
              unsigned t = 0;
              if ((threadIdx.x & 31) == 0) t = (unsigned)atomicAdd(&s_ncl, __popc(b));
              base = __shfl_sync(0xffffffffu, t, 0);
            }
            if (r == 2) cl[base + __popc(b & lanemask_lt())] = (uint16_t)sl;
          }
        } else if (other) {
          ok &= tbl_add(tk, tv, size, shift, cc[u], ww[u]);
        }
      }
    }
    if (!ok) atomicOr(&ctrl->error, kErrTableFull);
    Grp<G>::sync();
    kid = group_sum<G>(kid, red_h);

    // best community by the Eq. 2 numerator; the scan also clears the table.  The Sigma gathers of
    // U slots per lane are issued together.
    S best = M::lowest();
    int32_t bc = 0x7fffffff;
    // Warp and block groups score the slots listed at claim time (U per lane, their Sigma gathers
    // issued together) and clear them, which leaves the table all-empty; sub-warp groups scan their
    // small tables directly.
    if constexpr (kList) {
      const unsigned ncand = G == 32 ? ncl : (unsigned)*(volatile int*)&s_ncl;
      for (unsigned k0 = lane; k0 < ncand; k0 += (unsigned)G * U) {
        int32_t ck[U];
        H vv[U];
        A sg[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const unsigned k = k0 + (unsigned)u * G;
          ck[u] = kEmpty;
          vv[u] = H(0);
          if (k < ncand) {
            const unsigned s = cl[k];
            ck[u] = tk[s];
            vv[u] = tv[s];
            tk[s] = kEmpty;
            tv[s] = H(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) sg[u] = ck[u] != kEmpty ? a.st.Sig[ck[u]] : A(0);
#pragma unroll
        for (int u = 0; u < U; u++) {
          if (ck[u] == kEmpty) continue;
          ctr[3]++;
          const S sc = M::score(vv[u], kid, ki, sg[u], sd, two_m);
          if (better(sc, ck[u], best, bc)) { best = sc; bc = ck[u]; }
        }
      }
    } else {
      for (unsigned s0 = lane; s0 < size; s0 += (unsigned)G * U) {
        int32_t ck[U];
        H vv[U];
        A sg[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const unsigned s = s0 + (unsigned)u * G;
          ck[u] = s < size ? tk[s] : kEmpty;
          vv[u] = H(0);
          if (ck[u] != kEmpty) {
            vv[u] = tv[s];
            tk[s] = kEmpty;
            tv[s] = H(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) sg[u] = ck[u] != kEmpty ? a.st.Sig[ck[u]] : A(0);
#pragma unroll
        for (int u = 0; u < U; u++) {
          if (ck[u] == kEmpty) continue;
          ctr[3]++;
          const S sc = M::score(vv[u], kid, ki, sg[u], sd, two_m);
          if (better(sc, ck[u], best, bc)) { best = sc; bc = ck[u]; }
        }
      }
    }
    group_argmax<G>(best, bc, red_s, red_c);
    if (G > 32 && threadIdx.x == 0) s_ncl = 0;  // every thread read it before group_argmax's barriers
    Grp<G>::sync();

    int mv = (bc != 0x7fffffff && best > S(0)) ? 1 : 0;
    if (mv && a.fast) {
      // singleton guard against lock-step swaps: a lone vertex joins another singleton
      // community only if that community's id is smaller
      int okm = 1;
      if (lane == 0 && a.st.csize[d] == 1 && a.st.csize[bc] == 1 && bc > d) okm = 0;
      mv = group_bcast<G>(okm, red_i);
    }
    if (mv) {
      if (lane == 0) {
        if (a.fast) {
          atomic_add_a(&a.st.Sig[d], -ki);
          atomic_add_a(&a.st.Sig[bc], ki);
          atomicSub(&a.st.csize[d], 1);
          atomicAdd(&a.st.csize[bc], 1);
        } else {
          a.st.mv_from[i] = d;
          a.st.mv_to[i] = bc;
        }
        a.st.Cp[i] = bc;
        if (gcv) {
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
        ctr[4]++;
      }
      if (a.pruning)
        for (X e0 = rlo + (X)lane; e0 < rhi; e0 += (X)(G * U)) {
          int32_t jj[U];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const X e = e0 + (X)(u * G);
            jj[u] = e < rhi ? rtg[e] : i;
          }
#pragma unroll
          for (int u = 0; u < U; u++)
            if (jj[u] != i) { a.st.flags[jj[u]] = 1; ctr[5]++; }  // mark neighbours as unprocessed
        }
    }
  }
  flush_move_acc<M::is_fp>(ctrl, acc_lo, acc_hi, acc_mv, acc_f, r_lo, r_hi, r_mv, r_f);
  block_add_counters<6, NW>(ctrl->lm_stat[a.bucket], ctr);
}

template <class M, int G, int LOG>
static constexpr size_t lm_smem() {
  return (size_t)(G <= 32 ? lm_block<G, LOG>() / G : 1) * (1 << LOG) *
         (sizeof(int32_t) + sizeof(typename M::h_t) + (G >= 32 ? sizeof(uint16_t) / 2 : 0));
}

// Opts a kernel into more than 48 KB of dynamic shared memory, once per device (outside any graph
// capture: move_prepare runs it for every instantiation before an iteration is captured).
template <class M, int G, int LOG>
static void lm_attr() {
  constexpr size_t smem = lm_smem<M, G, LOG>();
  if (smem <= 48 * 1024) return;
  static std::atomic<unsigned long long> done{0};  // one bit per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (done.load() >> dev) & 1ULL) return;
  cudaFuncSetAttribute(lm_kernel<M, G, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (dev < 64) done.fetch_or(1ULL << dev);
}

void move_prepare() {
  lm_attr<IntMode, 32, 10>();
  lm_attr<IntMode, 256, 13>();
  lm_attr<FpMode, 32, 10>();
  lm_attr<FpMode, 256, 13>();
}

template <class M, int G, int LOG>
static void launch_lm(Ctx& c, const LmArgs<M>& a, int max_blocks) {
  constexpr int BS = lm_block<G, LOG>();
  constexpr int GPB = G <= 32 ? BS / G : 1;
  constexpr size_t smem = lm_smem<M, G, LOG>();
  lm_attr<M, G, LOG>();
  // device-resident range: a.count is then an upper bound of the range (a power of two)
  const int grid = grid_for(a.count, GPB, max_blocks * (kBlock / BS));
  lm_kernel<M, G, LOG><<<grid, BS, smem, c.s>>>(a);
  c.launches++;
}

template <class M>
void move_bucket(Ctx& c, int bucket, const GraphView<typename M::w_t>& g, const PassState<M>& st,
                 const int32_t* list, int64_t count, bool fast, bool pruning,
                 const int64_t* rng) {
  if (count <= 0 && !rng) return;
  LmArgs<M> a;
  a.g = g; a.st = st; a.list = list; a.count = count;
  a.rng = rng;
  a.fast = fast ? 1 : 0;
  a.pruning = pruning ? 1 : 0;
  a.bucket = bucket < kNumBuckets ? bucket : kNumBuckets - 1;
  a.tf = c.table_factor;
  const int cap = c.num_sms * c.lm_blocks_per_sm;
  switch (bucket) {
    case 0: launch_lm<M, 4, 3>(c, a, cap); break;
    case 1: launch_lm<M, 8, 5>(c, a, cap); break;
    case 2: launch_lm<M, 32, 8>(c, a, cap); break;
    case 3: launch_lm<M, 32, 10>(c, a, cap); break;
    case 4: launch_lm<M, 256, 12>(c, a, cap); break;
    case 5: launch_lm<M, 256, 13>(c, a, cap); break;
    default: break;  // giants go through giant_move
  }
}

// ---------------------------------------------------------------- deterministic apply
template <class M>
__global__ void lm_apply(PassState<M> st, const int32_t* list, int64_t count, const int64_t* rng) {
  if (*(volatile int32_t*)&st.ctrl->done) return;
  if (rng) {
    list += rng[0];
    count = rng[1];
  }
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = list[k];
    const int32_t t = st.mv_to[i];
    if (t >= 0) {
      const typename M::a_t ki = st.K[i];
      atomic_add_a(&st.Sig[st.mv_from[i]], -ki);
      atomic_add_a(&st.Sig[t], ki);
      st.mv_to[i] = -1;
    }
  }
}
template <class M>
void move_apply(Ctx& c, const PassState<M>& st, const int32_t* list, int64_t count, const int64_t* rng) {
  if (count <= 0 && !rng) return;
  const int grid = rng ? c.num_sms * 8 : grid_for(count, kBlock, c.num_sms * 8);
  lm_apply<M><<<grid, kBlock, 0, c.s>>>(st, list, count, rng);
  c.launches++;
}

// ---------------------------------------------------------------- iteration control
// Algorithm 2's tolerance test on the device: converged iff 2 sum N <= tau (2m)^2, with the
// 128-bit sum rounded once to double (integer mode) and the right side as tau * (t * t).
template <bool FP>
__global__ void lm_finish(Ctrl* c) {
  if (c->done) return;
  const int it = c->iterations + 1;
  c->iterations = it;
  bool conv;
  if (FP) {
    conv = __dmul_rn(2.0, c->sum_f) <= __dmul_rn(c->tau, __dmul_rn(c->two_m_f, c->two_m_f));
  } else {
    const unsigned long long hi = (c->sum_hi << 1) | (c->sum_lo >> 63), lo = c->sum_lo << 1;
    const double lhs = u128_to_double_rn(hi, lo);
    const double t = __ll2double_rn(c->two_m_i);
    conv = lhs <= __dmul_rn(c->tau, __dmul_rn(t, t));
  }
  c->moves_pass += c->moves;
  c->moves = 0;
  c->sum_lo = 0;
  c->sum_hi = 0;
  c->sum_f = 0.0;
  if (conv || it >= c->max_iterations) c->done = 1;
}
template <class M>
void move_finish(Ctx& c, Ctrl* ctrl) {
  lm_finish<M::is_fp><<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
}

__global__ void k_move_setup(Ctrl* c, double tau, int max_iterations) {
  c->done = max_iterations <= 0 ? 1 : 0;
  c->iterations = 0;
  c->max_iterations = max_iterations;
  c->tau = tau;
  c->sum_lo = 0;
  c->sum_hi = 0;
  c->sum_f = 0.0;
  c->moves = 0;
  c->moves_pass = 0;
}
void move_setup(Ctx& c, Ctrl* ctrl, double tau, int max_iterations) {
  k_move_setup<<<1, 1, 0, c.s>>>(ctrl, tau, max_iterations);
  c.launches++;
}

// ---------------------------------------------------------------- share of the arcs in hub rows
__global__ void k_hub_share(const int64_t* rbeg, const int64_t* rend, int64_t n, Ctrl* ctrl) {
  unsigned long long hub = 0, all = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)(rend[i] - rbeg[i]);
    all += d;
    if (d > 512) hub += d;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    hub += __shfl_xor_sync(0xffffffffu, hub, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if ((threadIdx.x & 31) == 0 && all) {
    atomicAdd(&ctrl->hub_arcs, hub);
    atomicAdd(&ctrl->all_arcs, all);
  }
}
template <class W>
void hub_share(Ctx& c, const GraphView<W>& g, Ctrl* ctrl) {
  cudaMemsetAsync(&ctrl->hub_arcs, 0, 2 * sizeof(unsigned long long), c.s);
  if (g.n <= 0) return;
  k_hub_share<<<grid_for(g.n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(g.rbeg, g.rend, g.n, ctrl);
  c.launches++;
}
template void hub_share<int32_t>(Ctx&, const GraphView<int32_t>&, Ctrl*);
template void hub_share<float>(Ctx&, const GraphView<float>&, Ctrl*);

// ---------------------------------------------------------------- per-pass vertex state
template <class M>
__global__ void k_vertex_init(PassState<M> st, int64_t n, int from_k) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    st.Cp[i] = (int32_t)i;
    st.flags[i] = 1;
    st.csize[i] = 1;
    st.mv_to[i] = -1;
    if (from_k) {
      st.Sig[i] = st.K[i];
    } else {
      st.K[i] = 0;
      st.Sig[i] = 0;
    }
  }
}
template <class M>
void vertex_init(Ctx& c, const PassState<M>& st, int64_t n, bool from_k) {
  if (n <= 0) return;
  k_vertex_init<M><<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(st, n, from_k ? 1 : 0);
  c.launches++;
}

// K_i = sum of row weights (self-loop once), one group per vertex.
template <class M, int G>
__global__ void __launch_bounds__(kBlock) k_row_sums(GraphView<typename M::w_t> g, const int32_t* list, int64_t count,
                                                     typename M::a_t* K, typename M::a_t* Sig, typename M::a_t* K0) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t i = list[idx];
    A s = A(0);
    for (int64_t e = g.rbeg[i] + lane; e < g.rend[i]; e += G) s += (A)g.w[e];
    s = group_sum<G>(s, red);
    if (lane == 0) { K[i] = s; Sig[i] = s; if (K0) K0[i] = s; }
  }
}
template <class M>
void row_sums(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* perm, const int64_t* hb,
              typename M::a_t* K, typename M::a_t* Sig, typename M::a_t* K0) {
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    int64_t cnt = hb[b + 1] - hb[b];
    if (cnt <= 0) continue;
    const int32_t* l = perm + hb[b];
    switch (b) {
      case 0: k_row_sums<M, 4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(g, l, cnt, K, Sig, K0); break;
      case 1: k_row_sums<M, 8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(g, l, cnt, K, Sig, K0); break;
      case 2:
      case 3: k_row_sums<M, 32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(g, l, cnt, K, Sig, K0); break;
      default: k_row_sums<M, 256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(g, l, cnt, K, Sig, K0); break;
    }
    c.launches++;
  }
}

template <class M>
__global__ void k_total(const typename M::a_t* K, int64_t n, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  A s = A(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += K[i];
  s = group_sum<kBlock>(s, red);
  if (threadIdx.x == 0) {
    if (M::is_fp) atomicAdd(&ctrl->two_m_f, (double)s);
    else atomic_add_a(&ctrl->two_m_i, (long long)s);
  }
}
template <class M>
void total_weight(Ctx& c, const typename M::a_t* K, int64_t n, Ctrl* ctrl) {
  if (n <= 0) return;
  k_total<M><<<grid_for(n, kBlock * 8, c.num_sms * 4), kBlock, 0, c.s>>>(K, n, ctrl);
  c.launches++;
}

#define LV_MOVE_INST(M)                                                                                           \
  template void vertex_init<M>(Ctx&, const PassState<M>&, int64_t, bool);                                        \
  template void row_sums<M>(Ctx&, const GraphView<M::w_t>&, const int32_t*, const int64_t*, M::a_t*, M::a_t*,    \
                            M::a_t*);                                                                            \
  template void total_weight<M>(Ctx&, const M::a_t*, int64_t, Ctrl*);                                            \
  template void move_bucket<M>(Ctx&, int, const GraphView<M::w_t>&, const PassState<M>&, const int32_t*, int64_t, \
                               bool, bool, const int64_t*);                                                      \
  template void move_apply<M>(Ctx&, const PassState<M>&, const int32_t*, int64_t, const int64_t*);               \
  template void move_finish<M>(Ctx&, Ctrl*);
LV_MOVE_INST(IntMode)
LV_MOVE_INST(FpMode)

}  // namespace lv
