// modularity.cu -- Eq. 1 (second form) on the GPU:
//   Q = sum_c [ sigma_c / 2m - (Sigma_c / 2m)^2 ],
// sigma = total weight of arcs whose ends share a community, Sigma_c = sum of K_i over c.
// Integer mode: Q = (2m * sigma - sum_c Sigma_c^2) / (2m)^2 from exact int64 sums (both terms are
// at most (2m)^2 < 2^62), one correctly rounded division -- the same value a CPU computes.
#include "flat.cuh"
#include "internal.cuh"

namespace lv {

template <class M>
__global__ void __launch_bounds__(kBlock) k_mod_rows(GraphView<typename M::w_t> g, const int32_t* C,
                                                     typename M::a_t* tot, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ FlatRows fr;
  __shared__ A rowk[kBlock];
  __shared__ int32_t rowc[kBlock];
  __shared__ A red[32];
  A sig = A(0), tm = A(0);
  for (int64_t r0 = (int64_t)blockIdx.x * kBlock; r0 < g.n; r0 += (int64_t)gridDim.x * kBlock) {
    const int64_t r = r0 + threadIdx.x;
    rowk[threadIdx.x] = A(0);
    rowc[threadIdx.x] = r < g.n ? C[r] : -1;
    const int64_t total = flat_load(fr, r0, g.n, g.rbeg, g.rend);  // syncs
    const int64_t nf = (total + kBlock - 1) / kBlock * kBlock;       // uniform trip count
    for (int64_t f = threadIdx.x; f < nf; f += kBlock) {
      int row = kBlock;  // sentinel for lanes past the end
      A w = A(0);
      if (f < total) {
        row = flat_row(fr, f);
        const int64_t e = fr.beg[row] + (f - fr.excl[row]);
        w = (A)g.w[e];
        if (C[g.tg[e]] == rowc[row]) sig += w;
      }
      bool tail;
      const A s = warp_seg_scan<A>(row, w, tail);
      if (tail && row < kBlock) atomic_add_a(&rowk[row], s);
    }
    __syncthreads();
    if (r < g.n) {
      const A k = rowk[threadIdx.x];
      if (k != A(0)) atomic_add_a(&tot[rowc[threadIdx.x]], k);
      tm += k;
    }
    __syncthreads();
  }
  sig = group_sum<kBlock>(sig, red);
  tm = group_sum<kBlock>(tm, red);
  if (threadIdx.x == 0) {
    if (M::is_fp) { atomicAdd(&ctrl->acc_f[0], (double)sig); atomicAdd(&ctrl->acc_f[1], (double)tm); }
    else { atomic_add_a(&ctrl->acc_i[0], (long long)sig); atomic_add_a(&ctrl->acc_i[1], (long long)tm); }
  }
}

template <class M>
__global__ void k_mod_squares(const typename M::a_t* tot, int64_t n, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  A s = A(0);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const A t = tot[c];
    s += t * t;
  }
  s = group_sum<kBlock>(s, red);
  if (threadIdx.x == 0) {
    if (M::is_fp) atomicAdd(&ctrl->acc_f[2], (double)s);
    else atomic_add_a(&ctrl->acc_i[2], (long long)s);
  }
}

template <bool FP>
__global__ void k_mod_final(Ctrl* c) {
  if (FP) {
    const double tm = c->acc_f[1];
    c->q = tm == 0.0 ? 0.0 : __dsub_rn(__ddiv_rn(c->acc_f[0], tm), __ddiv_rn(c->acc_f[2], __dmul_rn(tm, tm)));
  } else {
    const long long tm = c->acc_i[1];
    if (tm == 0) { c->q = 0.0; return; }
    const long long num = tm * c->acc_i[0] - c->acc_i[2];
    const long long den = tm * tm;
    c->q = __ddiv_rn(__ll2double_rn(num), __ll2double_rn(den));
  }
}

__global__ void k_mod_reset(Ctrl* c) {
  for (int k = 0; k < 4; k++) { c->acc_i[k] = 0; c->acc_f[k] = 0.0; }
  c->q = 0.0;
}

template <class M>
void modularity(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* C, typename M::a_t* tot, Ctrl* ctrl) {
  k_mod_reset<<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
  if (g.n > 0) {
    cudaMemsetAsync(tot, 0, (size_t)g.n * sizeof(typename M::a_t), c.s);
    k_mod_rows<M><<<grid_for(g.n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(g, C, tot, ctrl);
    k_mod_squares<M><<<grid_for(g.n, kBlock * 8, c.num_sms * 4), kBlock, 0, c.s>>>(tot, g.n, ctrl);
    c.launches += 2;
  }
  k_mod_final<M::is_fp><<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
}

// Degree-bucketed form: one group of G threads per vertex (the lists of a degree-bucket sort),
// giant rows by arc chunks, so no block is stuck with a hub's row.
template <class M, int G>
__global__ void __launch_bounds__(kBlock) k_mod_group(GraphView<typename M::w_t> g, const int32_t* list, int64_t count,
                                                      const int32_t* C, typename M::a_t* tot, Ctrl* ctrl) {
  typedef typename M::a_t A;
  __shared__ A red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  A sig = A(0), tm = A(0);
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t i = list[idx];
    const int32_t ci = C[i];
    A k = A(0);
    for (int64_t e = g.rbeg[i] + lane; e < g.rend[i]; e += G) {
      const A w = (A)g.w[e];
      k += w;
      if (C[g.tg[e]] == ci) sig += w;
    }
    k = group_sum<G>(k, red);
    if (lane == 0) {
      atomic_add_a(&tot[ci], k);
      tm += k;
    }
  }
  sig = group_sum<kBlock>(sig, red);
  tm = group_sum<kBlock>(tm, red);
  if (threadIdx.x == 0) {
    if (M::is_fp) { atomicAdd(&ctrl->acc_f[0], (double)sig); atomicAdd(&ctrl->acc_f[1], (double)tm); }
    else { atomic_add_a(&ctrl->acc_i[0], (long long)sig); atomic_add_a(&ctrl->acc_i[1], (long long)tm); }
  }
}

template <class M>
void modularity_bucketed(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* C, typename M::a_t* tot,
                         Ctrl* ctrl, const int32_t* dperm, const int64_t* hb, const GiantPlan& gp) {
  k_mod_reset<<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
  if (g.n > 0) {
    cudaMemsetAsync(tot, 0, (size_t)g.n * sizeof(typename M::a_t), c.s);
    const int cap = c.num_sms * 16;
    for (int b = 0; b < kNumBuckets; b++) {
      const int64_t cnt = hb[b + 1] - hb[b];
      if (cnt <= 0) continue;
      const int32_t* l = dperm + hb[b];
      switch (b) {
        case 0: k_mod_group<M, 4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(g, l, cnt, C, tot, ctrl); break;
        case 1: k_mod_group<M, 8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(g, l, cnt, C, tot, ctrl); break;
        case 2:
        case 3: k_mod_group<M, 32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(g, l, cnt, C, tot, ctrl); break;
        case 4:
        case 5: k_mod_group<M, 256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(g, l, cnt, C, tot, ctrl); break;
        default: giant_modularity<M>(c, g, l, cnt, C, tot, gp, ctrl); c.launches--; break;
      }
      c.launches++;
    }
    k_mod_squares<M><<<grid_for(g.n, kBlock * 8, c.num_sms * 4), kBlock, 0, c.s>>>(tot, g.n, ctrl);
    c.launches++;
  }
  k_mod_final<M::is_fp><<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
}

template void modularity_bucketed<IntMode>(Ctx&, const GraphView<int32_t>&, const int32_t*, long long*, Ctrl*,
                                           const int32_t*, const int64_t*, const GiantPlan&);
template void modularity_bucketed<FpMode>(Ctx&, const GraphView<float>&, const int32_t*, double*, Ctrl*,
                                          const int32_t*, const int64_t*, const GiantPlan&);
template void modularity<IntMode>(Ctx&, const GraphView<int32_t>&, const int32_t*, long long*, Ctrl*);
template void modularity<FpMode>(Ctx&, const GraphView<float>&, const int32_t*, double*, Ctrl*);

}  // namespace lv
