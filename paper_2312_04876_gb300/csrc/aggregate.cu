// aggregate.cu -- the aggregation phase of Algorithm 3 on the GPU.
//
//  1. community-vertex CSR: member counts and community total degrees by atomics, exclusive
//     scans (host side), then an unordered scatter of the members (countCommunityVertices /
//     exclusiveScan / "add edge (C'[i], i) atomically");
//  2. super-vertex graph: the holey offsets are the scan of the community total degrees (an
//     over-estimate of every super-degree, as the paper does); one group per community (G by
//     total-degree bucket) streams the arcs of all members -- flattened so that G lanes always
//     work on G arcs even when members have tiny rows -- and sums the arc weight per
//     neighbouring community, its own included (scanCommunities with self = true), in an
//     open-addressing table; the group then writes the (d, w) pairs at the start of its holey
//     row and records the row end;
//  3. compaction (optional): scan of the super-degrees, then a block-flat copy of the rows.
#include "internal.cuh"

namespace lv {

__global__ void k_comm_count(const int32_t* Cp, const int64_t* rbeg, const int64_t* rend, int64_t n, int32_t* counts,
                             int64_t* cdeg) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = Cp[i];
    if (c < 0) continue;  // batched: the graph of i left the pass loop
    atomicAdd(&counts[c], 1);
    const int64_t d = rend[i] - rbeg[i];
    if (d) atomicAdd(reinterpret_cast<unsigned long long*>(&cdeg[c]), (unsigned long long)d);
  }
}
void community_count(Ctx& c, const int32_t* Cp, const int64_t* rbeg, const int64_t* rend, int64_t n, int32_t* counts,
                     int64_t* cdeg) {
  if (n <= 0) return;
  k_comm_count<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(Cp, rbeg, rend, n, counts, cdeg);
  c.launches++;
}

__global__ void k_comm_fill(const int32_t* Cp, int64_t n, const int64_t* coff, int32_t* cursor, int32_t* cverts) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = Cp[i];
    if (c < 0) continue;
    cverts[coff[c] + atomicAdd(&cursor[c], 1)] = (int32_t)i;
  }
}
void community_fill(Ctx& c, const int32_t* Cp, int64_t n, const int64_t* coff, int32_t* cursor, int32_t* cverts) {
  if (n <= 0) return;
  k_comm_fill<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(Cp, n, coff, cursor, cverts);
  c.launches++;
}

// Owner of flat index f among W lanes holding inclusive prefix sums `incl` (non-decreasing):
// the number of lanes whose prefix is <= f.  All W lanes of the (sub-)warp must call it.
template <int W>
__device__ __forceinline__ int flat_owner(int64_t incl, int64_t f, unsigned mask) {
  int lo = 0;
#pragma unroll
  for (int step = W / 2; step >= 1; step >>= 1) {
    const int64_t v = __shfl_sync(mask, incl, lo + step - 1, W);
    if (v <= f) lo += step;
  }
  return lo;
}

// Inclusive scan over W lanes.
template <int W>
__device__ __forceinline__ int64_t lanes_incl_scan(int64_t x, unsigned mask) {
  const int l = threadIdx.x & (W - 1);
#pragma unroll
  for (int o = 1; o < W; o <<= 1) {
    const int64_t y = __shfl_up_sync(mask, x, o, W);
    if (l >= o) x += y;
  }
  return x;
}

// Insert the arcs of members [k0, k1) of a community, W lanes flattening W members at a time.
template <class M, int W>
__device__ __forceinline__ bool merge_members(const MergeArgs<M>& a, int64_t k0, int64_t k1, int64_t kstride,
                                              int32_t* tk, typename M::h_t* tv, unsigned size, int shift,
                                              unsigned mask, unsigned long long& arcs) {
  typedef typename M::h_t H;
  const int l = threadIdx.x & (W - 1);
  bool ok = true;
  for (int64_t kb = k0; kb < k1; kb += kstride) {
    const int64_t k = kb + l;
    int64_t b = 0, len = 0;
    if (k < k1) {
      const int32_t i = a.cverts[k];
      b = a.g.rbeg[i];
      len = a.g.rend[i] - b;
    }
    const int64_t incl = lanes_incl_scan<W>(len, mask);
    const int64_t total = __shfl_sync(mask, incl, W - 1, W);
    const int64_t excl = incl - len;
    arcs += (unsigned long long)len;
    // U flat arcs per lane per step: their target / weight loads, then their C'[j] gathers, then
    // the table updates, so each lane keeps U independent memory requests in flight
    constexpr int U = 4;
    for (int64_t f0 = 0; f0 < total; f0 += (int64_t)W * U) {
      int64_t ee[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t f = f0 + (int64_t)u * W + l;
        const int o = flat_owner<W>(incl, f, mask);
        const int64_t ob = __shfl_sync(mask, b, o, W);
        const int64_t oe = __shfl_sync(mask, excl, o, W);
        ee[u] = f < total ? ob + (f - oe) : -1;
      }
      int32_t jj[U];
      H ww[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        jj[u] = ee[u] >= 0 ? a.g.tg[ee[u]] : 0;
        ww[u] = ee[u] >= 0 ? (H)a.g.w[ee[u]] : H(0);
      }
      int32_t cc[U];
#pragma unroll
      for (int u = 0; u < U; u++) cc[u] = ee[u] >= 0 ? a.Cp[jj[u]] : kEmpty;
#pragma unroll
      for (int u = 0; u < U; u++)
        if (ee[u] >= 0) ok &= tbl_add(tk, tv, size, shift, cc[u], ww[u]);
    }
  }
  return ok;
}

// Block version for the one-community-per-block buckets: all kBlock threads flatten the arcs of
// kBlock members at a time (block-wide prefix of their row lengths in shared memory, a binary
// search per arc), so a community dominated by one long member row keeps every warp busy.
template <class M>
__device__ __forceinline__ bool merge_members_block(const MergeArgs<M>& a, int64_t k0, int64_t k1, int32_t* tk,
                                                    typename M::h_t* tv, unsigned size, int shift,
                                                    unsigned long long& arcs, int64_t* s_incl, int64_t* s_base,
                                                    int64_t* s_wsum) {
  typedef typename M::h_t H;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  bool ok = true;
  for (int64_t kb = k0; kb < k1; kb += kBlock) {
    const int64_t k = kb + t;
    int64_t b = 0, len = 0;
    if (k < k1) {
      const int32_t i = a.cverts[k];
      b = a.g.rbeg[i];
      len = a.g.rend[i] - b;
    }
    arcs += (unsigned long long)len;
    int64_t incl = lanes_incl_scan<32>(len, 0xffffffffu);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; w++) before += s_wsum[w];
    incl += before;
    s_incl[t] = incl;
    s_base[t] = b - (incl - len);  // arc of flat position f in this member: s_base + f
    __syncthreads();
    const int64_t total = s_incl[kBlock - 1];
    constexpr int U = 4;
    for (int64_t f0 = 0; f0 < total; f0 += (int64_t)kBlock * U) {
      int64_t ee[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int64_t f = f0 + (int64_t)u * kBlock + t;
        int lo = 0;  // members whose inclusive prefix is <= f
#pragma unroll
        for (int step = kBlock / 2; step >= 1; step >>= 1)
          if (s_incl[lo + step - 1] <= f) lo += step;
        ee[u] = f < total ? s_base[lo] + f : -1;
      }
      int32_t jj[U];
      H ww[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        jj[u] = ee[u] >= 0 ? a.g.tg[ee[u]] : 0;
        ww[u] = ee[u] >= 0 ? (H)a.g.w[ee[u]] : H(0);
      }
      int32_t cc[U];
#pragma unroll
      for (int u = 0; u < U; u++) cc[u] = ee[u] >= 0 ? a.Cp[jj[u]] : kEmpty;
#pragma unroll
      for (int u = 0; u < U; u++)
        if (ee[u] >= 0) ok &= tbl_add(tk, tv, size, shift, cc[u], ww[u]);
    }
    __syncthreads();  // s_incl / s_base / s_wsum are rewritten
  }
  return ok;
}

template <class M, int G, int LOG>
__global__ void __launch_bounds__(kBlock) merge_kernel(MergeArgs<M> a, const int32_t* list, int64_t count) {
  typedef typename M::h_t H;
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  constexpr int SL = 1 << LOG;
  extern __shared__ __align__(16) unsigned char mg_dyn[];  // GPB tables of SL (key, value) slots
  int32_t* skeys = reinterpret_cast<int32_t*>(mg_dyn);
  H* svals = reinterpret_cast<H*>(mg_dyn + sizeof(int32_t) * GPB * SL);
  __shared__ unsigned long long s_cnt;
  __shared__ int64_t s_incl[G > 32 ? kBlock : 1], s_base[G > 32 ? kBlock : 1], s_wsum[kBlock / 32];
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int t = threadIdx.x; t < GPB * SL; t += kBlock) { skeys[t] = kEmpty; svals[t] = H(0); }
  __syncthreads();
  int32_t* tk = skeys + gib * SL;
  H* tv = svals + gib * SL;
  unsigned long long ctr[4] = {0, 0, 0, 0};  // communities, members, arcs scanned, arcs written
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t c = list[idx];
    const int64_t m0 = a.coff[c], m1 = a.coff[c + 1];
    if (lane == 0) { ctr[0]++; ctr[1] += (unsigned long long)(m1 - m0); }
    const int64_t D = a.cdeg[c];
    const int lg = tbl_log2f(D, a.tf, 1, LOG);
    const unsigned size = 1u << lg;
    const int shift = 32 - lg;
    bool ok;
    if (G <= 32) {
      // each lane adds the row lengths of the members it loaded
      ok = merge_members<M, (G <= 32 ? G : 32)>(a, m0, m1, G, tk, tv, size, shift, Grp<G>::mask(), ctr[2]);
    } else {
      ok = merge_members_block<M>(a, m0, m1, tk, tv, size, shift, ctr[2], s_incl, s_base, s_wsum);
    }
    if (!ok) atomicOr(&a.ctrl->error, kErrTableFull);
    Grp<G>::sync();
    // emit the (community, weight) pairs at the start of the holey row of c
    const int64_t base = a.hoff[c];
    if (G <= 32) {
      const unsigned gm = Grp<G>::mask();
      unsigned cnt = 0;
      for (unsigned s0 = 0; s0 < size; s0 += G) {
        const unsigned s = s0 + lane;
        int32_t key = kEmpty;
        H val = H(0);
        if (s < size) { key = tk[s]; val = tv[s]; }
        const bool occ = key != kEmpty;
        const unsigned ball = __ballot_sync(gm, occ) & gm;
        if (occ) {
          const int64_t p = base + cnt + __popc(ball & lanemask_lt());
          a.otg[p] = key;
          a.ow[p] = (typename M::w_t)val;
          tk[s] = kEmpty;
          tv[s] = H(0);
        }
        cnt += __popc(ball);
      }
      if (lane == 0) { a.hend[c] = base + cnt; ctr[3] += cnt; }
    } else {
      if (threadIdx.x == 0) s_cnt = 0;
      __syncthreads();
      for (unsigned s0 = 0; s0 < size; s0 += G) {
        const unsigned s = s0 + threadIdx.x;
        int32_t key = kEmpty;
        H val = H(0);
        if (s < size) { key = tk[s]; val = tv[s]; }
        const bool occ = key != kEmpty;
        const unsigned ball = __ballot_sync(0xffffffffu, occ);
        unsigned long long wb = 0;
        if ((threadIdx.x & 31) == 0 && ball) wb = atomicAdd(&s_cnt, (unsigned long long)__popc(ball));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (occ) {
          const int64_t p = base + (int64_t)wb + __popc(ball & lanemask_lt());
          a.otg[p] = key;
          a.ow[p] = (typename M::w_t)val;
          tk[s] = kEmpty;
          tv[s] = H(0);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) { a.hend[c] = base + (int64_t)s_cnt; ctr[3] += s_cnt; }
      __syncthreads();
    }
  }
  block_add_counters<4>(a.ctrl->mg_stat[a.bucket], ctr);
}

template <class M, int G, int LOG>
static void launch_merge(Ctx& c, const MergeArgs<M>& a, const int32_t* list, int64_t count, int max_blocks) {
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  constexpr size_t smem = (size_t)GPB * (1 << LOG) * (sizeof(int32_t) + sizeof(typename M::h_t));
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(merge_kernel<M, G, LOG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  merge_kernel<M, G, LOG><<<grid_for(count, GPB, max_blocks), kBlock, smem, c.s>>>(a, list, count);
  c.launches++;
}

template <class M>
void merge_bucket(Ctx& c, int bucket, const MergeArgs<M>& args, const int32_t* list, int64_t count) {
  if (count <= 0) return;
  MergeArgs<M> a = args;
  a.bucket = bucket < kNumBuckets ? bucket : kNumBuckets - 1;
  const int cap = c.num_sms * 16;
  switch (bucket) {
    case 0: launch_merge<M, 4, 3>(c, a, list, count, cap); break;
    case 1: launch_merge<M, 8, 5>(c, a, list, count, cap); break;
    case 2: launch_merge<M, 32, 8>(c, a, list, count, cap); break;
    case 3: launch_merge<M, 32, 10>(c, a, list, count, cap); break;
    case 4: launch_merge<M, 256, 12>(c, a, list, count, cap); break;
    case 5: launch_merge<M, 256, 13>(c, a, list, count, cap); break;
    default: break;  // giant communities go through giant_merge
  }
}

// ---------------------------------------------------------------- compaction
__global__ void k_row_len(int64_t n, const int64_t* hbeg, const int64_t* hend, int64_t* len) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    len[r] = hend[r] - hbeg[r];
}
void row_lengths(Ctx& c, int64_t n, const int64_t* hbeg, const int64_t* hend, int64_t* len) {
  if (n <= 0) return;
  k_row_len<<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(n, hbeg, hend, len);
  c.launches++;
}

// A block copies the rows [r0, r0 + 256): the flat index space over their arcs is shared by all
// threads (owner row by binary search over the block's prefix sums), so one long row does not
// serialise on one warp.  Output positions are contiguous from doff[r0].
template <class W>
__global__ void __launch_bounds__(kBlock) k_compact(int64_t n, const int64_t* hbeg, const int64_t* hend,
                                                    const int64_t* doff, const int32_t* itg, const W* iw,
                                                    int32_t* otg, W* ow) {
  __shared__ int64_t excl[kBlock + 1];
  __shared__ int64_t sbeg[kBlock];
  for (int64_t r0 = (int64_t)blockIdx.x * kBlock; r0 < n; r0 += (int64_t)gridDim.x * kBlock) {
    const int64_t r = r0 + threadIdx.x;
    int64_t len = 0, b = 0;
    if (r < n) { b = hbeg[r]; len = hend[r] - b; }
    sbeg[threadIdx.x] = b;
    excl[threadIdx.x + 1] = len;
    if (threadIdx.x == 0) excl[0] = 0;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {
      int64_t v = threadIdx.x + 1 > (unsigned)o ? excl[threadIdx.x + 1 - o] : 0;
      __syncthreads();
      excl[threadIdx.x + 1] += v;
      __syncthreads();
    }
    const int64_t total = excl[kBlock];
    const int64_t dbase = doff[r0];
    for (int64_t f = threadIdx.x; f < total; f += kBlock) {
      int lo = 0, hi = kBlock - 1;  // last row with excl <= f
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (excl[mid] <= f) lo = mid; else hi = mid - 1;
      }
      const int64_t src = sbeg[lo] + (f - excl[lo]);
      otg[dbase + f] = itg[src];
      ow[dbase + f] = iw[src];
    }
    __syncthreads();
  }
}
template <class W>
void compact_rows(Ctx& c, int64_t n, const int64_t* hbeg, const int64_t* hend, const int64_t* doff, const int32_t* itg,
                  const W* iw, int32_t* otg, W* ow) {
  if (n <= 0) return;
  k_compact<W><<<grid_for(n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(n, hbeg, hend, doff, itg, iw, otg, ow);
  c.launches++;
}

// Bucketed compaction: one group of G lanes copies one holey row (rows listed by the community
// total-degree buckets of the merge, which bound the row lengths); giant rows go by chunks.
template <class W, int G>
__global__ void __launch_bounds__(kBlock) k_compact_group(const int32_t* list, int64_t count, const int64_t* hbeg,
                                                          const int64_t* hend, const int64_t* doff,
                                                          const int32_t* itg, const W* iw, int32_t* otg, W* ow) {
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t r = list[idx];
    const int64_t b = hbeg[r], len = hend[r] - b, d = doff[r];
    for (int64_t k = lane; k < len; k += G) {
      otg[d + k] = itg[b + k];
      ow[d + k] = iw[b + k];
    }
  }
}

template <class W>
void compact_bucketed(Ctx& c, const int32_t* cperm, const int64_t* cb, const int64_t* hbeg, const int64_t* hend,
                      const int64_t* doff, const int32_t* itg, const W* iw, int32_t* otg, W* ow, const GiantPlan& gp,
                      Ctrl* ctrl) {
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    const int64_t cnt = cb[b + 1] - cb[b];
    if (cnt <= 0) continue;
    const int32_t* l = cperm + cb[b];
    switch (b) {
      case 0: k_compact_group<W, 4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(l, cnt, hbeg, hend, doff, itg, iw, otg, ow); break;
      case 1: k_compact_group<W, 8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(l, cnt, hbeg, hend, doff, itg, iw, otg, ow); break;
      case 2:
      case 3: k_compact_group<W, 32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(l, cnt, hbeg, hend, doff, itg, iw, otg, ow); break;
      case 4:
      case 5: k_compact_group<W, 256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(l, cnt, hbeg, hend, doff, itg, iw, otg, ow); break;
      default: giant_compact<W>(c, l, cnt, hbeg, hend, doff, itg, iw, otg, ow, gp, ctrl); c.launches--; break;
    }
    c.launches++;
  }
}

template void compact_bucketed<int32_t>(Ctx&, const int32_t*, const int64_t*, const int64_t*, const int64_t*,
                                        const int64_t*, const int32_t*, const int32_t*, int32_t*, int32_t*,
                                        const GiantPlan&, Ctrl*);
template void compact_bucketed<float>(Ctx&, const int32_t*, const int64_t*, const int64_t*, const int64_t*,
                                      const int64_t*, const int32_t*, const float*, int32_t*, float*,
                                      const GiantPlan&, Ctrl*);

template void merge_bucket<IntMode>(Ctx&, int, const MergeArgs<IntMode>&, const int32_t*, int64_t);
template void merge_bucket<FpMode>(Ctx&, int, const MergeArgs<FpMode>&, const int32_t*, int64_t);
template void compact_rows<int32_t>(Ctx&, int64_t, const int64_t*, const int64_t*, const int64_t*, const int32_t*,
                                    const int32_t*, int32_t*, int32_t*);
template void compact_rows<float>(Ctx&, int64_t, const int64_t*, const int64_t*, const int64_t*, const int32_t*,
                                  const float*, int32_t*, float*);

}  // namespace lv
