// colour.cu -- Jones-Plassmann colouring for the deterministic (colour-synchronous) schedule.
//
// The paper cites ordering vertices by a graph colouring as one way to parallelise Louvain
// (Section 2).  Here: priority p(v) = hash3(seed, pass, v), u before v iff (p(u), u) > (p(v), v).
// A vertex is coloured once every higher-priority neighbour is, with the smallest colour none of
// them holds -- exactly greedy colouring in decreasing priority, whatever the round structure.
// Push form: cnt[v] = number of higher-priority neighbour arcs; a coloured vertex decrements the
// counters of its lower-priority neighbours and appends those reaching zero to the next ready
// list.  Rounds are launched in batches; a round with an empty ready list returns at once.
#include "internal.cuh"

namespace lv {

struct JpArgs {
  GraphView<int32_t> g;
  uint64_t seed;
  int32_t pass;
  int32_t* colour;
  int32_t* cnt;
  int32_t* lists[2];
  int64_t list_cap;             // capacity of each ready list
  unsigned long long* rcount;   // rcount[r] = size of the ready list of round r (zeroed up front)
  Ctrl* ctrl;                   // cnt[3] coloured total, cnt[4] max colour + 1, cnt[7] guard trips
  Segs seg;                     // batched run: priorities hash graph-local ids
};

template <int G>
__global__ void __launch_bounds__(kBlock) jp_count(JpArgs a, const int32_t* list, int64_t count) {
  __shared__ int32_t red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t v = list[idx];
    const uint64_t pv = hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, v));
    int32_t k = 0;
    for (int64_t e = a.g.rbeg[v] + lane; e < a.g.rend[v]; e += G) {
      const int32_t u = a.g.tg[e];
      if (u != v && higher(hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, u)), u, pv, v)) k++;
    }
    k = group_sum<G>(k, red);
    if (lane == 0) {
      a.cnt[v] = k;
      a.colour[v] = -1;
      if (k == 0) {
        const unsigned long long pos = atomicAdd(&a.rcount[0], 1ULL);
        if ((int64_t)pos < a.list_cap) a.lists[0][pos] = v;
        else atomicAdd(&a.ctrl->cnt[7], 1ULL);
      }
    }
  }
}

// One round: a warp per ready vertex; mex over windows of 1024 colours in a shared bitmap.
__global__ void __launch_bounds__(kBlock) jp_round(JpArgs a, int r) {
  __shared__ unsigned bm[kBlock / 32][32];
  __shared__ unsigned long long done_blk;
  __shared__ int32_t max_blk;
  const int32_t* in = a.lists[r & 1];
  int32_t* out = a.lists[(r + 1) & 1];
  unsigned long long count = *(volatile unsigned long long*)&a.rcount[r];
  if (count == 0) return;
  if ((int64_t)count > a.list_cap) count = (unsigned long long)a.list_cap;
  if (threadIdx.x == 0) { done_blk = 0; max_blk = 0; }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
  for (int64_t k = (int64_t)blockIdx.x * (kBlock / 32) + warp; k < (int64_t)count; k += nw) {
    const int32_t v = in[k];
    // guard: a ready vertex is uncoloured; anything else is recorded and skipped
    int32_t prev = 0;
    if (lane == 0) prev = a.colour[v];
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != -1) {
      if (lane == 0) atomicAdd(&a.ctrl->cnt[7], 1ULL);
      continue;
    }
    const uint64_t pv = hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, v));
    const int64_t beg = a.g.rbeg[v], end = a.g.rend[v];
    int32_t mex = -1;
    // colours of higher-priority neighbours are final; mex <= degree, so windows are bounded
    for (int32_t base = 0; base <= (int32_t)(end - beg); base += 1024) {
      bm[warp][lane] = 0u;
      __syncwarp();
      for (int64_t e = beg + lane; e < end; e += 32) {
        const int32_t u = a.g.tg[e];
        if (u == v || !higher(hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, u)), u, pv, v)) continue;
        const int32_t cu = a.colour[u] - base;
        if (cu >= 0 && cu < 1024) atomicOr(&bm[warp][cu >> 5], 1u << (cu & 31));
      }
      __syncwarp();
      const unsigned freeb = ~bm[warp][lane];
      const unsigned ball = __ballot_sync(0xffffffffu, freeb != 0u);
      __syncwarp();
      if (ball) {
        const int L = __ffs(ball) - 1;
        const unsigned fw = __shfl_sync(0xffffffffu, freeb, L);
        mex = base + 32 * L + (__ffs(fw) - 1);
        break;
      }
    }
    if (mex < 0) {  // unreachable: some colour <= degree is always free
      if (lane == 0) atomicOr(&a.ctrl->error, kErrRange);
      mex = 0;
    }
    if (lane == 0) {
      a.colour[v] = mex;
      atomicAdd(&done_blk, 1ULL);
      atomicMax(&max_blk, mex + 1);
    }
    __syncwarp();
    for (int64_t e = beg + lane; e < end; e += 32) {
      const int32_t u = a.g.tg[e];
      if (u == v || !higher(pv, v, hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, u)), u)) continue;
      if (atomicSub(&a.cnt[u], 1) == 1) {
        const unsigned long long pos = atomicAdd(&a.rcount[r + 1], 1ULL);
        if ((int64_t)pos < a.list_cap) out[pos] = u;
        else atomicAdd(&a.ctrl->cnt[7], 1ULL);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && done_blk) {
    atomicAdd(&a.ctrl->cnt[3], done_blk);
    atomicMax(reinterpret_cast<unsigned long long*>(&a.ctrl->cnt[4]), (unsigned long long)max_blk);
  }
}

__global__ void k_jp_reset(Ctrl* c) {
  c->cnt[3] = 0;
  c->cnt[4] = 0;
  c->cnt[7] = 0;
}

int32_t jp_colour(Ctx& c, const GraphView<int32_t>& g, const int32_t* perm, const int64_t* hb, uint64_t seed,
                  int32_t pass, int32_t* colour, const JpBuffers& jb, Ctrl* ctrl, unsigned long long* h_pinned,
                  cudaError_t* err, Segs seg) {
  *err = cudaSuccess;
  const int64_t listed = hb[kNumBuckets] - hb[0];
  // Each round colours at least one vertex while any is left, so `listed` rounds always suffice.
  const int batch = 8;
  const int64_t max_rounds = listed + batch;
  // isolated vertices (left out of the bucket lists) get colour 0
  fill_i32(c, colour, 0, g.n);
  cudaMemsetAsync(jb.rcount, 0, (size_t)(max_rounds + 2) * sizeof(unsigned long long), c.s);
  k_jp_reset<<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
  JpArgs a;
  a.g = g; a.seed = seed; a.pass = pass; a.colour = colour; a.cnt = jb.cnt;
  a.lists[0] = jb.list0; a.lists[1] = jb.list1; a.list_cap = jb.list_cap; a.rcount = jb.rcount; a.ctrl = ctrl;
  a.seg = seg;
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    int64_t cnt = hb[b + 1] - hb[b];
    if (cnt <= 0) continue;
    const int32_t* l = perm + hb[b];
    switch (b) {
      case 0: jp_count<4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      case 1: jp_count<8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      case 2:
      case 3: jp_count<32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      default: jp_count<256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
    }
    c.launches++;
  }
  if ((*err = cudaGetLastError()) != cudaSuccess) return -1;
  int64_t r = 0;
  h_pinned[3] = 0;
  while (r < max_rounds) {
    for (int k = 0; k < batch && r < max_rounds; k++, r++) {
      jp_round<<<c.num_sms * 8, kBlock, 0, c.s>>>(a, (int)r);
      c.launches++;
    }
    if ((*err = cudaGetLastError()) != cudaSuccess) return -1;
    cudaMemcpyAsync(h_pinned, &ctrl->cnt[0], 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.s);
    *err = cudaStreamSynchronize(c.s);
    if (*err != cudaSuccess) return -1;
    if ((int64_t)h_pinned[3] >= listed || h_pinned[7]) break;
  }
  if ((int64_t)h_pinned[3] != listed || h_pinned[7]) {
    h_pinned[5] = (unsigned long long)listed;
    h_pinned[6] = (unsigned long long)r;
    return -1;
  }
  int32_t ncol = (int32_t)h_pinned[4];
  return ncol > 0 ? ncol : 1;
}

}  // namespace lv
