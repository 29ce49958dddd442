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
  Ctrl* ctrl;  // cnt[0..2] rotating ready counts, cnt[3] coloured total, cnt[4] max colour + 1
};

template <int G>
__global__ void __launch_bounds__(kBlock) jp_count(JpArgs a, const int32_t* list, int64_t count) {
  __shared__ int32_t red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t v = list[idx];
    const uint64_t pv = hash3(a.seed, (uint64_t)a.pass, (uint64_t)v);
    int32_t k = 0;
    for (int64_t e = a.g.rbeg[v] + lane; e < a.g.rend[v]; e += G) {
      const int32_t u = a.g.tg[e];
      if (u != v && higher(hash3(a.seed, (uint64_t)a.pass, (uint64_t)u), u, pv, v)) k++;
    }
    k = group_sum<G>(k, red);
    if (lane == 0) {
      a.cnt[v] = k;
      a.colour[v] = -1;
      if (k == 0) {
        unsigned long long pos = atomicAdd(&a.ctrl->cnt[0], 1ULL);
        a.lists[0][pos] = v;
      }
    }
  }
}

// One round: a warp per ready vertex; mex over windows of 1024 colours in a shared bitmap.
__global__ void __launch_bounds__(kBlock) jp_round(JpArgs a, int r) {
  __shared__ unsigned bm[kBlock / 32][32];
  __shared__ unsigned long long done_blk;
  __shared__ int32_t max_blk;
  const int cur = r % 3, nxt = (r + 1) % 3, clr = (r + 2) % 3;
  const int32_t* in = a.lists[r & 1];
  int32_t* out = a.lists[(r + 1) & 1];
  const unsigned long long count = *(volatile unsigned long long*)&a.ctrl->cnt[cur];
  if (count == 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->cnt[clr] = 0;  // untouched by this round
  if (threadIdx.x == 0) { done_blk = 0; max_blk = 0; }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
  for (int64_t k = (int64_t)blockIdx.x * (kBlock / 32) + warp; k < (int64_t)count; k += nw) {
    const int32_t v = in[k];
    const uint64_t pv = hash3(a.seed, (uint64_t)a.pass, (uint64_t)v);
    const int64_t beg = a.g.rbeg[v], end = a.g.rend[v];
    int32_t mex = -1;
    // colours of higher-priority neighbours are final; mex <= degree, so windows are bounded
    for (int32_t base = 0; base <= (int32_t)(end - beg); base += 1024) {
      bm[warp][lane] = 0u;
      __syncwarp();
      for (int64_t e = beg + lane; e < end; e += 32) {
        const int32_t u = a.g.tg[e];
        if (u == v || !higher(hash3(a.seed, (uint64_t)a.pass, (uint64_t)u), u, pv, v)) continue;
        const int32_t cu = a.colour[u] - base;
        if (cu >= 0 && cu < 1024) atomicOr(&bm[warp][cu >> 5], 1u << (cu & 31));
      }
      __syncwarp();
      const unsigned freeb = ~bm[warp][lane];
      const unsigned ball = __ballot_sync(0xffffffffu, freeb != 0u);
      if (ball) {
        const int L = __ffs(ball) - 1;
        const unsigned fw = __shfl_sync(0xffffffffu, freeb, L);
        mex = base + 32 * L + (__ffs(fw) - 1);
        break;
      }
      __syncwarp();
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
      if (u == v || !higher(pv, v, hash3(a.seed, (uint64_t)a.pass, (uint64_t)u), u)) continue;
      if (atomicSub(&a.cnt[u], 1) == 1) {
        unsigned long long pos = atomicAdd(&a.ctrl->cnt[nxt], 1ULL);
        out[pos] = u;
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
  for (int k = 0; k < 5; k++) c->cnt[k] = 0;
}

int32_t jp_colour(Ctx& c, const GraphView<int32_t>& g, const int32_t* perm, const int64_t* hb, uint64_t seed,
                  int32_t pass, int32_t* colour, const JpBuffers& jb, Ctrl* ctrl, unsigned long long* h_pinned,
                  cudaError_t* err) {
  *err = cudaSuccess;
  // isolated vertices (left out of the bucket lists) get colour 0
  fill_i32(c, colour, 0, g.n);
  k_jp_reset<<<1, 1, 0, c.s>>>(ctrl);
  c.launches++;
  JpArgs a;
  a.g = g; a.seed = seed; a.pass = pass; a.colour = colour; a.cnt = jb.cnt;
  a.lists[0] = jb.list0; a.lists[1] = jb.list1; a.ctrl = ctrl;
  const int cap = c.num_sms * 16;
  for (int b = 0; b < kNumBuckets; b++) {
    int64_t cnt = hb[b + 1] - hb[b];
    if (cnt <= 0) continue;
    const int32_t* l = perm + hb[b];
    switch (b) {
      case 0: jp_count<4><<<grid_for(cnt, kBlock / 4, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      case 1: jp_count<8><<<grid_for(cnt, kBlock / 8, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      case 2: jp_count<32><<<grid_for(cnt, kBlock / 32, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
      default: jp_count<256><<<grid_for(cnt, 1, cap), kBlock, 0, c.s>>>(a, l, cnt); break;
    }
    c.launches++;
  }
  const int64_t listed = hb[kNumBuckets] - hb[0];
  // Each round colours at least one vertex while any is left, so `listed` rounds always suffice.
  const int batch = 8;
  int64_t r = 0;
  while (r < listed + batch) {
    for (int k = 0; k < batch; k++, r++) {
      jp_round<<<c.num_sms * 8, kBlock, 0, c.s>>>(a, (int)r);
      c.launches++;
    }
    cudaMemcpyAsync(h_pinned, &ctrl->cnt[0], 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.s);
    *err = cudaStreamSynchronize(c.s);
    if (*err != cudaSuccess) return -1;
    if ((int64_t)h_pinned[3] >= listed) break;
  }
  if ((int64_t)h_pinned[3] != listed) return -1;
  int32_t ncol = (int32_t)h_pinned[4];
  return ncol > 0 ? ncol : 1;
}

}  // namespace lv
