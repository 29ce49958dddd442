// colour.cu -- Jones-Plassmann colouring for the deterministic (colour-synchronous) schedule.
//
// The paper cites ordering vertices by a graph colouring as one way to parallelise Louvain
// (Section 2).  Here: priority p(v) = hash3(seed, pass, v), u before v iff (p(u), u) > (p(v), v).
// A vertex is coloured once every higher-priority neighbour is, with the smallest colour none of
// them holds -- exactly greedy colouring in decreasing priority, whatever the round structure.
//
// Push form.  cnt[v] = number of higher-priority neighbour arcs; used[v] = a bitmap of the colours
// its coloured higher-priority neighbours hold, ceil((deg + 1) / 32) words (its colour is at most
// its degree, so larger colours need no bit).  A round takes the ready list (cnt = 0): each vertex
// reads the first free bit of its bitmap as its colour, then pushes to every lower-priority
// neighbour -- sets the colour's bit and decrements the counter, appending the neighbours that
// reach zero to the next ready list.  The push of a vertex with more than kBigDeg arcs (in a busy
// round, kBigDegBusy) is spread over the whole grid by a second kernel, so a chain of hubs (a dense
// core needs one round per member) costs microseconds per round, not a warp's walk over 10^5
// arcs.  The round index lives on the device, so a batch of rounds is captured once as a CUDA
// graph and replayed until every vertex is coloured; a round with an empty ready list returns at
// once.
#include "internal.cuh"

namespace lv {

constexpr int64_t kBigDeg = 32;       // pushes of longer rows are spread over the grid in chunks,
constexpr int64_t kBigDegBusy = 256;  // in a round with a ready vertex per warp: of rows over this
constexpr int64_t kPushChunk = kBlock;  // arcs per chunk (one per thread of a block)
constexpr int kRoundsPerGraph = 16;

struct JpArgs {
  GraphView<int32_t> g;
  uint64_t seed;
  int32_t pass;
  int32_t* colour;
  int32_t* cnt;
  int32_t* lists[2];
  int64_t list_cap;             // capacity of each ready list (and of the big list)
  unsigned long long* rcount;   // rcount[r] = size of the ready list of round r (zeroed up front)
  unsigned long long* bcount;   // bcount[r] = vertices of round r whose push is spread (zeroed up front)
  int32_t* big;                 // those vertices
  int64_t* big_cb;              // first push chunk of each of them
  int32_t* cown;                // [chunk_cap] big-list entry of each push chunk of the round
  int64_t chunk_cap;
  unsigned long long* ccount;   // ccount[r] = push chunks of round r (zeroed up front)
  const int64_t* boff;          // [n + 1] first bitmap word of each vertex
  unsigned* used;               // the bitmaps (zeroed up front)
  unsigned long long* round;    // current round (device)
  Ctrl* ctrl;                   // cnt[3] coloured total, cnt[4] max colour + 1, cnt[7] guard trips
  Segs seg;                     // batched run: priorities hash graph-local ids
};

__device__ __forceinline__ uint64_t prio(const JpArgs& a, int32_t v) {
  return hash3(a.seed, (uint64_t)a.pass, local_id(a.seg, v));
}

// Bitmap words of every vertex: ceil((deg + 1) / 32).
__global__ void jp_words(GraphView<int32_t> g, int64_t* words) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += (int64_t)gridDim.x * blockDim.x)
    words[v] = (g.rend[v] - g.rbeg[v] + 1 + 31) / 32;
}

template <int G>
__global__ void __launch_bounds__(kBlock) jp_count(JpArgs a, const int32_t* list, int64_t count) {
  __shared__ int32_t red[32];
  constexpr int GPB = G <= 32 ? kBlock / G : 1;
  const int gib = G <= 32 ? (int)(threadIdx.x / G) : 0;
  const unsigned lane = Grp<G>::lane();
  for (int64_t idx = (int64_t)blockIdx.x * GPB + gib; idx < count; idx += (int64_t)gridDim.x * GPB) {
    const int32_t v = list[idx];
    const uint64_t pv = prio(a, v);
    int32_t k = 0;
    for (int64_t e = a.g.rbeg[v] + lane; e < a.g.rend[v]; e += G) {
      const int32_t u = a.g.tg[e];
      if (u != v && higher(prio(a, u), u, pv, v)) k++;
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

// Push of the colour c of v along arc e: the neighbour u of lower priority records c and, when its
// last higher-priority neighbour is done, joins the next ready list.  (The uncoloured neighbours of
// a ready vertex are exactly those of lower priority, but reading u's colour to tell them apart
// measured slower than hashing u's priority.)
__device__ __forceinline__ void jp_push(const JpArgs& a, int32_t v, uint64_t pv, int32_t c, int32_t u, int32_t* out,
                                        unsigned long long* next_count) {
  if (u == v || !higher(pv, v, prio(a, u), u)) return;
  const int64_t w0 = a.boff[u], nw = a.boff[u + 1] - w0;
  if ((int64_t)(c >> 5) < nw) atomicOr(&a.used[w0 + (c >> 5)], 1u << (c & 31));
  if (atomicSub(&a.cnt[u], 1) == 1) {
    const unsigned long long pos = atomicAdd(next_count, 1ULL);
    if ((int64_t)pos < a.list_cap) out[pos] = u;
    else atomicAdd(&a.ctrl->cnt[7], 1ULL);
  }
}

// One round, part 1: a warp per ready vertex takes the first free colour of its bitmap, then
// pushes along its arcs (rows longer than kBigDeg go to the big list instead).  Every thread of
// the block calls it.
__device__ __forceinline__ void jp_round_body(const JpArgs& a, unsigned long long r, unsigned long long* done_blk,
                                              int32_t* max_blk) {
  const int32_t* in = a.lists[r & 1];
  int32_t* out = a.lists[(r + 1) & 1];
  unsigned long long count = *(volatile unsigned long long*)&a.rcount[r];
  if (count == 0) return;
  if ((int64_t)count > a.list_cap) count = (unsigned long long)a.list_cap;
  if (threadIdx.x == 0) { *done_blk = 0; *max_blk = 0; }
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicMax(&a.ctrl->cnt[6], r + 1);  // rounds with work
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (kBlock / 32);
  // a round with few ready vertices spreads every push of more than a warp's width over the grid
  // (its time is the longest push); a busy round keeps rows up to kBigDegBusy on their warp, where
  // one 256-arc chunk per block would leave most of a block idle on a 40-arc row
  const int64_t big_deg = (int64_t)count >= nw ? kBigDegBusy : kBigDeg;
  for (int64_t k = (int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); k < (int64_t)count; k += nw) {
    const int32_t v = in[k];
    // guard: a ready vertex is uncoloured; anything else is recorded and skipped
    const int32_t prev = a.colour[v];
    if (prev != -1) {
      if (lane == 0) atomicAdd(&a.ctrl->cnt[7], 1ULL);
      continue;
    }
    // first free bit; it exists: the colours recorded number at most the degree
    const int64_t w0 = a.boff[v], words = a.boff[v + 1] - w0;
    int32_t col = -1;
    for (int64_t wb = 0; wb < words; wb += 32) {
      const unsigned freeb = wb + lane < words ? ~a.used[w0 + wb + lane] : 0u;
      const unsigned ball = __ballot_sync(0xffffffffu, freeb != 0u);
      if (ball) {
        const int L = __ffs(ball) - 1;
        const unsigned fw = __shfl_sync(0xffffffffu, freeb, L);
        col = (int32_t)(32 * (wb + L)) + (__ffs(fw) - 1);
        break;
      }
    }
    if (col < 0) {  // unreachable
      if (lane == 0) atomicOr(&a.ctrl->error, kErrRange);
      col = 0;
    }
    const int64_t beg = a.g.rbeg[v], end = a.g.rend[v];
    if (lane == 0) {
      a.colour[v] = col;
      atomicAdd(done_blk, 1ULL);
      atomicMax(max_blk, col + 1);
    }
    if (end - beg > big_deg) {
      // spread the push: the vertex joins the big list and reserves its chunks of kPushChunk arcs
      const int64_t nch = (end - beg + kPushChunk - 1) / kPushChunk;
      unsigned long long pos = 0, cb = 0;
      if (lane == 0) {
        pos = atomicAdd(&a.bcount[r], 1ULL);
        cb = atomicAdd(&a.ccount[r], (unsigned long long)nch);
        if ((int64_t)pos < a.list_cap && (int64_t)(cb + nch) <= a.chunk_cap) {
          a.big[pos] = v;
          a.big_cb[pos] = (int64_t)cb;
        } else {
          atomicAdd(&a.ctrl->cnt[7], 1ULL);
        }
      }
      pos = __shfl_sync(0xffffffffu, pos, 0);
      cb = __shfl_sync(0xffffffffu, cb, 0);
      if ((int64_t)pos < a.list_cap && (int64_t)(cb + nch) <= a.chunk_cap)
        for (int64_t t = lane; t < nch; t += 32) a.cown[cb + t] = (int32_t)pos;
      continue;
    }
    const uint64_t pv = prio(a, v);
    for (int64_t e = beg + lane; e < end; e += 32) jp_push(a, v, pv, col, a.g.tg[e], out, &a.rcount[r + 1]);
  }
  __syncthreads();
  if (threadIdx.x == 0 && *done_blk) {
    atomicAdd(&a.ctrl->cnt[3], *done_blk);
    atomicMax(reinterpret_cast<unsigned long long*>(&a.ctrl->cnt[4]), (unsigned long long)*max_blk);
  }
}

__global__ void __launch_bounds__(kBlock) jp_round(JpArgs a) {
  __shared__ unsigned long long done_blk;
  __shared__ int32_t max_blk;
  jp_round_body(a, *(volatile unsigned long long*)a.round, &done_blk, &max_blk);
}

// One round, part 2: the pushes of the big vertices, one block per chunk of kPushChunk arcs.
__device__ __forceinline__ void jp_big_body(const JpArgs& a, unsigned long long r) {
  unsigned long long nc = *(volatile unsigned long long*)&a.ccount[r];
  if (nc == 0) return;
  if ((int64_t)nc > a.chunk_cap) nc = (unsigned long long)a.chunk_cap;
  int32_t* out = a.lists[(r + 1) & 1];
  unsigned long long nb = *(volatile unsigned long long*)&a.bcount[r];
  if ((int64_t)nb > a.list_cap) nb = (unsigned long long)a.list_cap;
  for (unsigned long long q = blockIdx.x; q < nc; q += gridDim.x) {
    const int32_t pos = a.cown[q];
    if (pos < 0 || (unsigned long long)pos >= nb) continue;  // defensive: every chunk is owned
    const int32_t v = a.big[pos];
    const int64_t e = a.g.rbeg[v] + ((int64_t)q - a.big_cb[pos]) * kPushChunk + threadIdx.x;
    if (e < a.g.rend[v]) jp_push(a, v, prio(a, v), a.colour[v], a.g.tg[e], out, &a.rcount[r + 1]);
  }
}

__global__ void __launch_bounds__(kBlock) jp_round_big(JpArgs a) { jp_big_body(a, *(volatile unsigned long long*)a.round); }

// ---------------------------------------------------------------- persistent form
// All rounds in one cooperative launch (every block resident): two grid barriers per round
// instead of three kernel launches.  The barrier spins with a bound; a block that gives up sets
// ctrl->error (kErrTimeout) and every block leaves at its next barrier, so the kernel always ends.
constexpr long long kBarrierSpins = 1LL << 22;  // x ~64 ns sleep: about 0.3 s

struct GridBar {
  unsigned* count;
  unsigned* gen;
};

// Returns false (on every block, at this or the next barrier) once any block has timed out.
__device__ __forceinline__ bool grid_barrier(const GridBar& b, Ctrl* ctrl, long long max_spins) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = *(volatile unsigned*)b.gen;
    __threadfence();
    if (atomicAdd(b.count, 1u) == gridDim.x - 1) {
      *(volatile unsigned*)b.count = 0u;
      __threadfence();
      atomicAdd(b.gen, 1u);
    } else {
      long long spins = 0;
      while (*(volatile unsigned*)b.gen == g) {
        if (++spins > max_spins || (*(volatile int32_t*)&ctrl->error & kErrTimeout)) {
          atomicOr(&ctrl->error, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int32_t*)&ctrl->error & kErrTimeout) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__global__ void __launch_bounds__(kBlock) jp_persistent(JpArgs a, GridBar bar, unsigned long long max_rounds,
                                                       long long max_spins) {
  __shared__ unsigned long long done_blk;
  __shared__ int32_t max_blk;
  for (unsigned long long r = 0; r < max_rounds; r++) {
    if (*(volatile unsigned long long*)&a.rcount[r] == 0) break;  // nothing ready: coloured (or stuck)
    jp_round_body(a, r, &done_blk, &max_blk);
    if (!grid_barrier(bar, a.ctrl, max_spins)) return;
    jp_big_body(a, r);
    if (!grid_barrier(bar, a.ctrl, max_spins)) return;
  }
}

// Advances the round once both parts are done.
__global__ void jp_next(unsigned long long* round) { *round += 1; }

__global__ void k_jp_reset(Ctrl* c, unsigned long long* round) {
  c->cnt[3] = 0;
  c->cnt[4] = 0;
  c->cnt[6] = 0;
  c->cnt[7] = 0;
  *round = 0;
}

int32_t jp_colour(Ctx& c, const GraphView<int32_t>& g, const int32_t* perm, const int64_t* hb, uint64_t seed,
                  int32_t pass, int32_t* colour, const JpBuffers& jb, Ctrl* ctrl, unsigned long long* h_pinned,
                  cudaError_t* err, Segs seg, int64_t* rounds_out) {
  *err = cudaSuccess;
  const int64_t listed = hb[kNumBuckets] - hb[0];
  // Each round colours at least one vertex while any is left, so `listed` rounds always suffice.
  const int64_t max_rounds = listed + kRoundsPerGraph;
  // isolated vertices (left out of the bucket lists) get colour 0
  fill_i32(c, colour, 0, g.n);
  // the last replay may run up to kRoundsPerGraph - 1 rounds past max_rounds (they find empty lists)
  const size_t nrc = (size_t)(max_rounds + kRoundsPerGraph + 2);
  cudaMemsetAsync(jb.rcount, 0, nrc * sizeof(unsigned long long), c.s);
  cudaMemsetAsync(jb.bcount, 0, nrc * sizeof(unsigned long long), c.s);
  cudaMemsetAsync(jb.ccount, 0, nrc * sizeof(unsigned long long), c.s);
  // bitmap offsets (scan of the word counts) and zeroed bitmaps
  if (g.n > 0) {
    jp_words<<<grid_for(g.n, kBlock, c.num_sms * 8), kBlock, 0, c.s>>>(g, jb.boff);
    c.launches++;
  }
  scan_exclusive_i64(c, jb.boff, jb.boff, g.n, jb.tile_tmp);
  cudaMemsetAsync(jb.used, 0, (size_t)jb.used_cap * sizeof(unsigned), c.s);
  k_jp_reset<<<1, 1, 0, c.s>>>(ctrl, jb.round);
  c.launches++;
  JpArgs a;
  a.g = g; a.seed = seed; a.pass = pass; a.colour = colour; a.cnt = jb.cnt;
  a.lists[0] = jb.list0; a.lists[1] = jb.list1; a.list_cap = jb.list_cap; a.rcount = jb.rcount;
  a.bcount = jb.bcount; a.big = jb.big; a.big_cb = jb.big_cb; a.cown = jb.cown; a.chunk_cap = jb.chunk_cap;
  a.ccount = jb.ccount; a.boff = jb.boff; a.used = jb.used; a.round = jb.round; a.ctrl = ctrl;
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
  // Preferred: every round in one cooperative launch (grid barriers between the parts)
  {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jp_persistent, kBlock, 0) == cudaSuccess && per_sm > 0) {
      GridBar bar{reinterpret_cast<unsigned*>(jb.round + 1), reinterpret_cast<unsigned*>(jb.round + 2)};
      cudaMemsetAsync(jb.round + 1, 0, 2 * sizeof(unsigned long long), c.s);
      unsigned long long mr = (unsigned long long)max_rounds;
      long long spins = c.wait_spins > 0 ? c.wait_spins : kBarrierSpins;
      void* args[] = {(void*)&a, (void*)&bar, (void*)&mr, (void*)&spins};
      const int blocks = c.num_sms * (per_sm < 2 ? per_sm : 2);
      if (cudaLaunchCooperativeKernel((const void*)jp_persistent, blocks, kBlock, args, 0, c.s) == cudaSuccess) {
        c.launches++;
        cudaMemcpyAsync(h_pinned, &ctrl->cnt[0], 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.s);
        if ((*err = cudaStreamSynchronize(c.s)) != cudaSuccess) return -1;
        if ((int64_t)h_pinned[3] != listed || h_pinned[7]) {
          h_pinned[5] = (unsigned long long)listed;
          h_pinned[6] = (unsigned long long)max_rounds;
          return -1;
        }
        if (rounds_out) *rounds_out = (int64_t)h_pinned[6];
        const int32_t ncol = (int32_t)h_pinned[4];
        return ncol > 0 ? ncol : 1;
      }
      cudaGetLastError();  // not launchable cooperatively here: replayed rounds below
    } else {
      cudaGetLastError();
    }
  }
  // kRoundsPerGraph rounds (3 kernels each) captured once on a private stream, replayed on c.s
  cudaGraphExec_t exec = nullptr;
  {
    cudaStream_t cs = nullptr;
    if ((*err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return -1;
    cudaGraph_t graph = nullptr;
    *err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (*err == cudaSuccess) {
      for (int k = 0; k < kRoundsPerGraph; k++) {
        jp_round<<<c.num_sms * 8, kBlock, 0, cs>>>(a);
        jp_round_big<<<c.num_sms * 8, kBlock, 0, cs>>>(a);
        jp_next<<<1, 1, 0, cs>>>(jb.round);
      }
      *err = cudaStreamEndCapture(cs, &graph);
    }
    if (*err == cudaSuccess) *err = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (*err != cudaSuccess) return -1;
  }
  int64_t r = 0;
  h_pinned[3] = 0;
  while (r < max_rounds) {
    cudaGraphLaunch(exec, c.s);
    r += kRoundsPerGraph;
    c.launches += 3 * kRoundsPerGraph;
    cudaMemcpyAsync(h_pinned, &ctrl->cnt[0], 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.s);
    *err = cudaStreamSynchronize(c.s);
    if (*err != cudaSuccess) break;
    if ((int64_t)h_pinned[3] >= listed || h_pinned[7]) break;
  }
  cudaGraphExecDestroy(exec);
  if (*err != cudaSuccess) return -1;
  if ((int64_t)h_pinned[3] != listed || h_pinned[7]) {
    h_pinned[5] = (unsigned long long)listed;
    h_pinned[6] = (unsigned long long)r;
    return -1;
  }
  if (rounds_out) *rounds_out = (int64_t)h_pinned[6];
  int32_t ncol = (int32_t)h_pinned[4];
  return ncol > 0 ? ncol : 1;
}

}  // namespace lv
