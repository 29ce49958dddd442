// internal.cuh -- host-side launchers shared by the translation units of liblouvain.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lv {

// Launch context: the stream, a kernel-launch counter, the SM count.
struct Ctx {
  cudaStream_t s = nullptr;
  int64_t launches = 0;
  int num_sms = 152;
  int lm_blocks_per_sm = 16;  // grid cap of the local-moving kernels (blocks per SM)
  int64_t giant_min = 4096;   // rows longer than this take the giant path (2048..4096)
  long long wait_spins = 0;   // polls of a bounded device wait before it gives up (0 = built-in)
  int table_factor = 2;       // hash-table slots per key of a table's distinct-key bound (1, 2, 4)
  int fast_sync = -1;         // fast mode's schedule for this call, fixed by its first local-moving
                              // phase: -1 undecided, 0 asynchronous waves, 1 colour-synchronous
};

inline int grid_for(int64_t work_items, int items_per_block, int cap) {
  int64_t b = (work_items + items_per_block - 1) / items_per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// A graph as (row begin, row end) descriptors: a dense CSR passes rbeg = offsets,
// rend = offsets + 1; a holey CSR passes its begin and end arrays.
template <class W>
struct GraphView {
  int64_t n = 0;
  const int64_t* rbeg = nullptr;
  const int64_t* rend = nullptr;
  const int32_t* tg = nullptr;
  const W* w = nullptr;
};

// Device-resident ranges of a captured local-moving iteration: one record of kStepWords int64 per
// class step, written by the host before the iteration graph is launched, so one executable graph
// serves every pass over the same arrays (the kernels read their vertex ranges here):
//   [2b], [2b + 1]   start and count of degree bucket b < kNumBuckets - 1 in the perm list;
//   [kStepGiant]     offset of the class-ordered giant list, then the giant range k0, k1 (plan indices);
//   [kStepApply]     start and count of the deterministic Sigma apply.
constexpr int kStepWords = 20;
constexpr int kStepGiant = 12;
constexpr int kStepApply = 16;

// ---------------------------------------------------------------- prims.cu
// Exclusive scan of in[0, n) into out[0, n) and out[n] = total; tile_tmp needs
// scan_tmp_elems(n) int64 entries.  in == out allowed for int64 input.
int64_t scan_tmp_elems(int64_t n);
void scan_exclusive_i64(Ctx& c, const int64_t* in, int64_t* out, int64_t n, int64_t* tile_tmp);
void scan_exclusive_i32(Ctx& c, const int32_t* in, int64_t* out, int64_t n, int64_t* tile_tmp);

void fill_i32(Ctx& c, int32_t* p, int32_t v, int64_t n);
void iota_i32(Ctx& c, int32_t* p, int64_t n);

// Sort key of bucket_sort: kind 0 degree bucket; 1 colour[i] * kNumBuckets + bucket; 2 degree bucket
// of deg64[i]; 3 (hash3(seed, pass, i) % classes) * kNumBuckets + bucket.
struct KeyDesc {
  int kind = 0;
  int classes = 1;
  int pass = 0;
  uint64_t seed = 0;
  Segs seg;  // kind 3 hashes the graph-local id
  int giant_class = -1;  // kind 3: >= 0 puts every giant row in this class
  int64_t giant_min = 4096;  // rows longer than this are giant (set by bucket_sort from the Ctx)
  int table_factor = 2;      // giant-table slots per key bound (set by bucket_sort from the Ctx)
};

// Counting sort of vertex ids by key.  key_kind 0: degree bucket of (rend - rbeg); 1: colour *
// kNumBuckets + degree bucket; 2: degree bucket of deg64[i].  Vertices with a negative key are
// left out.  hist must hold nkeys + 1 int64; cursor nkeys int32.  Writes perm and offsets[nkeys+1]
// (device).
// max_deg (device, optional) receives the largest row length / deg64 value seen (atomicMax);
// giant_slots (device, optional) the summed table size of the giant-bucket items, each
// 2^tbl_log2(min(deg, n_bound), 6, 40).
void bucket_sort(Ctx& c, KeyDesc key_kind, int64_t n, const int64_t* rbeg, const int64_t* rend, const int32_t* colour,
                 const int64_t* deg64, int64_t nkeys, int32_t* perm, int64_t* offsets, int32_t* cursor,
                 int64_t* tile_tmp, unsigned long long* max_deg, unsigned long long* giant_slots = nullptr,
                 int64_t n_bound = 0);

// Renumbering (rank among occupied ids): occ[0, n) zeroed then marked from ids[0, m).
void mark_occupied(Ctx& c, const int32_t* ids, int64_t m, int32_t* occ, int64_t n);
void relabel(Ctx& c, int32_t* ids, int64_t m, const int64_t* newid);
void dendrogram_lookup(Ctx& c, int32_t* C, int64_t n0, const int32_t* Cp);
// K_next[newid[c]] = Sig[c] for occupied c.
template <class A>
void gather_totals(Ctx& c, const A* sig, const int32_t* occ, const int64_t* newid, int64_t n_old, A* k_next);
// Max of an int64 array into *out (device), out zeroed by the caller.
void max_i64(Ctx& c, const int64_t* p, int64_t n, unsigned long long* out);

// ---------------------------------------------------------------- move.cu
template <class M>
struct PassState {
  typename M::a_t* K;
  typename M::a_t* Sig;
  int32_t* Cp;
  uint8_t* flags;
  int32_t* csize;
  int32_t* mv_from;
  int32_t* mv_to;
  Ctrl* ctrl;
  GraphCtl* gc = nullptr;      // batched run: per-graph 2m, sums, convergence (null: one graph)
  const int32_t* vg = nullptr; // batched run: graph of each vertex
};

// ctrl->hub_arcs / all_arcs = arcs in rows over 512 arcs / all arcs of g (zeroed first).
template <class W>
void hub_share(Ctx& c, const GraphView<W>& g, Ctrl* ctrl);

// Per-pass vertex state: Cp = id, flags = 1, csize = 1, mv_to = -1; Sig = K if from_k else 0 with K = 0.
template <class M>
void vertex_init(Ctx& c, const PassState<M>& st, int64_t n, bool from_k);
// K[i] = Sig[i] = row weight sums for the vertices in the degree-bucketed lists; also K0.
template <class M>
void row_sums(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* perm, const int64_t* h_bucket_offs,
              typename M::a_t* K, typename M::a_t* Sig, typename M::a_t* K0);
// 2m = sum of K into ctrl.
template <class M>
void total_weight(Ctx& c, const typename M::a_t* K, int64_t n, Ctrl* ctrl);
// Reset the iteration state of a local-moving phase.
void move_setup(Ctx& c, Ctrl* ctrl, double tau, int max_iterations);


// One bucket's decide (+ apply in fast mode) over list[0, count).
// With `rng` (a step record's {start, count} of this bucket) the kernel reads its range there, list
// is the base it is offset from and count is an upper bound of the range that sizes the grid
// (blocks past the range return at once).
template <class M>
void move_bucket(Ctx& c, int bucket, const GraphView<typename M::w_t>& g, const PassState<M>& st,
                 const int32_t* list, int64_t count, bool fast, bool pruning, const int64_t* rng = nullptr);
// Shared-memory opt-ins of the local-move kernels (call before capturing launches into a graph).
void move_prepare();
// Deterministic mode: Sigma updates of the moves decided in list[0, count).
template <class M>
void move_apply(Ctx& c, const PassState<M>& st, const int32_t* list, int64_t count, const int64_t* rng = nullptr);
template <class M>
void move_finish(Ctx& c, Ctrl* ctrl);

// ---------------------------------------------------------------- colour.cu
struct JpBuffers {
  int32_t* cnt;                 // [n] uncoloured higher-priority neighbour arcs
  int32_t* list0;               // [list_cap] ready lists
  int32_t* list1;
  int64_t list_cap;
  unsigned long long* rcount;   // [n + 64] per-round ready-list sizes
  unsigned long long* bcount;   // [n + 64] per-round counts of vertices whose push is spread
  int32_t* big;                 // [list_cap] those vertices
  int64_t* big_cb;              // [list_cap] their first push chunk
  int32_t* cown;                // [chunk_cap] big-list entry of each push chunk
  int64_t chunk_cap;            // >= A / 256 + n
  unsigned long long* ccount;   // [n + 64] per-round push-chunk counts
  int64_t* boff;                // [n + 1] bitmap word offsets
  unsigned* used;               // [used_cap] colour bitmaps, ceil((deg + 1) / 32) words per vertex
  int64_t used_cap;             // >= A / 32 + n
  unsigned long long* round;    // [4] current round, grid-barrier counter and generation
  int64_t* tile_tmp;            // scan scratch
};
// Jones-Plassmann colouring of g (self-loops ignored).  Returns the number of colours.
// Uses ctrl->cnt[3, 4, 7]; synchronises the stream once per batch of rounds.
// In a batched run `seg` makes the priority hash the graph-local id.
int32_t jp_colour(Ctx& c, const GraphView<int32_t>& g_struct, const int32_t* perm, const int64_t* h_bucket_offs,
                  uint64_t seed, int32_t pass, int32_t* colour, const JpBuffers& jb, Ctrl* ctrl,
                  unsigned long long* h_pinned, cudaError_t* err, Segs seg = Segs(),
                  int64_t* rounds_out = nullptr);

// ---------------------------------------------------------------- aggregate.cu
// counts[c] = members, cdeg[c] = sum of member degrees (both zeroed by the caller).
void community_count(Ctx& c, const int32_t* Cp, const int64_t* rbeg, const int64_t* rend, int64_t n,
                     int32_t* counts, int64_t* cdeg);
// cverts[coff[c] + k] = k-th member (unordered); cursor zeroed by the caller.
void community_fill(Ctx& c, const int32_t* Cp, int64_t n, const int64_t* coff, int32_t* cursor, int32_t* cverts);

template <class M>
struct MergeArgs {
  GraphView<typename M::w_t> g;
  const int32_t* Cp;
  const int64_t* coff;
  const int32_t* cverts;
  const int64_t* cdeg;
  const int64_t* hoff;
  int64_t* hend;
  int32_t* otg;
  typename M::w_t* ow;
  int64_t nc;
  Ctrl* ctrl;
  int bucket = 0;  // set by merge_bucket (selects the traffic counters)
  int tf = 2;      // table slots per key of the distinct-key bound
};
template <class M>
void merge_bucket(Ctx& c, int bucket, const MergeArgs<M>& a, const int32_t* list, int64_t count);

// Dense copy of holey rows: out arcs at doff[r] for rows [0, n).
template <class W>
void compact_rows(Ctx& c, int64_t n, const int64_t* hbeg, const int64_t* hend, const int64_t* doff,
                  const int32_t* itg, const W* iw, int32_t* otg, W* ow);
// len[r] = hend[r] - hbeg[r]
void row_lengths(Ctx& c, int64_t n, const int64_t* hbeg, const int64_t* hend, int64_t* len);

// ---------------------------------------------------------------- giant.cu
// Sets n pool slots to {kEmpty, 0}.
void pool_init(Ctx& c, int32_t* slots, int64_t n);
// Plan of the multi-block path for giant rows: per giant k, ranges [off[k], off[k+1]) of arc
// chunks, table slots (in the shared pool) and table slices.
struct GiantPlan {
  int64_t* chunk_off = nullptr;  // [cap + 1]
  int64_t* tab_off = nullptr;    // [cap + 1]
  int64_t* slice_off = nullptr;  // [cap + 1]
  void* kid = nullptr;           // [cap] K_i->d accumulators (h_t)
  uint8_t* moved = nullptr;      // [cap]
  uint8_t* active = nullptr;     // [cap] local move: processed in the current class iteration
  void* part_s = nullptr;        // [slice_cap] best score per slice (s_t)
  int32_t* part_c = nullptr;     // [slice_cap] its community
  int32_t* cowner = nullptr;     // [chunk_cap] giant of each chunk
  int32_t* sowner = nullptr;     // [slice_cap] giant of each slice
  int64_t chunk_cap = 0, slice_cap = 0;
  int32_t* slots = nullptr;      // shared table pool, slot s = {key, value (h_t)} at slots[2s], [2s + 1]
                                 // (one 8-byte pair: a probe touches one sector); all {kEmpty, 0}
                                 // between uses
  unsigned* bits = nullptr;      // occupancy bitmap of the pool (local move), all zero between uses
  int64_t pool_slots = 0;
};
// Plan of the local-moving phase over every giant vertex of a pass, list[0, m) ordered class by
// class (chunks, tables, 1024-slot ranges); built once per pass.
template <class M>
void giant_move_plan(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* list, int64_t m, const GiantPlan& p,
                     Ctrl* ctrl);
// Local moving of the giants list[k0, k1) of one colour / random class under that plan.
// With `krng` (a step record's {list offset, k0, k1}) the range is read there.
template <class M>
void giant_move(Ctx& c, const GraphView<typename M::w_t>& g, const PassState<M>& st, const int32_t* list, int64_t k0,
                int64_t k1, const GiantPlan& p, bool fast, bool pruning, const int64_t* krng = nullptr);
// Plan kernels (kind: see giant.cu); slices of 2^slice_log table slots.
void giant_plan(Ctx& c, int kind, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                const int64_t* cdeg, int64_t n_bound, const int32_t* Cp, int32_t* gix, int slice_log,
                const GiantPlan& p, Ctrl* ctrl);
// Super-vertex rows of the giant communities clist[0, m): the concatenated member rows of each
// community (community-vertex CSR order) in chunks, community after community.  gix [nc] receives
// each community's giant index (-1 if not giant); deg_tmp [n] and memoff [n + 1] are scratch.
template <class M>
void giant_merge(Ctx& c, const MergeArgs<M>& a, const int32_t* clist, int64_t m, int32_t* gix, const GiantPlan& p,
                 int64_t* deg_tmp, int64_t* memoff, int64_t* tile_tmp);

// Chunk-only plan over the rows [rbeg, rend) of list[0, m).
void giant_chunk_plan(Ctx& c, const int32_t* list, int64_t m, const int64_t* rbeg, const int64_t* rend,
                      const GiantPlan& p, Ctrl* ctrl);
template <class M>
void giant_modularity(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* list, int64_t m, const int32_t* C,
                      typename M::a_t* tot, const GiantPlan& p, Ctrl* ctrl);
template <class W>
void giant_compact(Ctx& c, const int32_t* list, int64_t m, const int64_t* hbeg, const int64_t* hend,
                   const int64_t* doff, const int32_t* itg, const W* iw, int32_t* otg, W* ow, const GiantPlan& p,
                   Ctrl* ctrl);
// Compaction of holey rows listed by community-degree buckets (cperm, host offsets cb).
template <class W>
void compact_bucketed(Ctx& c, const int32_t* cperm, const int64_t* cb, const int64_t* hbeg, const int64_t* hend,
                      const int64_t* doff, const int32_t* itg, const W* iw, int32_t* otg, W* ow, const GiantPlan& gp,
                      Ctrl* ctrl);

// ---------------------------------------------------------------- modularity.cu
// Same value by degree-bucketed groups (dperm / hb: a degree-bucket sort of g), giant rows chunked.
template <class M>
void modularity_bucketed(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* C, typename M::a_t* tot,
                         Ctrl* ctrl, const int32_t* dperm, const int64_t* hb, const GiantPlan& gp);
// Q of membership C on dense CSR g; tot[n] scratch (zeroed inside); result in ctrl->q (and
// acc slots).  Integer mode exact.
template <class M>
void modularity(Ctx& c, const GraphView<typename M::w_t>& g, const int32_t* C, typename M::a_t* tot, Ctrl* ctrl);

// ---------------------------------------------------------------- batch.cu
// Union setup of a batch: vg0 (graph of every vertex), ao (arc range of every graph), graph-local
// targets -> union ids (bad targets counted in ctrl->cnt[1]), GraphCtl initialised from vo.
void batch_setup(Ctx& c, const int64_t* vo, int32_t G, int64_t n, const int64_t* offs, int64_t n_arcs,
                 const int32_t* tg_local, int32_t* tg_union, int64_t* ao, int32_t* vg0, GraphCtl* gc, Ctrl* ctrl);
// 2m per graph from K (pass 0); ctrl->cnt[6] counts integer graphs with 2m >= 2^31.
template <class M>
void batch_two_m(Ctx& c, GraphCtl* gc, int32_t G, const typename M::a_t* K, Ctrl* ctrl);
void batch_move_setup(Ctx& c, GraphCtl* gc, int32_t G, int max_iterations);
// Per-graph tolerance test after an iteration; ctrl->done once every graph is done.
template <class M>
void batch_finish(Ctx& c, Ctrl* ctrl, GraphCtl* gc, int32_t G);
// Pass tests per graph and next-level bases; ctrl->acc_i[3] = next level's vertex count.
void batch_pass_end(Ctx& c, GraphCtl* gc, int32_t G, const int64_t* newid, double tau_agg, bool last, Ctrl* ctrl);
// Renumbering, dendrogram lookup, next-level K and vg, graphs that stop leave the union.
template <class A>
void batch_next_level(Ctx& c, int32_t* Cp, int64_t n_cur, const int64_t* newid, const int32_t* vg, GraphCtl* gc,
                      int32_t G, int32_t* C, int64_t n0, const int32_t* vg0, const A* sig, const int32_t* occ,
                      A* k_next, int32_t* vg_next);
// Graphs still in the pass loop (max_passes = 0): singleton communities with local ids.
void batch_close(Ctx& c, int32_t* C, int64_t n0, const int32_t* vg0, GraphCtl* gc, int32_t G);
// Eq. 1 per graph on the input graphs (C graph-local); results in gc[g].q.
template <class M>
void batch_modularity(Ctx& c, const GraphView<typename M::w_t>& g0, const int32_t* C, const int32_t* vg0, GraphCtl* gc,
                      int32_t G, const int64_t* vo, const int32_t* dperm, const int64_t* hb, typename M::a_t* intra,
                      typename M::a_t* tot, int64_t n_comm_total);

// ---------------------------------------------------------------- api.cu hooks (host)
size_t handle_device_bytes(louvain_handle h);       // device bytes the handle holds
void handle_set_budget(louvain_handle h, size_t bytes);  // cap of its further allocations (0 = none)
void handle_trim(louvain_handle h);                 // free everything it caches

// ---------------------------------------------------------------- dynamic.cu
// Scratch (64-bit words) of a batch update: the deleted-pair set and the per-row counters.
int64_t update_scratch_words(int64_t n_new, int64_t n_del);
// Counts the arcs of every new row (surviving old arcs + inserted arcs) and scans them into
// out_off[n_new + 1]; ctrl->cnt[5] += ids out of range.  Returns the deleted-pair set's slot count.
int update_count(Ctx& c, int64_t n_old, int64_t n_arcs, const int64_t* off, const int32_t* tg, int64_t n_new,
                 const int32_t* du,
                 const int32_t* dv, int64_t n_del, const int32_t* iu, const int32_t* iv, const void* iw,
                 int64_t n_ins, unsigned long long* scratch, int64_t* out_off, int64_t* tile_tmp, Ctrl* ctrl);
// Writes the rows counted by update_count: surviving arcs first, then inserted arcs (each group in
// unspecified order).
void update_fill(Ctx& c, int64_t n_old, int64_t n_arcs, const int64_t* off, const int32_t* tg, const void* w,
                 int64_t n_new,
                 int64_t n_del, const int32_t* iu, const int32_t* iv, const void* iw, int64_t n_ins,
                 unsigned long long* scratch, unsigned slots, const int64_t* out_off, int32_t* otg, void* ow,
                 Ctrl* ctrl);
// Pass-0 state of a warm start: Cp = init, Sigma_c = sum of K_i over c's members, csize = member counts.
template <class M>
void warm_init(Ctx& c, const PassState<M>& st, const int32_t* init, int64_t n);

// ---------------------------------------------------------------- validate.cu
// ctrl->cnt[0..3] receive: bad offsets, bad targets, bad weights, asymmetry hash; ctrl->acc_f[0]
// the weight total (double), ctrl->acc_i[0] the integer weight total (saturating).
void validate_offsets(Ctx& c, int64_t n, int64_t n_arcs, const int64_t* offs, Ctrl* ctrl);
void validate_arcs(Ctx& c, int64_t n, const int64_t* offs, const int32_t* tg, const void* w, bool fp, Ctrl* ctrl);
// ctrl->cnt[5] += number of ids outside [0, hi).
void validate_range(Ctx& c, const int32_t* ids, int64_t m, int64_t hi, Ctrl* ctrl);
// zero ctrl->cnt[0..7], acc_i, acc_f
void validate_reset(Ctx& c, Ctrl* ctrl);

}  // namespace lv
