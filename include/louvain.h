/*
 * louvain.h -- C ABI of the GB300 Louvain library (liblouvain.so).
 *
 * The library computes the Louvain method as GVE-Louvain (arXiv 2312.04876) describes it:
 * passes of a local-moving phase (Algorithm 2, move score Eq. 2) and an aggregation phase
 * (Algorithm 3), driven by the pass loop of Algorithm 1, with modularity by Eq. 1.  Every step
 * runs in hand-written CUDA kernels for sm_103a on one GPU.
 *
 * Conventions shared by every entry point
 *   - Graphs are symmetric weighted CSR (Section 3: both arcs of every undirected edge are
 *     stored; a self-loop is stored once and counts once in K_i, sigma_c and 2m):
 *       offsets  int64 [n + 1], offsets[0] = 0, non-decreasing, offsets[n] = n_arcs
 *       targets  int32 [n_arcs], each in [0, n)
 *       weights  int32 (> 0) or float32 (> 0, finite) [n_arcs], as `wtype` says
 *     0 <= n < 2^31 - 1.  Duplicate arcs are summed.  Rows need not be sorted.
 *   - Pointers named `d_*` are DEVICE pointers on the handle's device; `h_*` are host pointers.
 *     The library never frees caller memory; inputs are read-only; outputs are written in place.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device outputs are complete
 *     when the call returns (the call synchronises the stream before returning).
 *   - Every call returns a louvain_status and never aborts, traps or prints.  On failure the
 *     handle keeps a message for louvain_last_error(); outputs are then unspecified.
 *   - Integer mode (LOUVAIN_W_INT32) computes exactly in integers and requires
 *     2m = sum of all arc weights < 2^31 (else LOUVAIN_ERR_OVERFLOW).  FP32 mode accumulates
 *     the per-vertex community sums in fp32 and keeps K, Sigma, 2m and scores in fp64.
 *   - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef LOUVAIN_H
#define LOUVAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct louvain_handle_s* louvain_handle;

typedef enum {
  LOUVAIN_OK = 0,
  LOUVAIN_ERR_INVALID = 1,   /* bad argument or malformed graph */
  LOUVAIN_ERR_OOM = 2,       /* device/host allocation failed or HBM budget exceeded */
  LOUVAIN_ERR_OVERFLOW = 3,  /* integer mode with 2m >= 2^31 */
  LOUVAIN_ERR_TIMEOUT = 4,   /* a bounded device wait gave up */
  LOUVAIN_ERR_CUDA = 5,      /* CUDA runtime error (message in louvain_last_error) */
  LOUVAIN_ERR_BUSY = 6       /* resource in use (serving: no free slot / ticket not ready) */
} louvain_status;

typedef enum { LOUVAIN_W_INT32 = 0, LOUVAIN_W_FP32 = 1 } louvain_wtype;

typedef enum {
  /* Colour-synchronous schedule: per pass a Jones-Plassmann colouring with priorities
   * hash(seed, pass, v); within a colour class every flagged vertex decides against the
   * class-start community totals, then all moves apply.  Integer mode is bit-exact and
   * run-to-run identical (the colouring-based ordering cited in Section 2). */
  LOUVAIN_MODE_DETERMINISTIC = 0,
  /* Asynchronous: vertices read and update live state with atomics (Section 4.1,
   * "asynchronous version"), with a singleton-swap guard against the GPU community-swap
   * pattern noted in Section 2.  Not reproducible run to run. */
  LOUVAIN_MODE_FAST = 1
} louvain_mode;

typedef struct {
  int32_t max_passes;            /* MAX_PASSES of Algorithm 1; unstated in the paper, default 10 */
  int32_t max_iterations;        /* MAX_ITERATIONS of Algorithm 2; Section 4.1.2: 20 */
  double tolerance;              /* initial per-iteration tolerance tau; Section 4.1.4: 0.01 */
  double tolerance_drop;         /* threshold scaling divisor; Section 4.1.3: 10 */
  double aggregation_tolerance;  /* tau_agg; Section 4.1.5: 0.8 (stop when |Gamma|/|V'| > tau_agg) */
  int32_t pruning;               /* vertex pruning (Section 4.1.6): 1 on (default), 0 off */
  int32_t mode;                  /* louvain_mode */
  uint64_t seed;                 /* colouring priority seed (deterministic mode) */
  int32_t validate;              /* 1: check the CSR (offsets, ranges, weights, symmetry, 2m) */
  int32_t compact;               /* 1: compact each super-vertex graph to dense CSR (default);
                                    0: run later passes on the holey CSR with degrees */
  int32_t pass_modularity;       /* 1: fill louvain_pass_stats.modularity (extra arc sweep) */
  int32_t profile;               /* 1: time every kernel launch with CUDA events on `stream` and
                                    keep per-kernel totals for louvain_kernel_profile() */
  int32_t fast_classes;          /* fast mode: vertices are split into this many random classes
                                    (hash3(seed, pass, v) mod K) processed one after another; moves
                                    inside a class stay asynchronous.  Default 16; 1 = all at once */
  int32_t fast_giant_class;      /* fast mode: 1 = every giant row (> 4096 arcs) of a pass in one class
                                    (one multi-block giant pipeline per iteration); 0 = hash classes */
  int32_t lm_blocks_per_sm;      /* grid cap of the local-moving kernels in blocks per SM (0 = 16); the
                                    degree buckets of a class run concurrently, so smaller grids let
                                    them share the SMs */
  int32_t giant_min_degree;      /* rows longer than this take the multi-block giant path; 2048..4096
                                    (0 = 4096: rows of 2049..4096 arcs use one block with a 64 KB table) */
  int32_t fast_classes_later;    /* fast mode: iterations after the first of a pass may run the classes
                                    in as few as this many groups of consecutive classes (default 1;
                                    0 = fast_classes, every class on its own).  The group count is
                                    raised to fast_classes * (1024 * SMs) / |V'| so that a group is
                                    grouped only where it is much larger than the vertices the GPU
                                    holds in flight (small graphs keep every class on its own).  The
                                    first iteration, where most vertices move, takes every class on
                                    its own */
  int32_t wait_spins;            /* bound of the device-side waits (the colouring's grid barrier in
                                    deterministic mode): polls of about 64 ns each before a waiting
                                    block gives up (0 = built-in, about 0.3 s).  A wait that runs out
                                    ends the kernel on every block and the call returns
                                    LOUVAIN_ERR_TIMEOUT; the handle stays usable */
  int32_t host_arcs;             /* 1: graphs whose arcs do not fit in HBM.  The super-vertex graphs'
                                    arc buffers (four of n_arcs entries) live in pinned host memory
                                    that the kernels read and write in place over NVLink-C2C, and
                                    louvain_run_host reads the input's targets and weights in place
                                    (registering them for the call unless already pinned) and copies
                                    only the offsets; per-vertex state stays in HBM.  Results are
                                    those of the default placement (0) */
  int32_t table_factor;          /* hash-table slots per key a table may have to hold: 1, 2 or 4
                                    (tables up to full, half full or a quarter full; 0 = 2), for the
                                    shared-memory tables of local moving and merging and the giant
                                    rows' global tables.  Integer-weight results do not depend on it
                                    (exact sums, ties by id); it trades probe length for memory */
  int32_t fast_sync_small;       /* fast mode on small graphs: 0 = where the input graph -- a batch:
                                    its mean graph -- fits in what the GPU holds in flight (1024
                                    vertices per SM) and rows over 512 arcs hold at most a fifth of
                                    its arcs, run every pass on the colour-synchronous schedule of
                                    the deterministic mode, else every pass asynchronously (each
                                    class is one wave there anyway; asynchronous waves left 2-3% of
                                    small planted-partition graphs 0.03-0.066 below it; a graph
                                    carried by hubs needs hundreds of colours); 1 = asynchronous
                                    random classes always; 2 = colour-synchronous always */
} louvain_params;

typedef struct {
  int32_t pass;
  int32_t iterations;            /* l_i of the pass */
  int64_t moves;                 /* vertex moves performed in the pass */
  int64_t n_vertices;            /* |V'| at the start of the pass */
  int64_t n_arcs;                /* arcs of G' at the start of the pass */
  int64_t n_communities;         /* |Gamma| after the local-moving phase */
  double modularity;             /* Q after the local-moving phase (NaN unless pass_modularity) */
  float ms_colour, ms_move, ms_aggregate, ms_other;
  int32_t colours;               /* deterministic mode: colour classes of the pass (0 in fast mode) */
  int32_t colour_rounds;         /* deterministic mode: Jones-Plassmann rounds that coloured vertices */
  float ms_graph;                /* host time of capturing the pass's iteration graphs and making them
                                    executable (the device waits meanwhile); 0 with profile = 1 */
  int32_t graphs_instantiated;   /* of those graphs, how many were instantiated anew (the others
                                    updated a cached executable of the same shape in place) */
} louvain_pass_stats;

typedef struct {
  double modularity;             /* Eq. 1 of the returned membership on the input graph */
  int32_t passes;
  int32_t total_iterations;
  int64_t n_communities;
  float ms_total;                /* device time of the whole run (CUDA events) */
  int32_t kernel_launches;       /* kernels this call launched */
  int32_t reserved;
} louvain_result;

/* Create a handle on CUDA device `device`.  hbm_budget_bytes caps the workspace the handle may
 * allocate (0 = no cap).  Returns LOUVAIN_ERR_CUDA if the device is unusable. */
louvain_status louvain_create(louvain_handle* h, int device, size_t hbm_budget_bytes);

/* Release the handle's workspace and events.  NULL is a no-op. */
void louvain_destroy(louvain_handle h);

/* Defaults from Section 4.1: max_iterations 20, tolerance 0.01, tolerance_drop 10,
 * aggregation_tolerance 0.8, pruning on; max_passes 10; deterministic mode; seed 0;
 * validate 1; compact 1; pass_modularity 0; profile 0; fast_classes 16; fast_classes_later 1;
 * fast_giant_class, lm_blocks_per_sm, giant_min_degree, wait_spins, host_arcs and table_factor 0
 * (their built-in choices). */
louvain_status louvain_default_params(louvain_params* p);

/* Algorithm 1 as louvain_run, but the first pass starts from the membership d_initial[n] (device,
 * ids in [0, n)) instead of singleton communities: C' = d_initial, Sigma_c = the sum of K_i over
 * c's members, every vertex flagged for processing; later passes are unchanged.  This is the warm
 * start of a dynamic graph -- pass the membership of the graph before a batch update (extended
 * with any new vertices, e.g. as singletons) and the updated graph (louvain_update_graph).  The
 * paper keeps the first pass's graph in a format open to batch updates (Section 4.2), gives later
 * passes an initial membership (Figure 2) and names dynamic graphs as its next step (Conclusion).
 * d_membership gets the canonical result as in louvain_run.  LOUVAIN_ERR_INVALID for an id out of
 * range.  A vertex can only join a neighbour's community, so a community of the initial membership
 * never splits (it can only grow or empty). */
louvain_status louvain_run_from(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, const int32_t* d_initial,
                                int32_t* d_membership, louvain_result* res, louvain_pass_stats* stats,
                                int32_t stats_cap, int32_t* n_stats);

/* A batch update of a symmetric CSR (Section 4.2: the first pass's graph in a format open to batch
 * updates) into caller buffers: rows grow from n_old to n_new (>= n_old; new rows start empty);
 * every arc between u and v of a deleted edge {d_del_u[k], d_del_v[k]} is removed, in both
 * directions and with all its duplicates (deleting a pair that is not an edge is a no-op); then
 * each inserted edge (d_ins_u[k], d_ins_v[k]) with weight d_ins_w[k] (the graph's wtype) adds the
 * arc u->v and, if u != v, the arc v->u (an edge that already exists gets a second arc, which the
 * method sums).  Row r of the result holds its surviving arcs, then its inserted arcs, each group in
 * unspecified order (no step of the method depends on the order of a row).  All arrays are device arrays; d_out_offsets [n_new + 1],
 * d_out_targets / d_out_weights hold out_cap arcs and must not overlap the input.  *out_arcs (host)
 * gets the updated arc count, also when it exceeds out_cap (then LOUVAIN_ERR_INVALID and only the
 * offsets are written).  LOUVAIN_ERR_INVALID for an id outside [0, n_new). */
louvain_status louvain_update_graph(louvain_handle h, int64_t n_old, int64_t n_arcs, const int64_t* d_offsets,
                                    const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                    int64_t n_new, int64_t n_del, const int32_t* d_del_u, const int32_t* d_del_v,
                                    int64_t n_ins, const int32_t* d_ins_u, const int32_t* d_ins_v,
                                    const void* d_ins_w, void* stream, int64_t* d_out_offsets,
                                    int32_t* d_out_targets, void* d_out_weights, int64_t out_cap,
                                    int64_t* out_arcs);

/* Device bytes the handle holds now: every workspace buffer it allocated and has not freed
 * (grown on demand, kept across calls, released by louvain_destroy).  *bytes (host). */
louvain_status louvain_workspace_bytes(louvain_handle h, size_t* bytes);

/* Fault injection for tests of the out-of-memory path (the paper has no counterpart): the k-th
 * device allocation the handle makes from now on (k >= 1) fails once, as if cudaMalloc had run
 * out of memory; k = 0 cancels.  The call that meets the failure returns LOUVAIN_ERR_OOM and the
 * handle stays usable.  LOUVAIN_ERR_INVALID for k < 0. */
louvain_status louvain_inject_alloc_failure(louvain_handle h, int32_t k);

/* Message of the last failure on this handle ("" if none).  Valid until the next call. */
const char* louvain_last_error(louvain_handle h);

/* Static name of a status code. */
const char* louvain_status_string(louvain_status s);

/* Algorithm 1 on a device-resident CSR.  Writes d_membership[n] (device, caller-owned) with the
 * community of every vertex, renumbered densely in order of the smallest member id's community
 * rank (id = rank of the community among occupied ids after the final dendrogram lookup).
 * res (optional) receives modularity (Eq. 1 on the input graph), passes, totals, device time;
 * stats (optional, host array of stats_cap) receives one entry per pass, *n_stats their count. */
louvain_status louvain_run(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                           const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                           const louvain_params* p, void* stream, int32_t* d_membership,
                           louvain_result* res, louvain_pass_stats* stats, int32_t stats_cap,
                           int32_t* n_stats);

/* Outcome of one graph of a batch (louvain_run_batch). */
typedef struct {
  double modularity;             /* Eq. 1 of the graph's membership on the graph */
  int32_t passes;
  int32_t total_iterations;      /* sum of l_i over the graph's passes */
  int64_t n_communities;
} louvain_graph_result;

/* Algorithm 1 on each of n_graphs independent graphs at once.  The paper runs one graph; this
 * entry point is a throughput extension that does not change the arithmetic: every graph gets
 * exactly the membership, modularity and pass/iteration counts louvain_run gives it alone (in
 * deterministic mode bit for bit; the colouring priorities and random classes hash graph-local
 * ids), while every kernel launch covers all graphs still running.
 *
 * Segmented CSR: graph k owns the vertex range [graph_vtx_offs[k], graph_vtx_offs[k+1]) of the
 * union (graph_vtx_offs: HOST int64 [n_graphs + 1], non-decreasing, graph_vtx_offs[0] = 0,
 * n = graph_vtx_offs[n_graphs] < 2^31).  d_offsets (DEVICE int64 [n + 1]) are the union's row
 * offsets, so graph k's arcs are [d_offsets[vo[k]], d_offsets[vo[k+1]]); d_targets (DEVICE int32
 * [n_arcs]) hold GRAPH-LOCAL vertex ids (0 .. n_k - 1); d_weights as in louvain_run.  Inputs are
 * read only.  d_membership (DEVICE int32 [n], caller-owned) receives graph-local canonical
 * community ids.  results (HOST [n_graphs], optional) one entry per graph; res (optional): passes
 * = the largest pass count, total_iterations and n_communities summed, modularity NaN, device time.
 * Errors: LOUVAIN_ERR_INVALID (bad ranges, a target outside its graph, validation failures),
 * LOUVAIN_ERR_OVERFLOW (integer weights with 2m >= 2^31 in some graph), LOUVAIN_ERR_OOM,
 * LOUVAIN_ERR_CUDA.  Scratch beyond louvain_run's: 4 bytes per arc and 12 per vertex. */
louvain_status louvain_run_batch(louvain_handle h, int32_t n_graphs, const int64_t* graph_vtx_offs, int64_t n_arcs,
                                 const int64_t* d_offsets, const int32_t* d_targets, const void* d_weights,
                                 louvain_wtype wtype, const louvain_params* p, void* stream, int32_t* d_membership,
                                 louvain_graph_result* results, louvain_result* res);

/* Autotuning (a systems extension; the paper tunes nothing at run time).  Times full runs of the
 * given graph (device time, best of `reps`, each candidate after one untimed run that builds its
 * iteration graphs and buffers) under every combination of the performance knobs that
 * leave the arithmetic unchanged -- giant_min_degree in {4096, 2048} (which kernel takes rows of
 * 2049..4096 arcs: the one-block 64 KB table or the multi-block giant path), lm_blocks_per_sm in
 * {16, 4} and compact in {1, 0}; then table_factor 4 against 2 (hash-table sizes) with the best of
 * those -- and writes *p with the fastest setting into *tuned (other fields copied; *best_ms its
 * time).  In deterministic mode every candidate returns the same
 * membership; d_membership (device, n entries) receives the last run's.  Costs 9 x (reps + 1) runs. */
louvain_status louvain_autotune(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, int32_t* d_membership, int32_t reps,
                                louvain_params* tuned, float* best_ms);

/* louvain_autotune for a batch (the arguments of louvain_run_batch). */
louvain_status louvain_autotune_batch(louvain_handle h, int32_t n_graphs, const int64_t* graph_vtx_offs,
                                      int64_t n_arcs, const int64_t* d_offsets, const int32_t* d_targets,
                                      const void* d_weights, louvain_wtype wtype, const louvain_params* p,
                                      void* stream, int32_t* d_membership, int32_t reps, louvain_params* tuned,
                                      float* best_ms);

/* ---------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop (a throughput extension; the paper has no
 * counterpart).  Requests are host CSRs (int64 offsets, graph-local int32 targets, weights).
 * `lanes` worker threads, each with its own CUDA stream and workspace, take the oldest queued
 * request and every other queued request of its class that fits (at most max_batch_graphs graphs
 * and max_batch_arcs arcs per batch, 0 = no arc cap) whenever they are free and run them as one
 * louvain_run_batch call.  A class is a weight type and a side of the in-flight window (1024
 * vertices per SM): fast mode picks a batch's schedule by its mean graph, and a small graph batched
 * with a large one would take the large one's.  So requests arriving while
 * others run are admitted as lanes and memory free up, and the lanes' work overlaps on the device.
 * Device memory: every batch reserves an upper bound of what it needs (256 B per vertex + 72 B
 * per arc + 64 MiB) and the reservations of all lanes never exceed hbm_budget_bytes; each result
 * is the one louvain_run gives the graph alone (deterministic mode: identical).
 * --------------------------------------------------------------------------------------------- */
typedef struct louvain_server_s* louvain_server;

typedef struct {
  int32_t ready;                 /* 1 when the request has finished (then the fields below are set) */
  int32_t status;                /* louvain_status of the request */
  louvain_graph_result result;
  double latency_ms;             /* submit -> membership in the caller's buffer (host steady clock) */
  double queue_ms;               /* submit -> its batch started */
  int32_t batch_graphs;          /* graphs in the batch it ran in */
  int32_t reserved;
  /* where its batch's time went (the whole batch's, shared by the graphs in it): */
  double prep_ms;                /* host: union offsets built from the requests' offsets */
  double upload_ms;              /* device: the copies of the union CSR to the lane's buffers */
  double run_ms;                 /* device: louvain_run_batch on the lane's stream */
  double download_ms;            /* device: the memberships' copies to the callers' buffers */
} louvain_serve_result;

/* Start a server on `device` with the given parameters (mode, tolerances, seed ...).
 * LOUVAIN_ERR_INVALID for lanes outside [1, 64], max_batch_graphs < 1, a zero budget. */
louvain_status louvain_serve_create(louvain_server* s, int device, size_t hbm_budget_bytes, int32_t lanes,
                                    int32_t max_batch_graphs, int64_t max_batch_arcs, const louvain_params* p);

/* Queue one graph.  The host arrays (offsets [n+1] with offsets[0] = 0 and offsets[n] = n_arcs,
 * targets and weights [n_arcs]) are read, and h_membership [n] written, by the server until the
 * request's result has been collected with louvain_serve_poll: the caller keeps them alive.
 * *ticket identifies the request.  LOUVAIN_ERR_OOM if the graph alone exceeds the budget,
 * LOUVAIN_ERR_BUSY after louvain_serve_destroy has begun. */
louvain_status louvain_serve_submit(louvain_server s, int64_t n, int64_t n_arcs, const int64_t* h_offsets,
                                    const int32_t* h_targets, const void* h_weights, louvain_wtype wtype,
                                    int32_t* h_membership, uint64_t* ticket);

/* Result of a request, waiting up to wait_ms milliseconds (0 = do not wait).  out->ready = 0 if it
 * has not finished; once a finished result is returned the ticket is released.  Unknown ticket:
 * LOUVAIN_ERR_INVALID. */
louvain_status louvain_serve_poll(louvain_server s, uint64_t ticket, int32_t wait_ms, louvain_serve_result* out);

/* Finish the queued and running requests, then stop the lanes and free everything. */
void louvain_serve_destroy(louvain_server s);

/* louvain_run for HOST buffers: copies the CSR to the device (through the handle's workspace),
 * runs, and copies the membership back to h_membership[n].  Pinned host memory gives the
 * fastest copies; pageable memory works.  The copies are part of the call. */
louvain_status louvain_run_host(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* h_offsets,
                                const int32_t* h_targets, const void* h_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, int32_t* h_membership,
                                louvain_result* res, louvain_pass_stats* stats, int32_t stats_cap,
                                int32_t* n_stats);

/* Eq. 1 (second form) of a membership on a CSR.  d_membership[n] ids must lie in [0, n).
 * Integer mode: Q = (2m sum sigma_c - sum Sigma_c^2) / (2m)^2 from exact int64 sums, one
 * division in double; FP32 mode: fp64 sums.  Q = 0 when 2m = 0.  Result in *q (host). */
louvain_status louvain_modularity(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                  const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                  const int32_t* d_membership, void* stream, double* q);

/* Jones-Plassmann colouring used by the deterministic schedule: colour(v) = smallest colour not
 * taken by a neighbour u != v of higher priority, priority (hash3(seed, pass, v), v).  Equals
 * greedy colouring in decreasing priority.  Writes d_colour[n], *n_colours (host). */
louvain_status louvain_colour(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                              const int32_t* d_targets, uint64_t seed, int32_t pass, void* stream,
                              int32_t* d_colour, int32_t* n_colours);

/* One local-moving phase (Algorithm 2) from singleton communities on a CSR, with the colouring
 * of pass `pass` (deterministic mode) and tolerance `tau`.  Writes d_cprime[n] (community ids,
 * not renumbered), *iterations (l_i) and *moves (host). */
louvain_status louvain_local_move(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                  const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                  const louvain_params* p, int32_t pass, double tau, void* stream,
                                  int32_t* d_cprime, int32_t* iterations, int64_t* moves);

/* Algorithm 3: super-vertex graph of a dense membership d_membership[n] in [0, n_comm).
 * Writes the compacted CSR: d_out_offsets[n_comm + 1], d_out_targets / d_out_weights (capacity
 * n_arcs each; weights in the input's wtype: int32 sums in integer mode, fp32 sums in FP32
 * mode) and *out_arcs (host).  Self-loops hold the intra-community weight.  Row order within a
 * super-vertex is unspecified. */
louvain_status louvain_aggregate(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                 const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                 const int32_t* d_membership, int64_t n_comm, void* stream,
                                 int64_t* d_out_offsets, int32_t* d_out_targets, void* d_out_weights,
                                 int64_t* out_arcs);

/* Per-kernel totals of the last louvain_run made with params.profile = 1: for each kernel class
 * (local-move buckets, Sigma apply, merge buckets, compaction, colouring, modularity) the number of
 * timed launches, their summed device time (CUDA events recorded on the run's stream around each
 * launch) and the algorithmic bytes those launches had to move (from device-side counters of
 * vertices, arcs, candidates and moves; formulas in the design notes).  Writes up to cap entries
 * to out (host), the count to *n. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double algorithmic_bytes;
} louvain_kernel_stat;

louvain_status louvain_kernel_profile(louvain_handle h, louvain_kernel_stat* out, int32_t cap, int32_t* n);

/* Exclusive prefix sum (Algorithm 3's exclusiveScan) of d_in[count] int64 into d_out[count + 1]
 * (d_out[count] = total); d_in == d_out is allowed.  *total (host, optional). */
louvain_status louvain_exclusive_scan(louvain_handle h, const int64_t* d_in, int64_t* d_out, int64_t count,
                                      void* stream, int64_t* total);

/* louvain_exclusive_scan without any allocation (the paper has no counterpart; it exists for
 * callers that cannot call cudaMalloc -- a host application whose memory manager owns all device
 * memory, e.g. a framework's caching allocator or a fixed HBM budget already handed out, or a
 * latency-critical loop that cannot take cudaMalloc / cudaFree's implicit device-wide
 * synchronisation).  Needs no handle.  Same result and layout as louvain_exclusive_scan:
 * d_out[0, count) = exclusive prefix sums of d_in[0, count) (int64, device), d_out[count] = total,
 * d_in == d_out allowed, *total (host, optional).  count must not exceed 2^26 (67,108,864) elements,
 * else LOUVAIN_ERR_INVALID.  The scratch is a 128 KiB __device__ array in the library that every GPU
 * loading the library keeps until the process exits; the call allocates and frees nothing (its
 * address is looked up on the first call on each device).  All calls on a device share the one
 * scratch array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.  Synchronises `stream`
 * before returning.  LOUVAIN_ERR_CUDA on a CUDA failure. */
louvain_status louvain_exclusive_scan_static(const int64_t* d_in, int64_t* d_out, int64_t count, void* stream,
                                             int64_t* total);

#ifdef __cplusplus
}
#endif

#endif /* LOUVAIN_H */
