// api.cu -- the C ABI of liblouvain.so and the host side of Algorithm 1.
//
// The pass loop runs on the host and drives device kernels on the caller's stream; the local
// moving iterations are enqueued in small batches and stop on a device-side convergence flag,
// so the host only synchronises a few times per pass (bucket counts, community count, end of
// the local-moving phase).  All scratch belongs to the handle, is allocated on first use and
// reused (the paper's preallocated CSRs, Section 4.1.7-8): two arc buffers (a holey merge target
// and a dense compaction target), two sets of row descriptors, and per-vertex state.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <unistd.h>

#include "internal.cuh"

using namespace lv;

namespace {

struct DevAlloc {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  bool host = false;  // pinned, mapped host memory (cudaHostAlloc) instead of device memory
};

struct RowSet {
  int64_t* hoff = nullptr;  // [n+1] holey offsets (scan of community total degree)
  int64_t* hend = nullptr;  // [n]   holey row ends
  int64_t* doff = nullptr;  // [n+1] dense offsets after compaction
};

struct Workspace {
  int64_t n_cap = -1, a_cap = -1;
  DevAlloc core;
  // per vertex
  void *K0 = nullptr, *K = nullptr, *Sig = nullptr, *tot = nullptr;  // 8-byte accumulators
  int32_t *Cp = nullptr, *colour = nullptr, *csize = nullptr, *mv_from = nullptr, *mv_to = nullptr;
  int32_t *perm = nullptr, *cperm = nullptr, *occ = nullptr, *counts = nullptr, *cursor = nullptr;
  int32_t *cverts = nullptr, *jcnt = nullptr, *jl0 = nullptr, *jl1 = nullptr, *jbig = nullptr;
  unsigned long long *jrc = nullptr, *jbc = nullptr, *jround = nullptr, *jcc = nullptr;
  int64_t* jbcb = nullptr;
  int32_t* jcown = nullptr;
  int64_t jchunk_cap = 0;
  int64_t* jboff = nullptr;
  unsigned* jused = nullptr;
  int64_t jused_cap = 0;
  uint8_t* flags = nullptr;
  int64_t *newid = nullptr, *coff = nullptr, *cdeg = nullptr, *len = nullptr, *tile_tmp = nullptr;
  RowSet rows[2];
  // arcs of the super-vertex graphs (holey merge target A, compaction target B), in HBM or, for
  // graphs whose arcs do not fit there, in pinned host memory the kernels reach over NVLink-C2C
  DevAlloc arc_alloc;
  int64_t arc_cap = -1;
  int32_t *tgA = nullptr, *tgB = nullptr;
  void *wA = nullptr, *wB = nullptr;
  Ctrl* ctrl = nullptr;
  // lazily sized
  DevAlloc keys_alloc;
  int64_t key_cap = 0;
  int64_t* keyoffs = nullptr;
  int32_t* keycur = nullptr;
  DevAlloc gt_alloc;
  int64_t gt_slots_total = 0;
  unsigned* gt_bits = nullptr;
  int32_t* pool = nullptr;    // giant-row table pool: gt_slots_total {key, value} pairs
  int32_t* dperm = nullptr;   // [n] vertex ids by degree bucket, kept for the whole pass
  DevAlloc desc_alloc;        // step records of captured iterations (kStepWords per class step)
  DevAlloc upd_alloc;         // batch graph update: deleted-pair set, row counters, scan scratch
  unsigned long long* upd = nullptr;
  int64_t upd_words = 0;
  int64_t* desc = nullptr;
  int64_t desc_cap = 0;       // int64 words
  int32_t* glist = nullptr;   // [gcap] giant vertices of a pass, class by class
  int32_t* csz = nullptr;     // [n] table size of each giant community
  GiantPlan gp, gpv;          // plans of giant vertices / communities and of giant members
  DevAlloc in_alloc;
  int64_t in_n = -1, in_a = -1;
  int64_t* in_offs = nullptr;
  int32_t* in_tg = nullptr;
  void* in_w = nullptr;
  int32_t* in_mem = nullptr;
  // batched runs (louvain_run_batch): per-graph control and the union's segmentation
  DevAlloc batch_alloc;
  int64_t b_graphs = -1, b_n = -1, b_a = -1;
  GraphCtl* gc = nullptr;     // [G]
  int64_t* vo = nullptr;      // [G + 1] input vertex ranges
  int64_t* ao = nullptr;      // [G + 1] input arc ranges
  int32_t* vg0 = nullptr;     // [n] graph of each input vertex
  int32_t *vgA = nullptr, *vgB = nullptr;  // [n] graph of each vertex of the current / next level
  int32_t* tgU = nullptr;     // [A] input targets as union ids
};

}  // namespace

// Kernel classes of the per-launch profile.
enum KClass {
  kLm0 = 0,            // local-move buckets 0..6
  kApply = kNumBuckets,
  kMg0,                // merge buckets 0..6
  kCompact = kMg0 + kNumBuckets,
  kColour,
  kModularity,
  kNumClasses
};
static const char* const kClassNames[kNumClasses] = {
    "local_move_b0_g4", "local_move_b1_g8", "local_move_b2_warp", "local_move_b3_warp1k", "local_move_b4_block4k",
    "local_move_b5_block8k", "local_move_b6_giant", "sigma_apply", "merge_b0_g4", "merge_b1_g8", "merge_b2_warp",
    "merge_b3_warp1k", "merge_b4_block4k", "merge_b5_block8k", "merge_b6_giant", "compact", "colour_jp",
    "modularity"};

struct Profile {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  struct Rec { int cls; size_t e0, e1; };
  std::vector<Rec> recs;
  int64_t launches[kNumClasses] = {};
  double ms[kNumClasses] = {};
  double bytes[kNumClasses] = {};
  bool valid = false;
};

struct louvain_handle_s {
  int device = 0;
  int num_sms = 152;
  size_t budget = 0;
  std::string err;
  Workspace ws;
  unsigned long long* pin = nullptr;  // pinned host staging
  size_t pin_bytes = 0;
  std::vector<cudaEvent_t> events;
  Profile prof;
  // CUDA-graph replay of local-moving iterations: one side stream per degree bucket (the buckets of
  // a colour / random class run concurrently) and fork / join events
  cudaStream_t side[kNumBuckets] = {};
  cudaStream_t cap = nullptr;  // capture origin (the caller's stream may be the legacy one)
  std::vector<cudaEvent_t> fork_ev, join_ev;
  bool use_graphs = true;
  // Executable graphs of earlier phases, keyed by everything their launches depend on: an
  // iteration with the same key replays one with no capture at all; a full cache updates one of the
  // same topology in place (cudaGraphExecUpdate, ~0.1 ms for a 16-class iteration) instead of
  // instantiating anew (~2.6 ms); least recently used evicted beyond kExecCache.
  struct CachedExec {
    cudaGraphExec_t e = nullptr;
    size_t nodes = 0;
    uint64_t used = 0;
    int64_t launches = 0;          // kernels per replay
    std::vector<int64_t> key;      // everything the captured launches depend on (see iteration_key)
    uint64_t call = 0;             // API call that last used it
  };
  std::vector<CachedExec> execs;
  uint64_t exec_clock = 0;
  int64_t* dpin = nullptr;         // pinned staging of the step records
  int64_t dpin_cap = 0;
  uint64_t call_seq = 0;           // API calls so far (begin_call)
  int64_t fail_alloc_in = 0;       // > 0: the fail_alloc_in-th device allocation from now fails (injected)
  bool arcs_host = false;          // params.host_arcs of the current call: arc buffers in host memory
};

constexpr size_t kExecCache = 16;

namespace {

// Device bytes (host-resident arc buffers are not HBM and do not count against the budget).
size_t total_bytes(const Workspace& ws) {
  return ws.core.bytes + ws.keys_alloc.bytes + ws.gt_alloc.bytes + ws.in_alloc.bytes + ws.batch_alloc.bytes +
         ws.desc_alloc.bytes + ws.upd_alloc.bytes + (ws.arc_alloc.host ? 0 : ws.arc_alloc.bytes);
}

void free_all(DevAlloc& a) {
  for (void* p : a.ptrs) {
    if (a.host) cudaFreeHost(p);
    else cudaFree(p);
  }
  a.ptrs.clear();
  a.bytes = 0;
}

louvain_status set_err(louvain_handle h, louvain_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

louvain_status cuda_err(louvain_handle h, cudaError_t e, const char* where) {
  return set_err(h, LOUVAIN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
bool dalloc(louvain_handle h, DevAlloc& a, T** p, int64_t count) {
  size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  bytes = (bytes + 255) & ~(size_t)255;
  if (!a.host && h->budget && total_bytes(h->ws) + bytes > h->budget) return false;
  if (h->fail_alloc_in > 0 && --h->fail_alloc_in == 0) return false;  // louvain_inject_alloc_failure
  void* q = nullptr;
  void* d = nullptr;
  if (a.host) {
    // pinned and mapped: the kernels read and write it in place over NVLink-C2C
    if (cudaHostAlloc(&q, bytes, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (cudaHostGetDevicePointer(&d, q, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(q);
      return false;
    }
  } else {
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    d = q;
  }
  a.ptrs.push_back(q);
  a.bytes += bytes;
  *p = reinterpret_cast<T*>(d);
  return true;
}

// The four arc buffers of the super-vertex graphs, `a` arcs each, placed as the current call asks
// (h->arcs_host); a placement change reallocates them.
louvain_status ensure_arcs(louvain_handle h, int64_t a) {
  Workspace& ws = h->ws;
  if (ws.arc_cap >= a && ws.arc_alloc.host == h->arcs_host && ws.tgA) return LOUVAIN_OK;
  const int64_t ac = (ws.arc_alloc.host == h->arcs_host && ws.arc_cap > a) ? ws.arc_cap : a;
  free_all(ws.arc_alloc);
  ws.arc_cap = -1;
  ws.tgA = ws.tgB = nullptr;
  ws.wA = ws.wB = nullptr;
  ws.arc_alloc.host = h->arcs_host;
  DevAlloc& d = ws.arc_alloc;
  if (!(dalloc(h, d, &ws.tgA, ac) && dalloc(h, d, &ws.tgB, ac) && dalloc(h, d, (int32_t**)&ws.wA, ac) &&
        dalloc(h, d, (int32_t**)&ws.wB, ac))) {
    free_all(ws.arc_alloc);
    ws.tgA = ws.tgB = nullptr;
    ws.wA = ws.wB = nullptr;
    return set_err(h, LOUVAIN_ERR_OOM, h->arcs_host ? "pinned host allocation of the arc buffers failed"
                                                    : "arc-buffer allocation failed or exceeds the HBM budget");
  }
  ws.arc_cap = ac;
  return LOUVAIN_OK;
}

louvain_status ensure_pinned(louvain_handle h, size_t bytes) {
  if (h->pin_bytes >= bytes) return LOUVAIN_OK;
  if (h->pin) cudaFreeHost(h->pin);
  h->pin = nullptr;
  size_t nb = bytes < 65536 ? 65536 : bytes * 2;
  if (cudaMallocHost(&h->pin, nb) != cudaSuccess) {
    cudaGetLastError();
    h->pin_bytes = 0;
    return set_err(h, LOUVAIN_ERR_OOM, "pinned host allocation failed");
  }
  h->pin_bytes = nb;
  return LOUVAIN_OK;
}

louvain_status ensure_workspace(louvain_handle h, int64_t n, int64_t a) {
  Workspace& ws = h->ws;
  if (ws.n_cap >= n && ws.a_cap >= a && ws.ctrl) return ensure_arcs(h, a);
  int64_t nc = n > ws.n_cap ? n : ws.n_cap;
  int64_t ac = a > ws.a_cap ? a : ws.a_cap;
  free_all(ws.core);
  ws.n_cap = ws.a_cap = -1;
  DevAlloc& d = ws.core;
  const int64_t n1 = nc + 1;
  bool ok = true;
  ok = ok && dalloc(h, d, (long long**)&ws.K0, n1) && dalloc(h, d, (long long**)&ws.K, n1) &&
       dalloc(h, d, (long long**)&ws.Sig, n1) && dalloc(h, d, (long long**)&ws.tot, n1);
  ok = ok && dalloc(h, d, &ws.Cp, n1) && dalloc(h, d, &ws.colour, n1) && dalloc(h, d, &ws.csize, n1) &&
       dalloc(h, d, &ws.mv_from, n1) && dalloc(h, d, &ws.mv_to, n1) && dalloc(h, d, &ws.perm, n1) &&
       dalloc(h, d, &ws.cperm, n1) && dalloc(h, d, &ws.occ, n1) && dalloc(h, d, &ws.counts, n1) &&
       dalloc(h, d, &ws.cursor, n1) && dalloc(h, d, &ws.cverts, n1) && dalloc(h, d, &ws.jcnt, n1) &&
       dalloc(h, d, &ws.jl0, n1) && dalloc(h, d, &ws.jl1, n1) && dalloc(h, d, &ws.jbig, n1);
  ws.jused_cap = ac / 32 + n1 + 64;
  ws.jchunk_cap = ac / 256 + n1 + 64;
  ok = ok && dalloc(h, d, &ws.jbcb, n1) && dalloc(h, d, &ws.jcown, ws.jchunk_cap) && dalloc(h, d, &ws.jcc, n1 + 64);
  ok = ok && dalloc(h, d, &ws.jboff, n1 + 1) && dalloc(h, d, &ws.jused, ws.jused_cap) &&
       dalloc(h, d, &ws.jbc, n1 + 64) && dalloc(h, d, &ws.jround, 4);
  ok = ok && dalloc(h, d, &ws.flags, n1) && dalloc(h, d, &ws.dperm, n1) && dalloc(h, d, &ws.csz, n1);
  // giant plans: giant rows have > 4096 arcs, so there are at most A / 4097 of them; chunks of >= 512
  // arcs over their rows: <= gcap + A / 512; slices of >= 128 slots over tables of < 4 x the arcs:
  // <= gcap + A / 32
  const int64_t gcap = ac / 4096 + 16, scap = gcap + ac / 32 + 16, ccap = gcap + ac / 512 + 16;
  for (GiantPlan* gp : {&ws.gp, &ws.gpv})
    ok = ok && dalloc(h, d, &gp->chunk_off, gcap + 1) && dalloc(h, d, &gp->tab_off, gcap + 1) &&
         dalloc(h, d, &gp->slice_off, gcap + 1) && dalloc(h, d, (int32_t**)&gp->kid, gcap) &&
         dalloc(h, d, &gp->moved, gcap) && dalloc(h, d, &gp->active, gcap) &&
         dalloc(h, d, (long long**)&gp->part_s, scap) &&
         dalloc(h, d, &gp->part_c, scap) && dalloc(h, d, &gp->cowner, ccap) && dalloc(h, d, &gp->sowner, scap);
  for (GiantPlan* gp : {&ws.gp, &ws.gpv}) {
    gp->chunk_cap = ccap;
    gp->slice_cap = scap;
  }
  ok = ok && dalloc(h, d, &ws.glist, gcap);
  ok = ok && dalloc(h, d, &ws.newid, n1 + 1) && dalloc(h, d, &ws.coff, n1 + 1) && dalloc(h, d, &ws.cdeg, n1 + 1) &&
       dalloc(h, d, &ws.len, n1 + 1) && dalloc(h, d, &ws.jrc, n1 + 64) &&
       dalloc(h, d, &ws.tile_tmp, scan_tmp_elems((int64_t)kNumBuckets * n1 + 8) + 8);  // class sort scans 5 n keys
  for (int r = 0; r < 2 && ok; r++)
    ok = dalloc(h, d, &ws.rows[r].hoff, n1 + 1) && dalloc(h, d, &ws.rows[r].hend, n1) &&
         dalloc(h, d, &ws.rows[r].doff, n1 + 1);
  ok = ok && dalloc(h, d, &ws.ctrl, 1);
  if (!ok) {
    free_all(ws.core);
    return set_err(h, LOUVAIN_ERR_OOM, "workspace allocation failed or exceeds the HBM budget");
  }
  // fresh device memory holds whatever its last owner left: the control block starts zeroed (error
  // bits, counters), complete before any stream of the caller's touches it
  if (cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), cudaStreamLegacy) != cudaSuccess ||
      cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
    free_all(ws.core);
    return cuda_err(h, cudaGetLastError(), "control block initialisation");
  }
  ws.n_cap = nc;
  ws.a_cap = ac;
  return ensure_arcs(h, ac);
}

louvain_status ensure_keys(louvain_handle h, int64_t nkeys) {
  Workspace& ws = h->ws;
  if (ws.key_cap >= nkeys) return LOUVAIN_OK;
  free_all(ws.keys_alloc);
  ws.key_cap = 0;
  int64_t cap = nkeys < 4096 ? 4096 : nkeys * 2;
  if (!dalloc(h, ws.keys_alloc, &ws.keyoffs, cap + 1) || !dalloc(h, ws.keys_alloc, &ws.keycur, cap)) {
    free_all(ws.keys_alloc);
    return set_err(h, LOUVAIN_ERR_OOM, "key-offset allocation failed");
  }
  ws.key_cap = cap;
  return ensure_pinned(h, (size_t)(cap + 1) * sizeof(int64_t) + 4096);
}

// Shared pool of global-memory hash tables for the giant rows (all-empty between uses).
louvain_status ensure_pool(louvain_handle h, Ctx& c, int64_t slots) {
  Workspace& ws = h->ws;
  if (slots > ws.gt_slots_total) {
    free_all(ws.gt_alloc);
    ws.gt_slots_total = 0;
    const int64_t total = (slots + slots / 4 + 4096 + 63) / 64 * 64;
    int32_t* kv = nullptr;
    unsigned* bits = nullptr;
    if (!dalloc(h, ws.gt_alloc, &kv, 2 * total) || !dalloc(h, ws.gt_alloc, &bits, total / 32)) {
      free_all(ws.gt_alloc);
      return set_err(h, LOUVAIN_ERR_OOM, "giant hash-table pool allocation failed");
    }
    pool_init(c, kv, total);
    cudaMemsetAsync(bits, 0, (size_t)(total / 32) * 4, c.s);
    ws.pool = kv;
    ws.gt_bits = bits;
    ws.gt_slots_total = total;
  }
  for (GiantPlan* gp : {&ws.gp, &ws.gpv}) {
    gp->slots = ws.pool;
    gp->bits = ws.gt_bits;
    gp->pool_slots = ws.gt_slots_total;
  }
  return LOUVAIN_OK;
}

// Device and pinned buffers for the step records of captured iterations (`words` int64).
louvain_status ensure_desc(louvain_handle h, int64_t words) {
  Workspace& ws = h->ws;
  if (words > ws.desc_cap) {
    const int64_t cap = words < 4096 ? 4096 : 2 * words;
    free_all(ws.desc_alloc);
    ws.desc = nullptr;
    ws.desc_cap = 0;
    if (!dalloc(h, ws.desc_alloc, &ws.desc, cap)) return set_err(h, LOUVAIN_ERR_OOM, "step-record allocation failed");
    ws.desc_cap = cap;
  }
  if (words > h->dpin_cap) {
    // the previous records' copy has completed: the host synchronised since it was enqueued
    if (h->dpin) cudaFreeHost(h->dpin);
    h->dpin = nullptr;
    h->dpin_cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&h->dpin), (size_t)ws.desc_cap * sizeof(int64_t),
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return set_err(h, LOUVAIN_ERR_OOM, "pinned host allocation failed");
    }
    h->dpin_cap = ws.desc_cap;
  }
  return LOUVAIN_OK;
}

// ---- per-launch profile: an event before and after each timed launch on the run's stream
int prof_begin(louvain_handle h, Ctx& c) {
  Profile& P = h->prof;
  if (!P.on) return -1;
  while (P.ev.size() < P.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); P.on = false; return -1; }
    P.ev.push_back(e);
  }
  cudaEventRecord(P.ev[P.used], c.s);
  P.used += 2;
  return (int)(P.used - 2);
}
void prof_end(louvain_handle h, Ctx& c, int cls, int mark) {
  Profile& P = h->prof;
  if (mark < 0 || !P.on) return;
  cudaEventRecord(P.ev[mark + 1], c.s);
  P.recs.push_back({cls, (size_t)mark, (size_t)mark + 1});
}
// After the final synchronisation: device times per class and algorithmic bytes from counters.
void prof_finish(louvain_handle h, const Ctrl& ctrl) {
  Profile& P = h->prof;
  if (!P.on) return;
  for (int k = 0; k < kNumClasses; k++) { P.launches[k] = 0; P.ms[k] = 0.0; P.bytes[k] = 0.0; }
  for (const Profile::Rec& r : P.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[r.e0], P.ev[r.e1]) == cudaSuccess) {
      P.ms[r.cls] += ms;
      P.launches[r.cls]++;
    } else {
      cudaGetLastError();
    }
  }
  for (int b = 0; b < kNumBuckets; b++) {
    const unsigned long long* l = ctrl.lm_stat[b];
    // list entry + flag; per processed vertex row bounds, C'[i], K_i, Sigma_d, flag clear; per arc
    // target, weight, C'[j]; per candidate Sigma_c; per move C' write and two Sigma updates; marks
    P.bytes[kLm0 + b] = 5.0 * l[0] + 37.0 * l[1] + 12.0 * l[2] + 8.0 * l[3] + 20.0 * l[4] + 1.0 * l[5];
    const unsigned long long* m = ctrl.mg_stat[b];
    // per community offsets, total degree, holey offset and end; per member id and row bounds; per
    // arc target, weight, C'[j]; per written super-arc (target, weight)
    P.bytes[kMg0 + b] = 32.0 * m[0] + 20.0 * m[1] + 12.0 * m[2] + 8.0 * m[3];
  }
  P.valid = true;
}

louvain_status sync(louvain_handle h, Ctx& c, const char* where) {
  cudaError_t e = cudaStreamSynchronize(c.s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(h, e, where);
  return LOUVAIN_OK;
}

// Reads `count` int64 from device into the pinned buffer (synchronising) and returns it.
const int64_t* read_i64(louvain_handle h, Ctx& c, const int64_t* d, int64_t count, louvain_status* st,
                        const char* where) {
  *st = ensure_pinned(h, (size_t)count * sizeof(int64_t) + 8192);
  if (*st != LOUVAIN_OK) return nullptr;
  int64_t* p = reinterpret_cast<int64_t*>(h->pin) + 128;  // first 1 KiB reserved for Ctrl copies
  cudaMemcpyAsync(p, d, (size_t)count * sizeof(int64_t), cudaMemcpyDeviceToHost, c.s);
  *st = sync(h, c, where);
  return *st == LOUVAIN_OK ? p : nullptr;
}

const Ctrl* read_ctrl(louvain_handle h, Ctx& c, louvain_status* st, const char* where) {
  *st = ensure_pinned(h, 65536);
  if (*st != LOUVAIN_OK) return nullptr;
  cudaMemcpyAsync(h->pin, h->ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c.s);
  *st = sync(h, c, where);
  return *st == LOUVAIN_OK ? reinterpret_cast<const Ctrl*>(h->pin) : nullptr;
}

cudaEvent_t event_at(louvain_handle h, size_t k) {
  while (h->events.size() <= k) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->events.push_back(e);
  }
  return h->events[k];
}

float elapsed(louvain_handle h, size_t a, size_t b) {
  float ms = 0.f;
  if (a < h->events.size() && b < h->events.size()) cudaEventElapsedTime(&ms, h->events[a], h->events[b]);
  return ms;
}

bool valid_params(const louvain_params* p) {
  return p && p->max_passes >= 0 && p->max_iterations >= 0 && p->tolerance >= 0.0 && p->tolerance_drop > 0.0 &&
         p->aggregation_tolerance >= 0.0 && p->fast_classes >= 0 && p->fast_classes <= 4096 &&
         p->lm_blocks_per_sm >= 0 && p->lm_blocks_per_sm <= 64 && p->fast_classes_later >= 0 &&
         (p->giant_min_degree == 0 || (p->giant_min_degree >= 2048 && p->giant_min_degree <= 4096)) &&
         p->wait_spins >= 0 && (p->host_arcs == 0 || p->host_arcs == 1) &&
         (p->table_factor == 0 || p->table_factor == 1 || p->table_factor == 2 || p->table_factor == 4) &&
         p->fast_sync_small >= 0 && p->fast_sync_small <= 2 &&
         (p->mode == LOUVAIN_MODE_DETERMINISTIC || p->mode == LOUVAIN_MODE_FAST);
}

// Full CSR validation on the device.  Returns OK / INVALID / OVERFLOW.
louvain_status validate_graph(louvain_handle h, Ctx& c, int64_t n, int64_t n_arcs, const int64_t* offs,
                              const int32_t* tg, const void* w, bool fp, bool check_two_m = true) {
  Ctrl* ctrl = h->ws.ctrl;
  validate_reset(c, ctrl);
  validate_offsets(c, n, n_arcs, offs, ctrl);
  louvain_status st;
  const Ctrl* hc = read_ctrl(h, c, &st, "validate offsets");
  if (!hc) return st;
  if (hc->cnt[0]) return set_err(h, LOUVAIN_ERR_INVALID, "offsets are not a monotone CSR offset array ending at n_arcs");
  validate_arcs(c, n, offs, tg, w, fp, ctrl);
  hc = read_ctrl(h, c, &st, "validate arcs");
  if (!hc) return st;
  if (hc->cnt[1]) return set_err(h, LOUVAIN_ERR_INVALID, "arc target outside [0, n)");
  if (hc->cnt[2]) return set_err(h, LOUVAIN_ERR_INVALID, "arc weight not positive (or not finite)");
  if (hc->cnt[3]) return set_err(h, LOUVAIN_ERR_INVALID, "graph is not symmetric (w_ij != w_ji)");
  if (check_two_m && !fp && (unsigned long long)hc->acc_i[0] >= (1ULL << 31))
    return set_err(h, LOUVAIN_ERR_OVERFLOW, "integer mode needs 2m < 2^31");
  return LOUVAIN_OK;
}

// ------------------------------------------------------------------ Algorithm 1 on the device
struct RunOut {
  double q = 0.0;
  int32_t passes = 0, total_iterations = 0;
  int64_t n_communities = 0;
};

// A colouring that did not colour every listed vertex: a grid-barrier wait that ran out (the
// kernel left on every block) is LOUVAIN_ERR_TIMEOUT, anything else an internal error.
louvain_status colour_failure(louvain_handle h, Ctx& c) {
  const unsigned long long* q = h->pin;
  char buf[256];
  snprintf(buf, sizeof buf,
           "colouring did not finish (coloured %llu of %llu after %llu rounds, max colour %llu, guard trips %llu)",
           q[3], q[5], q[6], q[4], q[7]);
  const std::string what = buf;
  louvain_status st;
  const Ctrl* hc = read_ctrl(h, c, &st, "colouring end");
  if (!hc) return st;
  if (hc->error & kErrTimeout)
    return set_err(h, LOUVAIN_ERR_TIMEOUT, "a bounded grid-barrier wait of the colouring ran out: " + what);
  return set_err(h, LOUVAIN_ERR_CUDA, "internal: " + what);
}

// Per-pass degree buckets of graph g into ws.dperm with host offsets hb[kNumBuckets + 1];
// *giant_slots = table slots its giant vertices need.
template <class W>
louvain_status degree_buckets(louvain_handle h, Ctx& c, const GraphView<W>& g, int64_t hb[kNumBuckets + 1],
                              int64_t* giant_slots) {
  Workspace& ws = h->ws;
  louvain_status st = ensure_keys(h, kNumBuckets);
  if (st != LOUVAIN_OK) return st;
  cudaMemsetAsync(&ws.ctrl->gslots, 0, sizeof(unsigned long long), c.s);
  bucket_sort(c, KeyDesc{0, 1, 0, 0}, g.n, g.rbeg, g.rend, nullptr, nullptr, kNumBuckets, ws.dperm, ws.keyoffs,
              ws.keycur, ws.tile_tmp, nullptr, &ws.ctrl->gslots, g.n);
  const int64_t* p = read_i64(h, c, ws.keyoffs, kNumBuckets + 1, &st, "degree buckets");
  if (!p) return st;
  for (int b = 0; b <= kNumBuckets; b++) hb[b] = p[b];
  const Ctrl* hc = read_ctrl(h, c, &st, "degree buckets");
  if (!hc) return st;
  *giant_slots = (int64_t)hc->gslots;
  return LOUVAIN_OK;
}

// One step of a local-moving iteration: the vertices of one colour class (deterministic) or of
// one group of random classes (fast), as perm ranges per degree bucket, the giant range of the
// class-ordered giant list, and (deterministic) the perm range the Sigma apply covers.
struct ClassStep {
  int64_t start[kNumBuckets] = {};
  int64_t count[kNumBuckets] = {};
  int64_t g0 = 0, g1 = 0;
  int64_t apply_start = 0, apply_count = 0;
};

// Upper bound of bucket b's count over the steps, rounded up to a power of two: it sizes the grid of
// a captured launch that reads its count from the step records (the rounding lets later passes and
// runs find the same executable).
int64_t bucket_bound(const std::vector<ClassStep>& steps, int b) {
  int64_t m = 0;
  for (const ClassStep& cs : steps) m = cs.count[b] > m ? cs.count[b] : m;
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}

// Launches one iteration (every step; the convergence test at the end).  With `streams` the
// degree buckets of a step fork to one side stream each and join before the next step (used
// while capturing a CUDA graph); otherwise they run in order on c.s with per-launch profiling.
// With `recs` (the device step records of `steps`) every launch reads its vertex range from device
// memory, so the captured graph serves any pass over the same arrays whose steps launch the same
// kernels; list bases are then ws.perm and gbase (the giant list), and the graph goes in with n = 0
// (the captured kernels do not read it), so that only its arrays tie a graph to a pass.
template <class M>
void enqueue_iteration(louvain_handle h, Ctx& c, const GraphView<typename M::w_t>& g, const PassState<M>& st,
                       const std::vector<ClassStep>& steps, const int32_t* glist, bool det, bool pruning,
                       GraphCtl* gc, int32_t n_graphs, bool streams, const int64_t* recs = nullptr,
                       const int32_t* gbase = nullptr) {
  Workspace& ws = h->ws;
  GraphView<typename M::w_t> gk = g;
  if (recs) gk.n = 0;
  int64_t bound[kNumBuckets] = {};
  if (recs)
    for (int b = 0; b < kNumBuckets - 1; b++) bound[b] = bucket_bound(steps, b);
  for (size_t k = 0; k < steps.size(); k++) {
    const ClassStep& cs = steps[k];
    const int64_t* rk = recs ? recs + k * kStepWords : nullptr;
    if (streams) cudaEventRecord(h->fork_ev[k], c.s);
    for (int b = 0; b < kNumBuckets; b++) {
      const bool giant = b == kNumBuckets - 1;
      const int64_t cnt = giant ? cs.g1 - cs.g0 : cs.count[b];
      if (cnt <= 0) continue;
      if (streams) {
        Ctx cb = c;
        cb.s = h->side[b];
        cb.launches = 0;
        cudaStreamWaitEvent(cb.s, h->fork_ev[k], 0);
        if (!giant)
          move_bucket<M>(cb, b, gk, st, rk ? ws.perm : ws.perm + cs.start[b], rk ? bound[b] : cnt, !det, pruning,
                         rk ? rk + 2 * b : nullptr);
        else
          giant_move<M>(cb, gk, st, rk ? gbase : glist, cs.g0, cs.g1, ws.gp, !det, pruning,
                        rk ? rk + kStepGiant : nullptr);
        c.launches += cb.launches;
        cudaEventRecord(h->join_ev[k * kNumBuckets + b], cb.s);
        cudaStreamWaitEvent(c.s, h->join_ev[k * kNumBuckets + b], 0);
      } else {
        const int pm = prof_begin(h, c);
        if (!giant) move_bucket<M>(c, b, g, st, ws.perm + cs.start[b], cnt, !det, pruning);
        else giant_move<M>(c, g, st, glist, cs.g0, cs.g1, ws.gp, !det, pruning);
        prof_end(h, c, kLm0 + b, pm);
      }
    }
    if (det && cs.apply_count > 0) {
      const int pm = streams ? -1 : prof_begin(h, c);
      move_apply<M>(c, st, rk ? ws.perm : ws.perm + cs.apply_start, cs.apply_count, rk ? rk + kStepApply : nullptr);
      if (!streams) prof_end(h, c, kApply, pm);
    }
  }
  if (gc) batch_finish<M>(c, ws.ctrl, gc, n_graphs);
  else move_finish<M>(c, ws.ctrl);
}

// Everything a captured iteration's launches depend on besides its device step records: the
// kernel instances (mode, schedule, which buckets / giant chains / applies each step launches),
// grid sizes, and every pointer and scalar passed by value.  Equal keys mean equal launches.
template <class M>
std::vector<int64_t> iteration_key(louvain_handle h, const Ctx& c, const GraphView<typename M::w_t>& g,
                                   const PassState<M>& st, const std::vector<ClassStep>& steps, const int64_t* recs,
                                   const int32_t* gbase, bool det, bool pruning, GraphCtl* gc, int32_t n_graphs) {
  static_assert(sizeof(PassState<M>) % 8 == 0 && sizeof(GiantPlan) % 8 == 0, "pointer-only records");
  const Workspace& ws = h->ws;
  std::vector<int64_t> k = {M::is_fp ? 1 : 0, det ? 1 : 0, pruning ? 1 : 0, n_graphs, (int64_t)(intptr_t)gc,
                            c.num_sms, c.lm_blocks_per_sm, c.giant_min, (int64_t)(intptr_t)ws.perm,
                            (int64_t)(intptr_t)gbase, (int64_t)(intptr_t)recs, (int64_t)(intptr_t)ws.desc,
                            (int64_t)(intptr_t)g.rbeg, (int64_t)(intptr_t)g.rend, (int64_t)(intptr_t)g.tg,
                            (int64_t)(intptr_t)g.w, (int64_t)steps.size()};
  const size_t n0 = k.size();
  k.resize(n0 + sizeof(PassState<M>) / 8 + sizeof(GiantPlan) / 8);
  std::memcpy(&k[n0], &st, sizeof(PassState<M>));
  std::memcpy(&k[n0 + sizeof(PassState<M>) / 8], &ws.gp, sizeof(GiantPlan));
  for (int b = 0; b < kNumBuckets - 1; b++) k.push_back(bucket_bound(steps, b));  // grid sizes
  for (const ClassStep& cs : steps) {
    int64_t mask = 0;
    for (int b = 0; b < kNumBuckets - 1; b++)
      if (cs.count[b] > 0) mask |= 1 << b;
    if (cs.g1 > cs.g0) mask |= 1 << (kNumBuckets - 1);
    if (det && cs.apply_count > 0) mask |= 1 << kNumBuckets;
    k.push_back(mask);
  }
  return k;
}

// Host image of the step records of `steps` (kStepWords each; the giant list offset from its base).
void write_step_records(const std::vector<ClassStep>& steps, int64_t goff, int64_t* out) {
  for (size_t k = 0; k < steps.size(); k++) {
    int64_t* r = out + k * kStepWords;
    std::memset(r, 0, sizeof(int64_t) * kStepWords);
    const ClassStep& cs = steps[k];
    for (int b = 0; b < kNumBuckets - 1; b++) {
      r[2 * b] = cs.start[b];
      r[2 * b + 1] = cs.count[b];
    }
    r[kStepGiant] = goff;
    r[kStepGiant + 1] = cs.g0;
    r[kStepGiant + 2] = cs.g1;
    r[kStepApply] = cs.apply_start;
    r[kStepApply + 1] = cs.apply_count;
  }
}

// The cached executable with exactly this key, or null.
louvain_handle_s::CachedExec* find_exec(louvain_handle h, const std::vector<int64_t>& key) {
  for (auto& x : h->execs)
    if (x.key == key) {
      x.used = ++h->exec_clock;
      x.call = h->call_seq;
      return &x;
    }
  return nullptr;
}

// Captures one iteration into an executable CUDA graph owned by the handle's cache (launches
// recorded on a private stream, the graph runs on the caller's).  *launches = kernels per replay.
template <class M>
louvain_status capture_iteration(louvain_handle h, Ctx& c0, const GraphView<typename M::w_t>& g, const PassState<M>& st,
                                 const std::vector<ClassStep>& steps, const int32_t* glist, bool det, bool pruning,
                                 GraphCtl* gc, int32_t n_graphs, cudaGraphExec_t exclude, cudaGraphExec_t* exec,
                                 int64_t* launches, int32_t* instantiated, const int64_t* recs,
                                 const int32_t* gbase, const std::vector<int64_t>& key) {
  *exec = nullptr;
  if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_err(h, cudaGetLastError(), "capture stream creation");
  Ctx c = c0;
  c.s = h->cap;
  c.launches = 0;
  for (int b = 0; b < kNumBuckets; b++)
    if (!h->side[b] && cudaStreamCreateWithFlags(&h->side[b], cudaStreamNonBlocking) != cudaSuccess)
      return cuda_err(h, cudaGetLastError(), "side stream creation");
  while (h->fork_ev.size() < steps.size()) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return cuda_err(h, cudaGetLastError(), "event creation");
    h->fork_ev.push_back(e);
  }
  while (h->join_ev.size() < steps.size() * kNumBuckets) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return cuda_err(h, cudaGetLastError(), "event creation");
    h->join_ev.push_back(e);
  }
  move_prepare();
  cudaError_t e = cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_err(h, e, "graph capture begin");
  enqueue_iteration<M>(h, c, g, st, steps, glist, det, pruning, gc, n_graphs, true, recs, gbase);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(c.s, &graph);
  *launches = c.launches;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_err(h, e, "graph capture end");
  }
  // A miss updates, in place, an executable of the same node count that no phase of this API call
  // has used (one from an earlier graph: a new graph's keys never repeat, and an update costs ~0.1
  // ms against ~2.6 ms for an instantiation), least recently used first.  Executables of this call
  // are kept, so the passes of a graph that is run again all hit; when every candidate belongs to
  // this call the graph gets an executable of its own while the cache has room, and a full cache
  // updates its least recently used one of the same node count.  `exclude` (the other graph of
  // this phase) is never touched; all work launched from the others has completed (the host
  // synchronised on the class offsets before this capture).
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  auto lru_first = [&](std::vector<size_t>& v) {
    std::sort(v.begin(), v.end(), [&](size_t a, size_t b) { return h->execs[a].used < h->execs[b].used; });
  };
  std::vector<size_t> stale, any;
  for (size_t k = 0; k < h->execs.size(); k++)
    if (h->execs[k].nodes == nodes && h->execs[k].e != exclude) {
      any.push_back(k);
      if (h->execs[k].call != h->call_seq) stale.push_back(k);
    }
  lru_first(stale);
  lru_first(any);
  std::vector<size_t> cand = stale;
  if (cand.empty() && h->execs.size() >= kExecCache) cand = any;
  for (size_t k : cand) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(h->execs[k].e, graph, &info) == cudaSuccess) {
      h->execs[k].used = ++h->exec_clock;
      h->execs[k].call = h->call_seq;
      h->execs[k].launches = *launches;
      h->execs[k].key = key;
      *exec = h->execs[k].e;
      cudaGraphDestroy(graph);
      return LOUVAIN_OK;
    }
    cudaGetLastError();  // a topology mismatch is not an error of the run
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return cuda_err(h, e, "graph instantiation");
  }
  ++*instantiated;
  if (h->execs.size() >= kExecCache) {
    size_t lru = h->execs.size();
    for (size_t k = 0; k < h->execs.size(); k++)
      if (h->execs[k].e != exclude && (lru == h->execs.size() || h->execs[k].used < h->execs[lru].used)) lru = k;
    cudaGraphExecDestroy(h->execs[lru].e);
    h->execs.erase(h->execs.begin() + (std::ptrdiff_t)lru);
  }
  h->execs.push_back({*exec, nodes, ++h->exec_clock, *launches, key, h->call_seq});
  return LOUVAIN_OK;
}

// One local-moving phase (Algorithm 2) on g from the state in ws (K, Sig, Cp, flags set).
// Fills *li and *moves.  Deterministic mode colours g first.
template <class M>
louvain_status local_move_phase(louvain_handle h, Ctx& c, const GraphView<typename M::w_t>& g, const int64_t hb[],
                                int64_t giant_slots, const louvain_params& p, int32_t pass, double tau, int32_t* li,
                                int64_t* moves, size_t ev_colour_done, GraphCtl* gc = nullptr,
                                const int32_t* vg = nullptr, int32_t n_graphs = 0, int32_t* colours = nullptr,
                                int32_t* colour_rounds = nullptr, float* ms_graph = nullptr,
                                int32_t* graphs_new = nullptr) {
  Workspace& ws = h->ws;
  PassState<M> st{reinterpret_cast<typename M::a_t*>(ws.K), reinterpret_cast<typename M::a_t*>(ws.Sig), ws.Cp,
                  ws.flags, ws.csize, ws.mv_from, ws.mv_to, ws.ctrl};
  st.gc = gc;
  st.vg = vg;
  Segs seg;
  seg.vg = vg;
  seg.gc = gc;
  // Fast mode on an input graph that the GPU holds in flight (a batch: its mean graph) and whose
  // rows over 512 arcs hold at most a fifth of its arcs runs the colour-synchronous schedule in
  // every pass: there every class is one wave either way, and asynchronous waves left 2-3% of small
  // planted-partition graphs 0.03-0.066 below the oracle (random classes and colour classes alike).
  // A graph carried by hubs needs hundreds of colours (a class step each; R-MAT scale 17: ~300), and
  // asynchronous waves hold the bar there.  The first phase of the call decides for all: the late
  // super-vertex graphs of a large input are few vertices with long rows (SBM, 4.9M vertices: pass
  // 5 has 108k vertices of 238 arcs), which colour-synchronous moves cost 62 colours a sweep.
  const int64_t n_eff = gc && n_graphs > 0 ? g.n / n_graphs : g.n;
  const int64_t window = (int64_t)c.num_sms * kInFlightPerSm;
  louvain_status s;
  bool det = p.mode == LOUVAIN_MODE_DETERMINISTIC || p.fast_sync_small == 2;
  if (!det && p.fast_sync_small == 0) {
    if (c.fast_sync < 0) {
      c.fast_sync = 0;
      if (n_eff <= window) {
        hub_share(c, g, ws.ctrl);
        const Ctrl* hs = read_ctrl(h, c, &s, "hub share");
        if (!hs) return s;
        c.fast_sync = hs->hub_arcs * 5 <= hs->all_arcs ? 1 : 0;
      }
    }
    det = c.fast_sync == 1;
  }
  if (p.lm_blocks_per_sm > 0) c.lm_blocks_per_sm = p.lm_blocks_per_sm;
  std::vector<int64_t> ho;  // bucket-sort offsets: colour-major (deterministic) or bucket-major (fast)
  int32_t ncol = 1;
  if (det) {
    GraphView<int32_t> gs{g.n, g.rbeg, g.rend, g.tg, nullptr};
    JpBuffers jb{ws.jcnt, ws.jl0, ws.jl1, ws.n_cap + 1, ws.jrc, ws.jbc, ws.jbig, ws.jbcb, ws.jcown, ws.jchunk_cap,
                 ws.jcc, ws.jboff, ws.jused, ws.jused_cap, ws.jround, ws.tile_tmp};
    if ((s = ensure_pinned(h, 65536)) != LOUVAIN_OK) return s;
    cudaError_t ce;
    const int pm = prof_begin(h, c);
    int64_t rounds = 0;
    ncol = jp_colour(c, gs, ws.dperm, hb, p.seed, pass, ws.colour, jb, ws.ctrl, h->pin, &ce, seg, &rounds);
    prof_end(h, c, kColour, pm);
    if (ce != cudaSuccess) return cuda_err(h, ce, "colouring");
    if (ncol < 0) return colour_failure(h, c);
    if (colours) *colours = ncol;
    if (colour_rounds) *colour_rounds = (int32_t)rounds;
    const int64_t nkeys = (int64_t)ncol * kNumBuckets;
    if ((s = ensure_keys(h, nkeys)) != LOUVAIN_OK) return s;
    bucket_sort(c, KeyDesc{1, 1, 0, 0}, g.n, g.rbeg, g.rend, ws.colour, nullptr, nkeys, ws.perm, ws.keyoffs, ws.keycur, ws.tile_tmp,
                nullptr);
    const int64_t* q = read_i64(h, c, ws.keyoffs, nkeys + 1, &s, "class buckets");
    if (!q) return s;
    ho.assign(q, q + nkeys + 1);
  } else {
    // fast schedule: random vertex classes processed one after another, asynchronous inside a class;
    // keys bucket-major, so a bucket's vertices of consecutive classes are one contiguous range
    ncol = p.fast_classes > 0 ? p.fast_classes : 1;
    const int64_t nkeys = (int64_t)ncol * kNumBuckets;
    if ((s = ensure_keys(h, nkeys)) != LOUVAIN_OK) return s;
    KeyDesc kd{3, ncol, pass, p.seed ^ 0x46A57C1A55E5ULL};
    kd.seg = seg;
    // giant rows all in one class per pass (one giant pipeline per iteration instead of one per class)
    if (p.fast_giant_class) kd.giant_class = (int)(hash3(p.seed, (uint64_t)pass, 0x6A09E667ULL) % (uint64_t)ncol);
    bucket_sort(c, kd, g.n, g.rbeg, g.rend, nullptr, nullptr, nkeys, ws.perm, ws.keyoffs, ws.keycur, ws.tile_tmp,
                nullptr);
    const int64_t* q = read_i64(h, c, ws.keyoffs, nkeys + 1, &s, "fast classes");
    if (!q) return s;
    ho.assign(q, q + nkeys + 1);
  }
  if (event_at(h, ev_colour_done)) cudaEventRecord(h->events[ev_colour_done], c.s);
  // giant vertices of every class in one class-ordered list and one plan for the whole pass (each
  // giant owns a table of the pool; the scans leave every table empty)
  std::vector<int64_t> gofs((size_t)ncol + 1, 0);
  const int32_t* glist = ws.glist;
  if (det) {
    for (int cl = 0; cl < ncol; cl++) {
      const size_t base = (size_t)cl * kNumBuckets;
      const int64_t cnt = ho[base + kNumBuckets] - ho[base + kNumBuckets - 1];
      if (cnt > 0)
        cudaMemcpyAsync(ws.glist + gofs[cl], ws.perm + ho[base + kNumBuckets - 1], (size_t)cnt * sizeof(int32_t),
                        cudaMemcpyDeviceToDevice, c.s);
      gofs[cl + 1] = gofs[cl] + (cnt > 0 ? cnt : 0);
    }
  } else {
    const size_t gb = (size_t)(kNumBuckets - 1) * ncol;  // the giants of all classes, in class order
    glist = ws.perm + ho[gb];
    for (int cl = 0; cl <= ncol; cl++) gofs[cl] = ho[gb + cl] - ho[gb];
  }
  if (giant_slots > 0 && (s = ensure_pool(h, c, giant_slots)) != LOUVAIN_OK) return s;
  if (gofs[ncol] > 0) giant_move_plan<M>(c, g, glist, gofs[ncol], ws.gp, ws.ctrl);
  // the steps of an iteration: every class on its own; in fast mode the iterations after the first
  // may merge consecutive classes into groups (fewer, larger launches once most vertices are pruned)
  auto make_steps = [&](int group) {
    std::vector<ClassStep> v;
    for (int c0 = 0; c0 < ncol; c0 += group) {
      const int c1 = c0 + group < ncol ? c0 + group : ncol;
      ClassStep cs;
      for (int b = 0; b < kNumBuckets - 1; b++) {
        if (det) {
          cs.start[b] = ho[(size_t)c0 * kNumBuckets + b];
          cs.count[b] = ho[(size_t)c0 * kNumBuckets + b + 1] - cs.start[b];
        } else {
          cs.start[b] = ho[(size_t)b * ncol + c0];
          cs.count[b] = ho[(size_t)b * ncol + c1] - cs.start[b];
        }
      }
      cs.g0 = gofs[c0];
      cs.g1 = gofs[c1];
      if (det) {
        cs.apply_start = ho[(size_t)c0 * kNumBuckets];
        cs.apply_count = ho[(size_t)c0 * kNumBuckets + kNumBuckets] - cs.apply_start;
      }
      v.push_back(cs);
    }
    return v;
  };
  // Grouping keeps the share of vertices that decide at the same time at or below one class's
  // (1/fast_classes) only where a group is much larger than what the GPU holds in flight
  // (kInFlightPerSm vertices per SM); a small graph sits wholly in flight, so there each class stays
  // on its own.  A batch counts by its mean graph, as moves never cross graphs.
  int later = ncol;
  if (!det && p.fast_classes_later > 0 && p.fast_classes_later < ncol) {
    const int64_t need = n_eff > 0 ? ((int64_t)ncol * window + n_eff - 1) / n_eff : ncol;
    later = (int)std::min<int64_t>(ncol, std::max<int64_t>(p.fast_classes_later, need));
  }
  const std::vector<ClassStep> first = make_steps(1);
  const std::vector<ClassStep> rest = later == ncol ? first : make_steps((ncol + later - 1) / later);
  move_setup(c, ws.ctrl, tau, p.max_iterations);
  if (gc) batch_move_setup(c, gc, n_graphs, p.max_iterations);
  const bool pruning = p.pruning != 0;
  int enq = 0;
  const int batch = det ? 2 : 4;
  // Without per-launch profiling an iteration runs as a CUDA graph -- per step a fork to one stream
  // per degree bucket and a join -- whose launches read their vertex ranges from the step records
  // copied here; a cached executable with the same key serves again with no capture.
  cudaGraphExec_t g_first = nullptr, g_rest = nullptr;
  int64_t l_first = 0, l_rest = 0;
  const bool graphs = !h->prof.on && h->use_graphs;
  int32_t n_new = 0;
  double host_ms = 0.0;
  auto now = [] { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count(); };
  double t0 = now();
  const int32_t* gbase = det ? ws.glist : ws.perm;  // giant lists: ws.glist (deterministic) or inside perm
  const int64_t* recs_first = nullptr;
  const int64_t* recs_rest = nullptr;
  std::vector<int64_t> key_rest;
  if (graphs) {
    const int64_t words = (int64_t)(first.size() + rest.size()) * kStepWords;
    if ((s = ensure_desc(h, words)) != LOUVAIN_OK) return s;
    int64_t* hp = h->dpin;
    const int64_t goff = glist - gbase;
    write_step_records(first, goff, hp);
    write_step_records(rest, goff, hp + first.size() * kStepWords);
    cudaMemcpyAsync(ws.desc, hp, (size_t)words * sizeof(int64_t), cudaMemcpyHostToDevice, c.s);
    recs_first = ws.desc;
    recs_rest = ws.desc + first.size() * kStepWords;
    const std::vector<int64_t> key =
        iteration_key<M>(h, c, g, st, first, recs_first, gbase, det, pruning, gc, n_graphs);
    if (auto* x = find_exec(h, key)) {
      g_first = x->e;
      l_first = x->launches;
    } else {
      if ((s = capture_iteration<M>(h, c, g, st, first, glist, det, pruning, gc, n_graphs, nullptr, &g_first, &l_first,
                                    &n_new, recs_first, gbase, key)) != LOUVAIN_OK)
        return s;
    }
    if (rest.size() != first.size())
      key_rest = iteration_key<M>(h, c, g, st, rest, recs_rest, gbase, det, pruning, gc, n_graphs);
  }
  host_ms += now() - t0;
  while (true) {
    for (int k = 0; k < batch && enq < p.max_iterations; k++, enq++) {
      const bool is_first = enq == 0 || rest.size() == first.size();
      if (graphs && !is_first && !g_rest) {  // found or captured while the first iteration runs
        t0 = now();
        if (auto* x = find_exec(h, key_rest)) {
          g_rest = x->e;
          l_rest = x->launches;
        } else if ((s = capture_iteration<M>(h, c, g, st, rest, glist, det, pruning, gc, n_graphs, g_first, &g_rest,
                                             &l_rest, &n_new, recs_rest, gbase, key_rest)) != LOUVAIN_OK) {
          return s;
        }
        host_ms += now() - t0;
      }
      const cudaGraphExec_t ex = is_first ? g_first : g_rest;
      if (ex) {
        cudaGraphLaunch(ex, c.s);
        c.launches += is_first ? l_first : l_rest;
        continue;
      }
      enqueue_iteration<M>(h, c, g, st, is_first ? first : rest, glist, det, pruning, gc, n_graphs, false);
    }
    const Ctrl* hc = read_ctrl(h, c, &s, "local move");
    if (!hc) return s;
    if (hc->error) return set_err(h, LOUVAIN_ERR_CUDA, "internal: hash table overflow in the local-moving phase");
    if (hc->done || enq >= p.max_iterations) {
      *li = hc->iterations;
      *moves = (int64_t)hc->moves_pass;
      if (ms_graph) *ms_graph = (float)host_ms;
      if (graphs_new) *graphs_new = n_new;
      return LOUVAIN_OK;
    }
  }
}

template <class M>
louvain_status aggregate_phase(louvain_handle h, Ctx& c, const GraphView<typename M::w_t>& g, const int64_t* hb,
                               int64_t nc, RowSet& rs, int32_t* otg_holey, typename M::w_t* ow_holey,
                               int64_t* cb_out) {
  Workspace& ws = h->ws;
  louvain_status s;
  // community-vertex CSR (countCommunityVertices, exclusiveScan, atomic fill)
  cudaMemsetAsync(ws.counts, 0, (size_t)nc * sizeof(int32_t), c.s);
  cudaMemsetAsync(ws.cdeg, 0, (size_t)nc * sizeof(int64_t), c.s);
  community_count(c, ws.Cp, g.rbeg, g.rend, g.n, ws.counts, ws.cdeg);
  scan_exclusive_i32(c, ws.counts, ws.coff, nc, ws.tile_tmp);
  cudaMemsetAsync(ws.cursor, 0, (size_t)nc * sizeof(int32_t), c.s);
  community_fill(c, ws.Cp, g.n, ws.coff, ws.cursor, ws.cverts);
  // holey offsets (communityTotalDegree, exclusiveScan)
  scan_exclusive_i64(c, ws.cdeg, rs.hoff, nc, ws.tile_tmp);
  cudaMemcpyAsync(rs.hend, rs.hoff, (size_t)nc * sizeof(int64_t), cudaMemcpyDeviceToDevice, c.s);
  // communities by total-degree bucket
  if ((s = ensure_keys(h, kNumBuckets)) != LOUVAIN_OK) return s;
  cudaMemsetAsync(&ws.ctrl->gslots, 0, sizeof(unsigned long long), c.s);
  bucket_sort(c, KeyDesc{2, 1, 0, 0}, nc, nullptr, nullptr, nullptr, ws.cdeg, kNumBuckets, ws.cperm, ws.keyoffs,
              ws.keycur, ws.tile_tmp, nullptr, &ws.ctrl->gslots, nc);
  const int64_t* q = read_i64(h, c, ws.keyoffs, kNumBuckets + 1, &s, "community buckets");
  if (!q) return s;
  int64_t cb[kNumBuckets + 1];
  for (int b = 0; b <= kNumBuckets; b++) cb[b] = cb_out[b] = q[b];
  const Ctrl* hc = read_ctrl(h, c, &s, "community buckets");
  if (!hc) return s;
  const int64_t giant_slots = (int64_t)hc->gslots;
  if (giant_slots > 0 && (s = ensure_pool(h, c, giant_slots)) != LOUVAIN_OK) return s;
  MergeArgs<M> a;
  a.g = g; a.Cp = ws.Cp; a.coff = ws.coff; a.cverts = ws.cverts; a.cdeg = ws.cdeg; a.hoff = rs.hoff; a.hend = rs.hend;
  a.otg = otg_holey; a.ow = ow_holey; a.nc = nc; a.ctrl = ws.ctrl;
  a.tf = c.table_factor;
  for (int b = 0; b < kNumBuckets; b++) {
    if (cb[b + 1] - cb[b] <= 0) continue;
    const int pm = prof_begin(h, c);
    if (b < kNumBuckets - 1) merge_bucket<M>(c, b, a, ws.cperm + cb[b], cb[b + 1] - cb[b]);
    else giant_merge<M>(c, a, ws.cperm + cb[b], cb[b + 1] - cb[b], ws.csz, ws.gp, reinterpret_cast<int64_t*>(ws.tot),
                        ws.len, ws.tile_tmp);
    prof_end(h, c, kMg0 + b, pm);
  }
  return LOUVAIN_OK;
}

template <class M>
louvain_status run_impl(louvain_handle h, Ctx& c, int64_t n, int64_t n_arcs, const int64_t* offs, const int32_t* tg,
                        const typename M::w_t* w, const louvain_params& p, int32_t* C, RunOut* out,
                        louvain_pass_stats* stats, int32_t stats_cap, int32_t* n_stats, const int32_t* init) {
  typedef typename M::a_t A;
  typedef typename M::w_t W;
  Workspace& ws = h->ws;
  louvain_status s;
  if (n_stats) *n_stats = 0;
  iota_i32(c, C, n);
  GraphView<W> g0{n, offs, offs + 1, tg, w};
  GraphView<W> g = g0;
  PassState<M> st{reinterpret_cast<A*>(ws.K), reinterpret_cast<A*>(ws.Sig), ws.Cp, ws.flags, ws.csize, ws.mv_from,
                  ws.mv_to, ws.ctrl};
  cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), c.s);
  double tau = p.tolerance;
  bool pending = false, q_done = false;
  int64_t g_arcs = n_arcs;
  for (int32_t lp = 0; lp < p.max_passes; lp++) {
    const size_t e0 = (size_t)lp * 6 + 1;
    if (event_at(h, e0 + 5) == nullptr) return set_err(h, LOUVAIN_ERR_CUDA, "event creation failed");
    cudaEventRecord(h->events[e0], c.s);
    const int64_t n_cur = g.n;
    // (a1) pass init: buckets, K' / Sigma' / C' / flags
    int64_t hb[kNumBuckets + 1], gslots = 0;
    if ((s = degree_buckets(h, c, g, hb, &gslots)) != LOUVAIN_OK) return s;
    if (lp == 0) {
      vertex_init<M>(c, st, n_cur, false);
      row_sums<M>(c, g, ws.dperm, hb, st.K, st.Sig, reinterpret_cast<A*>(ws.K0));
      total_weight<M>(c, st.K, n_cur, ws.ctrl);
      const Ctrl* hc = read_ctrl(h, c, &s, "pass init");
      if (!hc) return s;
      if (!M::is_fp && hc->two_m_i >= (1LL << 31))
        return set_err(h, LOUVAIN_ERR_OVERFLOW, "integer mode needs 2m < 2^31");
      if (init) warm_init<M>(c, st, init, n_cur);  // a warm start: pass 0 from the given membership
    } else {
      vertex_init<M>(c, st, n_cur, true);
    }
    cudaEventRecord(h->events[e0 + 1], c.s);
    // (a2-a5) local-moving phase
    int32_t li = 0;
    int64_t moves = 0;
    int32_t ncolours = 0, nrounds = 0, ngraphs = 0;
    float gms = 0.f;
    if ((s = local_move_phase<M>(h, c, g, hb, gslots, p, lp, tau, &li, &moves, e0 + 2, nullptr, nullptr, 0, &ncolours,
                                 &nrounds, &gms, &ngraphs)) != LOUVAIN_OK)
      return s;
    cudaEventRecord(h->events[e0 + 3], c.s);
    pending = true;
    out->passes = lp + 1;
    out->total_iterations += li;
    // communities after the local-moving phase
    mark_occupied(c, ws.Cp, n_cur, ws.occ, n_cur);
    scan_exclusive_i32(c, ws.occ, ws.newid, n_cur, ws.tile_tmp);
    const int64_t* q = read_i64(h, c, ws.newid + n_cur, 1, &s, "community count");
    if (!q) return s;
    const int64_t nc = q[0];
    double pass_q = __builtin_nan("");
    if (p.pass_modularity) {
      modularity<M>(c, g, ws.Cp, reinterpret_cast<A*>(ws.tot), ws.ctrl);
      const Ctrl* hc = read_ctrl(h, c, &s, "pass modularity");
      if (!hc) return s;
      pass_q = hc->q;
    }
    louvain_pass_stats* ps = (stats && lp < stats_cap) ? &stats[lp] : nullptr;
    if (ps) {
      ps->pass = lp; ps->iterations = li; ps->moves = moves; ps->n_vertices = n_cur; ps->n_arcs = g_arcs;
      ps->n_communities = nc; ps->modularity = pass_q;
      ps->colours = ncolours; ps->colour_rounds = nrounds;
      ps->ms_graph = gms; ps->graphs_instantiated = ngraphs;
      if (n_stats) *n_stats = lp + 1;
    }
    const bool stop = li <= 1 || (double)nc / (double)n_cur > p.aggregation_tolerance;
    if (!M::is_fp && (stop || lp + 1 == p.max_passes)) {
      // (a10) Eq. 1 of the returned membership, evaluated on this pass's graph and communities: the
      // aggregation keeps every community's internal weight and total (R1), so with integer weights
      // (exact super-arc sums) Q(G', C') has the same int64 numerator and denominator as Q on the
      // input graph of the membership C' maps to, and this pass's degree-bucket lists serve as they
      // are.  fp32 super-arc weights are rounded sums, so fp32 graphs are evaluated on the input.
      const int pm = prof_begin(h, c);
      modularity_bucketed<M>(c, g, ws.Cp, reinterpret_cast<A*>(ws.tot), ws.ctrl, ws.dperm, hb, ws.gpv);
      prof_end(h, c, kModularity, pm);
      q_done = true;
    }
    if (!stop) {
      // (a6) renumber C', dendrogram lookup, K of the next pass = Sigma by new id
      relabel(c, ws.Cp, n_cur, ws.newid);
      dendrogram_lookup(c, C, n, ws.Cp);
      pending = false;
      gather_totals<A>(c, st.Sig, ws.occ, ws.newid, n_cur, st.K);
      cudaEventRecord(h->events[e0 + 4], c.s);
      // (a7-a9) aggregation
      RowSet& rs = ws.rows[lp & 1];
      int32_t* htg = ws.tgA;
      W* hw = reinterpret_cast<W*>(ws.wA);
      if (!p.compact && (lp & 1)) { htg = ws.tgB; hw = reinterpret_cast<W*>(ws.wB); }
      int64_t cb[kNumBuckets + 1];
      if ((s = aggregate_phase<M>(h, c, g, hb, nc, rs, htg, hw, cb)) != LOUVAIN_OK) return s;
      if (p.compact) {
        row_lengths(c, nc, rs.hoff, rs.hend, ws.len);
        scan_exclusive_i64(c, ws.len, rs.doff, nc, ws.tile_tmp);
        const int pm = prof_begin(h, c);
        compact_bucketed<W>(c, ws.cperm, cb, rs.hoff, rs.hend, rs.doff, htg, hw, ws.tgB, reinterpret_cast<W*>(ws.wB),
                            ws.gpv, ws.ctrl);
        prof_end(h, c, kCompact, pm);
        g = GraphView<W>{nc, rs.doff, rs.doff + 1, ws.tgB, reinterpret_cast<W*>(ws.wB)};
        const int64_t* t = read_i64(h, c, rs.doff + nc, 1, &s, "compaction");
        if (!t) return s;
        g_arcs = t[0];
      } else {
        g = GraphView<W>{nc, rs.hoff, rs.hend, htg, hw};
        g_arcs = -1;
      }
      cudaEventRecord(h->events[e0 + 5], c.s);
      tau /= p.tolerance_drop;
    } else {
      cudaEventRecord(h->events[e0 + 4], c.s);
      cudaEventRecord(h->events[e0 + 5], c.s);
    }
    if (ps) {
      // event times become available after the final synchronisation below
      ps->ms_other = 0.f;
    }
    if (stop) break;
  }
  if (pending) dendrogram_lookup(c, C, n, ws.Cp);
  // canonical ids: rank of each occupied community id
  mark_occupied(c, C, n, ws.occ, g.n);
  scan_exclusive_i32(c, ws.occ, ws.newid, g.n, ws.tile_tmp);
  relabel(c, C, n, ws.newid);
  if (!q_done) {
    // (a10) fp32 weights, or no pass ran: Eq. 1 on the input graph
    const int pm = prof_begin(h, c);
    int64_t hb0[kNumBuckets + 1], gs0 = 0;
    if ((s = degree_buckets(h, c, g0, hb0, &gs0)) != LOUVAIN_OK) return s;
    modularity_bucketed<M>(c, g0, C, reinterpret_cast<A*>(ws.tot), ws.ctrl, ws.dperm, hb0, ws.gpv);
    prof_end(h, c, kModularity, pm);
  }
  const Ctrl* hc = read_ctrl(h, c, &s, "final modularity");
  if (!hc) return s;
  if (hc->error) return set_err(h, LOUVAIN_ERR_CUDA, "internal: hash table overflow");
  prof_finish(h, *hc);
  out->q = hc->q;
  const int64_t* q = read_i64(h, c, ws.newid + g.n, 1, &s, "final communities");
  if (!q) return s;
  out->n_communities = q[0];
  if (stats) {
    for (int32_t lp = 0; lp < out->passes && lp < stats_cap; lp++) {
      const size_t e0 = (size_t)lp * 6 + 1;
      stats[lp].ms_other = elapsed(h, e0, e0 + 1) + elapsed(h, e0 + 3, e0 + 4);
      stats[lp].ms_colour = elapsed(h, e0 + 1, e0 + 2);
      stats[lp].ms_move = elapsed(h, e0 + 2, e0 + 3);
      stats[lp].ms_aggregate = elapsed(h, e0 + 4, e0 + 5);
    }
  }
  return LOUVAIN_OK;
}

louvain_status ensure_batch(louvain_handle h, int64_t G, int64_t n, int64_t a) {
  Workspace& ws = h->ws;
  if (ws.b_graphs >= G && ws.b_n >= n && ws.b_a >= a && ws.gc) return LOUVAIN_OK;
  const int64_t gc_ = G > ws.b_graphs ? G : ws.b_graphs, nc = n > ws.b_n ? n : ws.b_n, ac = a > ws.b_a ? a : ws.b_a;
  free_all(ws.batch_alloc);
  ws.b_graphs = ws.b_n = ws.b_a = -1;
  DevAlloc& d = ws.batch_alloc;
  bool ok = dalloc(h, d, &ws.gc, gc_) && dalloc(h, d, &ws.vo, gc_ + 1) && dalloc(h, d, &ws.ao, gc_ + 1) &&
            dalloc(h, d, &ws.vg0, nc + 1) && dalloc(h, d, &ws.vgA, nc + 1) && dalloc(h, d, &ws.vgB, nc + 1) &&
            dalloc(h, d, &ws.tgU, ac);
  if (!ok) {
    free_all(ws.batch_alloc);
    return set_err(h, LOUVAIN_ERR_OOM, "batch workspace allocation failed or exceeds the HBM budget");
  }
  ws.b_graphs = gc_; ws.b_n = nc; ws.b_a = ac;
  return LOUVAIN_OK;
}

// Algorithm 1 over a batch of graphs as one union graph (batch.cu holds the per-graph steps).
// The pass loop runs until every graph has stopped; each launch covers all graphs still in it.
template <class M>
louvain_status run_batch_impl(louvain_handle h, Ctx& c, int32_t G, int64_t n, int64_t n_arcs, const int64_t* offs,
                              const typename M::w_t* w, const louvain_params& p, int32_t* C, int32_t* passes_out) {
  typedef typename M::a_t A;
  typedef typename M::w_t W;
  Workspace& ws = h->ws;
  louvain_status s;
  iota_i32(c, C, n);
  GraphView<W> g0{n, offs, offs + 1, ws.tgU, w};
  GraphView<W> g = g0;
  PassState<M> st{reinterpret_cast<A*>(ws.K), reinterpret_cast<A*>(ws.Sig), ws.Cp, ws.flags, ws.csize, ws.mv_from,
                  ws.mv_to, ws.ctrl};
  cudaMemcpyAsync(ws.vgA, ws.vg0, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.s);
  int32_t* vg = ws.vgA;
  int32_t* vg_next = ws.vgB;
  double tau = p.tolerance;
  int32_t passes = 0;
  for (int32_t lp = 0; lp < p.max_passes && g.n > 0; lp++) {
    const int64_t n_cur = g.n;
    int64_t hb[kNumBuckets + 1], gslots = 0;
    if ((s = degree_buckets(h, c, g, hb, &gslots)) != LOUVAIN_OK) return s;
    if (lp == 0) {
      vertex_init<M>(c, st, n_cur, false);
      row_sums<M>(c, g, ws.dperm, hb, st.K, st.Sig, reinterpret_cast<A*>(ws.K0));
      batch_two_m<M>(c, ws.gc, G, st.K, ws.ctrl);
      const Ctrl* hc = read_ctrl(h, c, &s, "pass init");
      if (!hc) return s;
      if (!M::is_fp && hc->cnt[6]) return set_err(h, LOUVAIN_ERR_OVERFLOW, "integer mode needs 2m < 2^31 per graph");
    } else {
      vertex_init<M>(c, st, n_cur, true);
    }
    int32_t li = 0;
    int64_t moves = 0;
    if ((s = local_move_phase<M>(h, c, g, hb, gslots, p, lp, tau, &li, &moves, 1, ws.gc, vg, G)) != LOUVAIN_OK)
      return s;
    passes = lp + 1;
    // renumbering, pass tests per graph, dendrogram lookup, next level
    mark_occupied(c, ws.Cp, n_cur, ws.occ, n_cur);
    scan_exclusive_i32(c, ws.occ, ws.newid, n_cur, ws.tile_tmp);
    batch_pass_end(c, ws.gc, G, ws.newid, p.aggregation_tolerance, lp + 1 == p.max_passes, ws.ctrl);
    batch_next_level<A>(c, ws.Cp, n_cur, ws.newid, vg, ws.gc, G, C, n, ws.vg0, st.Sig, ws.occ, st.K, vg_next);
    const Ctrl* hc = read_ctrl(h, c, &s, "batch pass end");
    if (!hc) return s;
    const int64_t nc = hc->acc_i[3];
    if (nc == 0) break;
    // aggregation of the continuing graphs (vertices of the others carry Cp < 0 and are skipped)
    RowSet& rs = ws.rows[lp & 1];
    int32_t* htg = ws.tgA;
    W* hw = reinterpret_cast<W*>(ws.wA);
    if (!p.compact && (lp & 1)) { htg = ws.tgB; hw = reinterpret_cast<W*>(ws.wB); }
    int64_t cb[kNumBuckets + 1];
    if ((s = aggregate_phase<M>(h, c, g, hb, nc, rs, htg, hw, cb)) != LOUVAIN_OK) return s;
    if (p.compact) {
      row_lengths(c, nc, rs.hoff, rs.hend, ws.len);
      scan_exclusive_i64(c, ws.len, rs.doff, nc, ws.tile_tmp);
      const int pm = prof_begin(h, c);
      compact_bucketed<W>(c, ws.cperm, cb, rs.hoff, rs.hend, rs.doff, htg, hw, ws.tgB, reinterpret_cast<W*>(ws.wB),
                          ws.gpv, ws.ctrl);
      prof_end(h, c, kCompact, pm);
      g = GraphView<W>{nc, rs.doff, rs.doff + 1, ws.tgB, reinterpret_cast<W*>(ws.wB)};
    } else {
      g = GraphView<W>{nc, rs.hoff, rs.hend, htg, hw};
    }
    int32_t* t = vg; vg = vg_next; vg_next = t;
    tau /= p.tolerance_drop;
  }
  batch_close(c, C, n, ws.vg0, ws.gc, G);
  // (a10) Eq. 1 per graph on the input graphs
  const int pm = prof_begin(h, c);
  int64_t hb0[kNumBuckets + 1], gs0 = 0;
  if ((s = degree_buckets(h, c, g0, hb0, &gs0)) != LOUVAIN_OK) return s;
  batch_modularity<M>(c, g0, C, ws.vg0, ws.gc, G, ws.vo, ws.dperm, hb0, st.Sig, reinterpret_cast<A*>(ws.tot), n);
  prof_end(h, c, kModularity, pm);
  const Ctrl* hc = read_ctrl(h, c, &s, "batch modularity");
  if (!hc) return s;
  if (hc->error) return set_err(h, LOUVAIN_ERR_CUDA, "internal: hash table overflow");
  prof_finish(h, *hc);
  *passes_out = passes;
  return LOUVAIN_OK;
}

louvain_status begin_call(louvain_handle h) {
  if (!h) return LOUVAIN_ERR_INVALID;
  h->err.clear();
  h->call_seq++;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaSetDevice");
  return LOUVAIN_OK;
}

louvain_status check_graph_args(louvain_handle h, int64_t n, int64_t n_arcs, const void* offs, const void* tg,
                                const void* w, louvain_wtype wt) {
  if (n < 0 || n >= 0x7fffffffLL) return set_err(h, LOUVAIN_ERR_INVALID, "n must be in [0, 2^31 - 1)");
  if (n_arcs < 0) return set_err(h, LOUVAIN_ERR_INVALID, "n_arcs must be >= 0");
  if (!offs) return set_err(h, LOUVAIN_ERR_INVALID, "offsets pointer is NULL");
  if (n_arcs > 0 && (!tg || !w)) return set_err(h, LOUVAIN_ERR_INVALID, "targets / weights pointer is NULL");
  if (wt != LOUVAIN_W_INT32 && wt != LOUVAIN_W_FP32) return set_err(h, LOUVAIN_ERR_INVALID, "unknown weight type");
  return LOUVAIN_OK;
}

}  // namespace

// ------------------------------------------------------------------ autotuning
// Candidates of the performance knobs that leave the arithmetic unchanged: the giant-row
// threshold (which kernel takes rows of 2049..4096 arcs), the local-move grid cap and super-graph
// compaction (every combination), then the hash-table sizing (4 slots per key instead of 2) with
// the best of those.  Each is timed by full runs (device time, best of `reps`) after one untimed run
// that builds its iteration graphs and buffers, as a run in steady use finds them; the fastest wins.
template <class RunFn>
static louvain_status autotune_impl(louvain_handle h, const louvain_params* p, int32_t reps, RunFn run,
                                    louvain_params* tuned, float* best_ms) {
  static const int32_t kGiant[] = {4096, 2048};
  static const int32_t kGrid[] = {16, 4};
  static const int32_t kCompact[] = {1, 0};
  louvain_params best = *p;
  float best_t = -1.f;
  auto trial = [&](const louvain_params& q) -> louvain_status {
    float t = -1.f;
    float warm = 0.f;
    louvain_status s0 = run(q, &warm);
    if (s0 != LOUVAIN_OK) return s0;
    for (int32_t r = 0; r < (reps > 0 ? reps : 1); r++) {
      float ms = 0.f;
      louvain_status s = run(q, &ms);
      if (s != LOUVAIN_OK) return s;
      if (t < 0.f || ms < t) t = ms;
    }
    if (best_t < 0.f || t < best_t) { best_t = t; best = q; }
    return LOUVAIN_OK;
  };
  louvain_status s;
  for (int32_t gm : kGiant)
    for (int32_t gr : kGrid)
      for (int32_t cp : kCompact) {
        louvain_params q = *p;
        q.giant_min_degree = gm;
        q.lm_blocks_per_sm = gr;
        q.compact = cp;
        q.table_factor = 2;
        q.profile = 0;
        if ((s = trial(q)) != LOUVAIN_OK) return s;
      }
  louvain_params q4 = best;
  q4.table_factor = 4;
  if ((s = trial(q4)) != LOUVAIN_OK) return s;
  best.profile = p->profile;
  *tuned = best;
  if (best_ms) *best_ms = best_t;
  return LOUVAIN_OK;
}

// ------------------------------------------------------------------ hooks of the serving runtime
namespace lv {
size_t handle_device_bytes(louvain_handle h) { return h ? total_bytes(h->ws) : 0; }
void handle_set_budget(louvain_handle h, size_t bytes) {
  if (h) h->budget = bytes;
}
// Frees every device buffer the handle caches (they are re-allocated on the next call).
void handle_trim(louvain_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  Workspace& ws = h->ws;
  free_all(ws.core);
  free_all(ws.keys_alloc);
  free_all(ws.gt_alloc);
  free_all(ws.in_alloc);
  free_all(ws.batch_alloc);
  free_all(ws.desc_alloc);
  free_all(ws.upd_alloc);
  free_all(ws.arc_alloc);
  ws.upd_words = 0;
  ws.arc_cap = -1;
  ws.tgA = ws.tgB = nullptr;
  ws.wA = ws.wB = nullptr;
  ws.desc = nullptr;
  ws.desc_cap = 0;
  ws.n_cap = ws.a_cap = -1;
  ws.key_cap = 0;
  ws.gt_slots_total = 0;
  ws.in_n = ws.in_a = -1;
  ws.b_graphs = ws.b_n = ws.b_a = -1;
  ws.gc = nullptr;
  ws.ctrl = nullptr;
}
}  // namespace lv

// =====================================================================================
extern "C" {

const char* louvain_status_string(louvain_status s) {
  switch (s) {
    case LOUVAIN_OK: return "LOUVAIN_OK";
    case LOUVAIN_ERR_INVALID: return "LOUVAIN_ERR_INVALID";
    case LOUVAIN_ERR_OOM: return "LOUVAIN_ERR_OOM";
    case LOUVAIN_ERR_OVERFLOW: return "LOUVAIN_ERR_OVERFLOW";
    case LOUVAIN_ERR_TIMEOUT: return "LOUVAIN_ERR_TIMEOUT";
    case LOUVAIN_ERR_CUDA: return "LOUVAIN_ERR_CUDA";
    case LOUVAIN_ERR_BUSY: return "LOUVAIN_ERR_BUSY";
  }
  return "LOUVAIN_UNKNOWN";
}

louvain_status louvain_default_params(louvain_params* p) {
  if (!p) return LOUVAIN_ERR_INVALID;
  std::memset(p, 0, sizeof(*p));
  p->max_passes = 10;
  p->max_iterations = 20;
  p->tolerance = 1e-2;
  p->tolerance_drop = 10.0;
  p->aggregation_tolerance = 0.8;
  p->pruning = 1;
  p->mode = LOUVAIN_MODE_DETERMINISTIC;
  p->seed = 0;
  p->validate = 1;
  p->compact = 1;
  p->pass_modularity = 0;
  p->profile = 0;
  p->fast_classes = 16;
  p->fast_classes_later = 1;
  return LOUVAIN_OK;
}

louvain_status louvain_create(louvain_handle* out, int device, size_t hbm_budget_bytes) {
  if (!out) return LOUVAIN_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  louvain_handle h = new (std::nothrow) louvain_handle_s();
  if (!h) return LOUVAIN_ERR_OOM;
  h->device = device;
  h->budget = hbm_budget_bytes;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0) h->num_sms = sms;
  *out = h;
  return LOUVAIN_OK;
}

void louvain_destroy(louvain_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_all(h->ws.core);
  free_all(h->ws.keys_alloc);
  free_all(h->ws.gt_alloc);
  free_all(h->ws.in_alloc);
  free_all(h->ws.batch_alloc);
  free_all(h->ws.desc_alloc);
  free_all(h->ws.upd_alloc);
  free_all(h->ws.arc_alloc);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->fork_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->join_ev) cudaEventDestroy(e);
  for (cudaStream_t st : h->side)
    if (st) cudaStreamDestroy(st);
  for (auto& x : h->execs) cudaGraphExecDestroy(x.e);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->pin) cudaFreeHost(h->pin);
  if (h->dpin) cudaFreeHost(h->dpin);
  delete h;
}

const char* louvain_last_error(louvain_handle h) { return h ? h->err.c_str() : "invalid handle"; }

louvain_status louvain_workspace_bytes(louvain_handle h, size_t* bytes) {
  if (!h || !bytes) return LOUVAIN_ERR_INVALID;
  *bytes = total_bytes(h->ws);
  return LOUVAIN_OK;
}

louvain_status louvain_inject_alloc_failure(louvain_handle h, int32_t k) {
  if (!h || k < 0) return LOUVAIN_ERR_INVALID;
  h->fail_alloc_in = k;
  return LOUVAIN_OK;
}

louvain_status louvain_run_batch(louvain_handle h, int32_t n_graphs, const int64_t* graph_vtx_offs, int64_t n_arcs,
                                 const int64_t* d_offsets, const int32_t* d_targets, const void* d_weights,
                                 louvain_wtype wtype, const louvain_params* p, void* stream, int32_t* d_membership,
                                 louvain_graph_result* results, louvain_result* res) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if (n_graphs < 0 || (n_graphs > 0 && !graph_vtx_offs))
    return set_err(h, LOUVAIN_ERR_INVALID, "n_graphs < 0 or graph_vtx_offs is NULL");
  if (!valid_params(p)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid louvain_params");
  if (res) std::memset(res, 0, sizeof(*res));
  if (results && n_graphs > 0) std::memset(results, 0, sizeof(*results) * (size_t)n_graphs);
  if (n_graphs == 0) return LOUVAIN_OK;
  if (graph_vtx_offs[0] != 0) return set_err(h, LOUVAIN_ERR_INVALID, "graph_vtx_offs[0] must be 0");
  for (int32_t k = 0; k < n_graphs; k++)
    if (graph_vtx_offs[k + 1] < graph_vtx_offs[k])
      return set_err(h, LOUVAIN_ERR_INVALID, "graph_vtx_offs must be non-decreasing");
  const int64_t n = graph_vtx_offs[n_graphs];
  if ((s = check_graph_args(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (n > 0 && !d_membership) return set_err(h, LOUVAIN_ERR_INVALID, "membership pointer is NULL");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if (p && p->giant_min_degree > 0) c.giant_min = p->giant_min_degree;
  if (p) c.wait_spins = p->wait_spins;
  if (p && p->table_factor > 0) c.table_factor = p->table_factor;
  h->prof.on = p->profile != 0;
  h->arcs_host = p->host_arcs != 0;
  h->prof.used = 0;
  h->prof.recs.clear();
  h->prof.valid = false;
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  if ((s = ensure_batch(h, n_graphs, n, n_arcs)) != LOUVAIN_OK) return s;
  const size_t gbytes = sizeof(GraphCtl) * (size_t)n_graphs;
  if ((s = ensure_pinned(h, gbytes + 65536)) != LOUVAIN_OK) return s;
  if (!event_at(h, 2)) return set_err(h, LOUVAIN_ERR_CUDA, "event creation failed");
  cudaEventRecord(h->events[0], c.s);
  Workspace& ws = h->ws;
  // vertex ranges to the device through the pinned buffer (after the Ctrl area)
  unsigned char* stage = reinterpret_cast<unsigned char*>(h->pin) + 1024;
  std::memcpy(stage, graph_vtx_offs, sizeof(int64_t) * ((size_t)n_graphs + 1));
  cudaMemcpyAsync(ws.vo, stage, sizeof(int64_t) * ((size_t)n_graphs + 1), cudaMemcpyHostToDevice, c.s);
  cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), c.s);
  batch_setup(c, ws.vo, n_graphs, n, d_offsets, n_arcs, d_targets, ws.tgU, ws.ao, ws.vg0, ws.gc, ws.ctrl);
  {
    const Ctrl* hc = read_ctrl(h, c, &s, "batch setup");
    if (!hc) return s;
    if (hc->cnt[1]) return set_err(h, LOUVAIN_ERR_INVALID, "arc target outside its graph's vertex range");
  }
  const bool fp = wtype == LOUVAIN_W_FP32;
  if (p->validate) {
    if ((s = validate_graph(h, c, n, n_arcs, d_offsets, ws.tgU, d_weights, fp, false)) != LOUVAIN_OK) return s;
    cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), c.s);
  }
  int32_t passes = 0;
  if (n > 0) {
    if (fp)
      s = run_batch_impl<FpMode>(h, c, n_graphs, n, n_arcs, d_offsets, reinterpret_cast<const float*>(d_weights), *p,
                                 d_membership, &passes);
    else
      s = run_batch_impl<IntMode>(h, c, n_graphs, n, n_arcs, d_offsets, reinterpret_cast<const int32_t*>(d_weights),
                                  *p, d_membership, &passes);
    if (s != LOUVAIN_OK) {
      cudaStreamSynchronize(c.s);
      cudaGetLastError();
      return s;
    }
  }
  if ((s = ensure_pinned(h, gbytes + 65536)) != LOUVAIN_OK) return s;
  stage = reinterpret_cast<unsigned char*>(h->pin) + 1024;  // the buffer may have grown during the run
  cudaMemcpyAsync(stage, ws.gc, gbytes, cudaMemcpyDeviceToHost, c.s);
  cudaEventRecord(h->events[2], c.s);
  if ((s = sync(h, c, "batch end")) != LOUVAIN_OK) return s;
  const GraphCtl* gcs = reinterpret_cast<const GraphCtl*>(stage);
  int64_t ncomm = 0;
  int32_t max_pass = 0, iters = 0;
  for (int32_t k = 0; k < n_graphs; k++) {
    if (results) {
      results[k].modularity = gcs[k].q;
      results[k].passes = gcs[k].passes;
      results[k].total_iterations = gcs[k].total_iterations;
      results[k].n_communities = gcs[k].n_comm;
      if (graph_vtx_offs[k + 1] == graph_vtx_offs[k] && p->max_passes > 0) {
        results[k].passes = 1;  // as louvain_run: one empty pass
        results[k].total_iterations = p->max_iterations > 0 ? 1 : 0;
      }
    }
    ncomm += gcs[k].n_comm;
    if (gcs[k].passes > max_pass) max_pass = gcs[k].passes;
    iters += gcs[k].total_iterations;
  }
  if (res) {
    res->modularity = __builtin_nan("");
    res->passes = max_pass;
    res->total_iterations = iters;
    res->n_communities = ncomm;
    res->ms_total = elapsed(h, 0, 2);
    res->kernel_launches = (int32_t)c.launches;
  }
  (void)passes;
  return LOUVAIN_OK;
}

namespace {
louvain_status run_entry(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                         const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                         const louvain_params* p, void* stream, const int32_t* d_init, int32_t* d_membership,
                         louvain_result* res, louvain_pass_stats* stats, int32_t stats_cap, int32_t* n_stats) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (!valid_params(p)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid louvain_params");
  if (n > 0 && !d_membership) return set_err(h, LOUVAIN_ERR_INVALID, "membership pointer is NULL");
  if (stats_cap < 0) return set_err(h, LOUVAIN_ERR_INVALID, "stats_cap < 0");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if (p && p->giant_min_degree > 0) c.giant_min = p->giant_min_degree;
  if (p) c.wait_spins = p->wait_spins;
  if (p && p->table_factor > 0) c.table_factor = p->table_factor;
  if (res) std::memset(res, 0, sizeof(*res));
  if (n_stats) *n_stats = 0;
  h->prof.on = p->profile != 0;
  h->arcs_host = p->host_arcs != 0;
  h->prof.used = 0;
  h->prof.recs.clear();
  h->prof.valid = false;
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  if ((s = ensure_pinned(h, 65536)) != LOUVAIN_OK) return s;
  if (!event_at(h, 0)) return set_err(h, LOUVAIN_ERR_CUDA, "event creation failed");
  cudaEventRecord(h->events[0], c.s);
  const bool fp = wtype == LOUVAIN_W_FP32;
  if (p->validate) {
    if ((s = validate_graph(h, c, n, n_arcs, d_offsets, d_targets, d_weights, fp)) != LOUVAIN_OK) return s;
  }
  if (d_init && n > 0) {
    validate_reset(c, h->ws.ctrl);
    validate_range(c, d_init, n, n, h->ws.ctrl);
    const Ctrl* hc = read_ctrl(h, c, &s, "initial membership range");
    if (!hc) return s;
    if (hc->cnt[5]) return set_err(h, LOUVAIN_ERR_INVALID, "initial membership id outside [0, n)");
  }
  RunOut out;
  if (n == 0 && p->max_passes > 0) {
    // an empty graph still takes one (empty) pass whose single iteration converges at once
    out.passes = 1;
    out.total_iterations = p->max_iterations > 0 ? 1 : 0;
    if (stats && stats_cap > 0) {
      std::memset(&stats[0], 0, sizeof(stats[0]));
      stats[0].iterations = out.total_iterations;
      if (n_stats) *n_stats = 1;
    }
  }
  if (n > 0) {
    if (fp)
      s = run_impl<FpMode>(h, c, n, n_arcs, d_offsets, d_targets, reinterpret_cast<const float*>(d_weights), *p,
                           d_membership, &out, stats, stats_cap, n_stats, d_init);
    else
      s = run_impl<IntMode>(h, c, n, n_arcs, d_offsets, d_targets, reinterpret_cast<const int32_t*>(d_weights), *p,
                            d_membership, &out, stats, stats_cap, n_stats, d_init);
    if (s != LOUVAIN_OK) {
      cudaStreamSynchronize(c.s);
      cudaGetLastError();
      return s;
    }
  }
  size_t e_end = (size_t)(p->max_passes + 1) * 6 + 2;
  if (!event_at(h, e_end)) return set_err(h, LOUVAIN_ERR_CUDA, "event creation failed");
  cudaEventRecord(h->events[e_end], c.s);
  if ((s = sync(h, c, "run end")) != LOUVAIN_OK) return s;
  if (res) {
    res->modularity = out.q;
    res->passes = out.passes;
    res->total_iterations = out.total_iterations;
    res->n_communities = out.n_communities;
    res->ms_total = elapsed(h, 0, e_end);
    res->kernel_launches = (int32_t)c.launches;
  }
  return LOUVAIN_OK;
}
}  // namespace

louvain_status louvain_run(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                           const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                           const louvain_params* p, void* stream, int32_t* d_membership, louvain_result* res,
                           louvain_pass_stats* stats, int32_t stats_cap, int32_t* n_stats) {
  return run_entry(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype, p, stream, nullptr, d_membership, res, stats,
                   stats_cap, n_stats);
}

louvain_status louvain_run_from(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, const int32_t* d_initial,
                                int32_t* d_membership, louvain_result* res, louvain_pass_stats* stats,
                                int32_t stats_cap, int32_t* n_stats) {
  if (h && n > 0 && !d_initial) return set_err(h, LOUVAIN_ERR_INVALID, "initial membership pointer is NULL");
  return run_entry(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype, p, stream, d_initial, d_membership, res,
                   stats, stats_cap, n_stats);
}

louvain_status louvain_update_graph(louvain_handle h, int64_t n_old, int64_t n_arcs, const int64_t* d_offsets,
                                    const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                    int64_t n_new, int64_t n_del, const int32_t* d_del_u, const int32_t* d_del_v,
                                    int64_t n_ins, const int32_t* d_ins_u, const int32_t* d_ins_v,
                                    const void* d_ins_w, void* stream, int64_t* d_out_offsets,
                                    int32_t* d_out_targets, void* d_out_weights, int64_t out_cap,
                                    int64_t* out_arcs) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n_old, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (n_new < n_old || n_new >= 0x7fffffffLL) return set_err(h, LOUVAIN_ERR_INVALID, "n_new must be in [n_old, 2^31 - 1)");
  if (n_del < 0 || n_ins < 0 || out_cap < 0 || !out_arcs || !d_out_offsets)
    return set_err(h, LOUVAIN_ERR_INVALID, "invalid counts or NULL output");
  if (n_del > 0 && (!d_del_u || !d_del_v)) return set_err(h, LOUVAIN_ERR_INVALID, "deletion pointer is NULL");
  if (n_ins > 0 && (!d_ins_u || !d_ins_v || !d_ins_w)) return set_err(h, LOUVAIN_ERR_INVALID, "insertion pointer is NULL");
  if (out_cap > 0 && (!d_out_targets || !d_out_weights)) return set_err(h, LOUVAIN_ERR_INVALID, "output pointer is NULL");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  Workspace& ws = h->ws;
  if ((s = ensure_workspace(h, 1, 1)) != LOUVAIN_OK) return s;  // the control block
  const int64_t words = update_scratch_words(n_new, n_del) + scan_tmp_elems(n_new) + 8;
  if (ws.upd_words < words) {
    free_all(ws.upd_alloc);
    ws.upd_words = 0;
    if (!dalloc(h, ws.upd_alloc, &ws.upd, words)) {
      free_all(ws.upd_alloc);
      return set_err(h, LOUVAIN_ERR_OOM, "graph-update scratch allocation failed");
    }
    ws.upd_words = words;
  }
  int64_t* tile_tmp = reinterpret_cast<int64_t*>(ws.upd + update_scratch_words(n_new, n_del));
  validate_reset(c, ws.ctrl);
  const int slots = update_count(c, n_old, n_arcs, d_offsets, d_targets, n_new, d_del_u, d_del_v, n_del, d_ins_u, d_ins_v,
                                 d_ins_w, n_ins, ws.upd, d_out_offsets, tile_tmp, ws.ctrl);
  const Ctrl* hc = read_ctrl(h, c, &s, "graph update counts");
  if (!hc) return s;
  if (hc->cnt[5]) return set_err(h, LOUVAIN_ERR_INVALID, "update vertex id outside [0, n_new)");
  const int64_t* tot = read_i64(h, c, d_out_offsets + n_new, 1, &s, "graph update size");
  if (!tot) return s;
  const int64_t total = tot[0];
  *out_arcs = total;
  if (total > out_cap) return set_err(h, LOUVAIN_ERR_INVALID, "output capacity below the updated arc count");
  update_fill(c, n_old, n_arcs, d_offsets, d_targets, d_weights, n_new, n_del, d_ins_u, d_ins_v, d_ins_w, n_ins, ws.upd,
              (unsigned)slots, d_out_offsets, d_out_targets, d_out_weights, ws.ctrl);
  return sync(h, c, "graph update");
}

namespace {
// Host arrays the GPU reads in place.  Where the device reads pageable host memory through the
// host's page tables (Grace: ATS over NVLink-C2C) the arrays are used as they are.  Elsewhere the
// pages holding them are registered (mapped, read-only where supported) for the call -- arrays whose
// pages touch are registered as one range -- unless they are pinned already.
struct HostViews {
  std::vector<void*> registered;
  ~HostViews() {
    for (void* b : registered) cudaHostUnregister(b);
  }
};

bool pinned_throughout(const void* p, size_t bytes) {
  for (const char* q : {static_cast<const char*>(p), static_cast<const char*>(p) + bytes - 1}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return false;
    }
  }
  return true;
}

cudaError_t host_views(HostViews& v, int device, const void* const* ptrs, const size_t* bytes, int k,
                       const void** dptrs) {
  int pageable = 0;
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
  cudaGetLastError();
  const uintptr_t page = (uintptr_t)sysconf(_SC_PAGESIZE);
  std::vector<std::pair<uintptr_t, uintptr_t>> ranges;  // page-aligned ranges still to register
  for (int i = 0; i < k; i++) {
    dptrs[i] = ptrs[i];
    if (pageable || bytes[i] == 0 || pinned_throughout(ptrs[i], bytes[i])) continue;
    ranges.push_back({(uintptr_t)ptrs[i] & ~(page - 1), ((uintptr_t)ptrs[i] + bytes[i] + page - 1) & ~(page - 1)});
  }
  std::sort(ranges.begin(), ranges.end());
  std::vector<std::pair<uintptr_t, uintptr_t>> merged;
  for (const auto& r : ranges) {
    if (!merged.empty() && r.first <= merged.back().second) merged.back().second = std::max(merged.back().second, r.second);
    else merged.push_back(r);
  }
  for (const auto& r : merged) {
    void* base = reinterpret_cast<void*>(r.first);
    cudaError_t e = cudaHostRegister(base, r.second - r.first, cudaHostRegisterMapped | cudaHostRegisterReadOnly);
    if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {
      cudaGetLastError();
      e = cudaHostRegister(base, r.second - r.first, cudaHostRegisterMapped);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    v.registered.push_back(base);
  }
  if (pageable) return cudaSuccess;
  for (int i = 0; i < k; i++) {
    if (bytes[i] == 0) continue;
    void* dp = nullptr;
    cudaError_t e = cudaHostGetDevicePointer(&dp, const_cast<void*>(ptrs[i]), 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    dptrs[i] = dp;
  }
  return cudaSuccess;
}
}  // namespace

louvain_status louvain_run_host(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* h_offsets,
                                const int32_t* h_targets, const void* h_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, int32_t* h_membership, louvain_result* res,
                                louvain_pass_stats* stats, int32_t stats_cap, int32_t* n_stats) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n, n_arcs, h_offsets, h_targets, h_weights, wtype)) != LOUVAIN_OK) return s;
  if (n > 0 && !h_membership) return set_err(h, LOUVAIN_ERR_INVALID, "membership pointer is NULL");
  if (!valid_params(p)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid louvain_params");
  // host_arcs: the arcs stay in host memory and are read in place; only the offsets are copied
  const bool in_place = p->host_arcs != 0;
  const int64_t a_in = in_place ? 0 : n_arcs;
  Workspace& ws = h->ws;
  if (ws.in_n < n || ws.in_a < a_in || (in_place && ws.in_a > 0)) {
    free_all(ws.in_alloc);
    ws.in_n = ws.in_a = -1;
    if (!dalloc(h, ws.in_alloc, &ws.in_offs, n + 1) || !dalloc(h, ws.in_alloc, &ws.in_tg, a_in) ||
        !dalloc(h, ws.in_alloc, (int32_t**)&ws.in_w, a_in) || !dalloc(h, ws.in_alloc, &ws.in_mem, n)) {
      free_all(ws.in_alloc);
      return set_err(h, LOUVAIN_ERR_OOM, "input staging allocation failed");
    }
    ws.in_n = n;
    ws.in_a = a_in;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int32_t* d_tg = ws.in_tg;
  const void* d_w = ws.in_w;
  HostViews views;
  cudaMemcpyAsync(ws.in_offs, h_offsets, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (n_arcs > 0) {
    if (in_place) {
      const void* hp[2] = {h_targets, h_weights};
      const size_t hb[2] = {(size_t)n_arcs * sizeof(int32_t), (size_t)n_arcs * 4};
      const void* dp[2] = {nullptr, nullptr};
      cudaError_t e = host_views(views, h->device, hp, hb, 2, dp);
      if (e != cudaSuccess) return cuda_err(h, e, "making the host arcs readable by the device");
      d_tg = static_cast<const int32_t*>(dp[0]);
      d_w = dp[1];
    } else {
      cudaMemcpyAsync(ws.in_tg, h_targets, (size_t)n_arcs * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(ws.in_w, h_weights, (size_t)n_arcs * 4, cudaMemcpyHostToDevice, st);
    }
  }
  s = louvain_run(h, n, n_arcs, ws.in_offs, d_tg, d_w, wtype, p, stream, ws.in_mem, res, stats, stats_cap, n_stats);
  if (s != LOUVAIN_OK) return s;
  if (n > 0) cudaMemcpyAsync(h_membership, ws.in_mem, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(h, e, "run_host copy back");
  return LOUVAIN_OK;
}

louvain_status louvain_modularity(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                  const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                  const int32_t* d_membership, void* stream, double* q) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (!q || (n > 0 && !d_membership)) return set_err(h, LOUVAIN_ERR_INVALID, "NULL output / membership");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  const bool fp = wtype == LOUVAIN_W_FP32;
  if ((s = validate_graph(h, c, n, n_arcs, d_offsets, d_targets, d_weights, fp)) != LOUVAIN_OK) return s;
  validate_range(c, d_membership, n, n, h->ws.ctrl);
  const Ctrl* hc = read_ctrl(h, c, &s, "membership range");
  if (!hc) return s;
  if (hc->cnt[5]) return set_err(h, LOUVAIN_ERR_INVALID, "membership id outside [0, n)");
  int64_t hb[kNumBuckets + 1], gs = 0;
  if (fp) {
    GraphView<float> g{n, d_offsets, d_offsets + 1, d_targets, reinterpret_cast<const float*>(d_weights)};
    if ((s = degree_buckets(h, c, g, hb, &gs)) != LOUVAIN_OK) return s;
    modularity_bucketed<FpMode>(c, g, d_membership, reinterpret_cast<double*>(h->ws.tot), h->ws.ctrl, h->ws.dperm, hb,
                                h->ws.gpv);
  } else {
    GraphView<int32_t> g{n, d_offsets, d_offsets + 1, d_targets, reinterpret_cast<const int32_t*>(d_weights)};
    if ((s = degree_buckets(h, c, g, hb, &gs)) != LOUVAIN_OK) return s;
    modularity_bucketed<IntMode>(c, g, d_membership, reinterpret_cast<long long*>(h->ws.tot), h->ws.ctrl, h->ws.dperm,
                                 hb, h->ws.gpv);
  }
  hc = read_ctrl(h, c, &s, "modularity");
  if (!hc) return s;
  *q = hc->q;
  return LOUVAIN_OK;
}

louvain_status louvain_colour(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                              const int32_t* d_targets, uint64_t seed, int32_t pass, void* stream, int32_t* d_colour,
                              int32_t* n_colours) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if (n < 0 || n >= 0x7fffffffLL || n_arcs < 0 || !d_offsets || (n_arcs > 0 && !d_targets) || !n_colours ||
      (n > 0 && !d_colour))
    return set_err(h, LOUVAIN_ERR_INVALID, "invalid arguments");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  // the colour bitmaps and push chunks are sized from the arcs (ceil((deg + 1) / 32) words a vertex)
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  *n_colours = 0;
  if (n == 0) return LOUVAIN_OK;
  Ctrl* ctrl = h->ws.ctrl;
  cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), c.s);  // error bits of an earlier call must not stop this one
  validate_offsets(c, n, n_arcs, d_offsets, ctrl);
  const Ctrl* hc = read_ctrl(h, c, &s, "validate offsets");
  if (!hc) return s;
  if (hc->cnt[0]) return set_err(h, LOUVAIN_ERR_INVALID, "bad offsets");
  validate_range(c, d_targets, n_arcs, n, ctrl);
  hc = read_ctrl(h, c, &s, "validate targets");
  if (!hc) return s;
  if (hc->cnt[5]) return set_err(h, LOUVAIN_ERR_INVALID, "arc target outside [0, n)");
  GraphView<int32_t> g{n, d_offsets, d_offsets + 1, d_targets, nullptr};
  int64_t hb[kNumBuckets + 1], gslots;
  if ((s = degree_buckets(h, c, g, hb, &gslots)) != LOUVAIN_OK) return s;
  JpBuffers jb{h->ws.jcnt, h->ws.jl0, h->ws.jl1, h->ws.n_cap + 1, h->ws.jrc, h->ws.jbc, h->ws.jbig, h->ws.jbcb,
               h->ws.jcown, h->ws.jchunk_cap, h->ws.jcc, h->ws.jboff, h->ws.jused, h->ws.jused_cap, h->ws.jround,
               h->ws.tile_tmp};
  cudaError_t ce;
  int32_t nc = jp_colour(c, g, h->ws.dperm, hb, seed, pass, d_colour, jb, ctrl, h->pin, &ce);
  if (ce != cudaSuccess) return cuda_err(h, ce, "colouring");
  if (nc < 0) return colour_failure(h, c);
  *n_colours = nc;
  return sync(h, c, "colour end");
}

louvain_status louvain_local_move(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                  const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                  const louvain_params* p, int32_t pass, double tau, void* stream, int32_t* d_cprime,
                                  int32_t* iterations, int64_t* moves) {
  louvain_status s = begin_call(h);
  h->prof.on = false;
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (!valid_params(p) || !iterations || !moves || (n > 0 && !d_cprime) || tau < 0.0)
    return set_err(h, LOUVAIN_ERR_INVALID, "invalid arguments");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if (p && p->giant_min_degree > 0) c.giant_min = p->giant_min_degree;
  if (p) c.wait_spins = p->wait_spins;
  if (p && p->table_factor > 0) c.table_factor = p->table_factor;
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  if ((s = ensure_pinned(h, 65536)) != LOUVAIN_OK) return s;
  const bool fp = wtype == LOUVAIN_W_FP32;
  if ((s = validate_graph(h, c, n, n_arcs, d_offsets, d_targets, d_weights, fp)) != LOUVAIN_OK) return s;
  *iterations = 0;
  *moves = 0;
  if (n == 0) return LOUVAIN_OK;
  Workspace& ws = h->ws;
  cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), c.s);
  auto body = [&](auto mode_tag) -> louvain_status {
    typedef decltype(mode_tag) M;
    typedef typename M::a_t A;
    typedef typename M::w_t W;
    GraphView<W> g{n, d_offsets, d_offsets + 1, d_targets, reinterpret_cast<const W*>(d_weights)};
    PassState<M> st{reinterpret_cast<A*>(ws.K), reinterpret_cast<A*>(ws.Sig), ws.Cp, ws.flags, ws.csize, ws.mv_from,
                    ws.mv_to, ws.ctrl};
    int64_t hb[kNumBuckets + 1], gslots;
    louvain_status r = degree_buckets(h, c, g, hb, &gslots);
    if (r != LOUVAIN_OK) return r;
    vertex_init<M>(c, st, n, false);
    row_sums<M>(c, g, ws.dperm, hb, st.K, st.Sig, reinterpret_cast<A*>(ws.K0));
    total_weight<M>(c, st.K, n, ws.ctrl);
    if (!event_at(h, 3)) return set_err(h, LOUVAIN_ERR_CUDA, "event creation failed");
    r = local_move_phase<M>(h, c, g, hb, gslots, *p, pass, tau, iterations, moves, 3);
    if (r != LOUVAIN_OK) return r;
    cudaMemcpyAsync(d_cprime, ws.Cp, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.s);
    return sync(h, c, "local move end");
  };
  return fp ? body(FpMode()) : body(IntMode());
}

louvain_status louvain_aggregate(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                 const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                 const int32_t* d_membership, int64_t n_comm, void* stream, int64_t* d_out_offsets,
                                 int32_t* d_out_targets, void* d_out_weights, int64_t* out_arcs) {
  louvain_status s = begin_call(h);
  h->prof.on = false;
  if (s != LOUVAIN_OK) return s;
  if ((s = check_graph_args(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype)) != LOUVAIN_OK) return s;
  if (n_comm < 0 || n_comm > n || !d_out_offsets || !out_arcs || (n > 0 && !d_membership) ||
      (n_arcs > 0 && (!d_out_targets || !d_out_weights)))
    return set_err(h, LOUVAIN_ERR_INVALID, "invalid arguments");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if ((s = ensure_workspace(h, n, n_arcs)) != LOUVAIN_OK) return s;
  const bool fp = wtype == LOUVAIN_W_FP32;
  if ((s = validate_graph(h, c, n, n_arcs, d_offsets, d_targets, d_weights, fp)) != LOUVAIN_OK) return s;
  Workspace& ws = h->ws;
  validate_range(c, d_membership, n, n_comm, ws.ctrl);
  const Ctrl* hc = read_ctrl(h, c, &s, "membership range");
  if (!hc) return s;
  if (hc->cnt[5]) return set_err(h, LOUVAIN_ERR_INVALID, "membership id outside [0, n_comm)");
  *out_arcs = 0;
  if (n_comm == 0) {
    cudaMemsetAsync(d_out_offsets, 0, sizeof(int64_t), c.s);
    return sync(h, c, "aggregate end");
  }
  cudaMemcpyAsync(ws.Cp, d_membership, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c.s);
  cudaMemsetAsync(ws.ctrl, 0, sizeof(Ctrl), c.s);
  auto body = [&](auto mode_tag) -> louvain_status {
    typedef decltype(mode_tag) M;
    typedef typename M::w_t W;
    GraphView<W> g{n, d_offsets, d_offsets + 1, d_targets, reinterpret_cast<const W*>(d_weights)};
    RowSet& rs = ws.rows[0];
    int64_t hb[kNumBuckets + 1], gslots;
    louvain_status r = degree_buckets(h, c, g, hb, &gslots);
    if (r != LOUVAIN_OK) return r;
    int64_t cb[kNumBuckets + 1];
    r = aggregate_phase<M>(h, c, g, hb, n_comm, rs, ws.tgA, reinterpret_cast<W*>(ws.wA), cb);
    if (r != LOUVAIN_OK) return r;
    row_lengths(c, n_comm, rs.hoff, rs.hend, ws.len);
    scan_exclusive_i64(c, ws.len, d_out_offsets, n_comm, ws.tile_tmp);
    compact_bucketed<W>(c, ws.cperm, cb, rs.hoff, rs.hend, d_out_offsets, ws.tgA, reinterpret_cast<W*>(ws.wA),
                        d_out_targets, reinterpret_cast<W*>(d_out_weights), ws.gpv, ws.ctrl);
    const int64_t* t = read_i64(h, c, d_out_offsets + n_comm, 1, &r, "aggregate total");
    if (!t) return r;
    *out_arcs = t[0];
    const Ctrl* cc = read_ctrl(h, c, &r, "aggregate end");
    if (!cc) return r;
    if (cc->error) return set_err(h, LOUVAIN_ERR_CUDA, "internal: hash table overflow in aggregation");
    return LOUVAIN_OK;
  };
  return fp ? body(FpMode()) : body(IntMode());
}

louvain_status louvain_kernel_profile(louvain_handle h, louvain_kernel_stat* out, int32_t cap, int32_t* n) {
  if (!h || !n || (cap > 0 && !out)) return LOUVAIN_ERR_INVALID;
  *n = 0;
  if (!h->prof.valid) return set_err(h, LOUVAIN_ERR_INVALID, "no profiled run (set params.profile = 1)");
  int32_t k = 0;
  for (int cls = 0; cls < kNumClasses && k < cap; cls++) {
    if (h->prof.launches[cls] == 0) continue;
    std::memset(&out[k], 0, sizeof(out[k]));
    std::strncpy(out[k].name, kClassNames[cls], sizeof(out[k].name) - 1);
    out[k].launches = h->prof.launches[cls];
    out[k].ms = h->prof.ms[cls];
    out[k].algorithmic_bytes = h->prof.bytes[cls];
    k++;
  }
  *n = k;
  return LOUVAIN_OK;
}

louvain_status louvain_autotune(louvain_handle h, int64_t n, int64_t n_arcs, const int64_t* d_offsets,
                                const int32_t* d_targets, const void* d_weights, louvain_wtype wtype,
                                const louvain_params* p, void* stream, int32_t* d_membership, int32_t reps,
                                louvain_params* tuned, float* best_ms) {
  if (!h || !p || !tuned) return LOUVAIN_ERR_INVALID;
  if (!valid_params(p)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid louvain_params");
  return autotune_impl(h, p, reps, [&](const louvain_params& q, float* ms) {
    louvain_result r;
    louvain_status s = louvain_run(h, n, n_arcs, d_offsets, d_targets, d_weights, wtype, &q, stream, d_membership, &r,
                                   nullptr, 0, nullptr);
    *ms = r.ms_total;
    return s;
  }, tuned, best_ms);
}

louvain_status louvain_autotune_batch(louvain_handle h, int32_t n_graphs, const int64_t* graph_vtx_offs,
                                      int64_t n_arcs, const int64_t* d_offsets, const int32_t* d_targets,
                                      const void* d_weights, louvain_wtype wtype, const louvain_params* p,
                                      void* stream, int32_t* d_membership, int32_t reps, louvain_params* tuned,
                                      float* best_ms) {
  if (!h || !p || !tuned) return LOUVAIN_ERR_INVALID;
  if (!valid_params(p)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid louvain_params");
  return autotune_impl(h, p, reps, [&](const louvain_params& q, float* ms) {
    louvain_result r;
    louvain_status s = louvain_run_batch(h, n_graphs, graph_vtx_offs, n_arcs, d_offsets, d_targets, d_weights, wtype,
                                         &q, stream, d_membership, nullptr, &r);
    *ms = r.ms_total;
    return s;
  }, tuned, best_ms);
}

louvain_status louvain_exclusive_scan(louvain_handle h, const int64_t* d_in, int64_t* d_out, int64_t count,
                                      void* stream, int64_t* total) {
  louvain_status s = begin_call(h);
  if (s != LOUVAIN_OK) return s;
  if (count < 0 || !d_out || (count > 0 && !d_in)) return set_err(h, LOUVAIN_ERR_INVALID, "invalid arguments");
  Ctx c;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.num_sms = h->num_sms;
  if ((s = ensure_workspace(h, count, 0)) != LOUVAIN_OK) return s;
  scan_exclusive_i64(c, d_in, d_out, count, h->ws.tile_tmp);
  if (total) {
    const int64_t* t = read_i64(h, c, d_out + count, 1, &s, "scan total");
    if (!t) return s;
    *total = t[0];
  }
  return sync(h, c, "scan end");
}

}  // extern "C"
