// serve.cu -- continuous-batching request loop over louvain_run_batch (host runtime).
//
// Requests (host CSRs) enter a FIFO queue.  Each of L lanes -- a worker thread with its own CUDA
// stream, library handle and union buffers -- takes, whenever it is free, the oldest request and
// every queued request of its class (weight type; inside or outside the in-flight window) that
// fits its limits and the server's device-memory budget, runs them as ONE batched call
// (batch.cu: every graph gets exactly its single-graph result), copies each membership back to
// the caller's buffer and releases the memory.  Requests that arrive while lanes are busy wait
// only for the next free lane and for memory; lanes run concurrently on the device, so their
// work overlaps.  Admission: a lane reserves an upper bound of the device bytes its batch needs
// (its handle's cap is set to exactly that reservation, so it cannot exceed it); the sum of all
// lanes' reservations never exceeds the budget.  A request larger than the whole budget fails
// with LOUVAIN_ERR_OOM.  Latency = submit to membership-on-host, on the host's steady clock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

using namespace lv;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, a = 0;
  const int64_t* offs = nullptr;
  const int32_t* tg = nullptr;
  const void* w = nullptr;
  louvain_wtype wtype = LOUVAIN_W_INT32;
  int32_t* out = nullptr;
  size_t est = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int32_t batch_graphs = 0;
  double prep_ms = 0, upload_ms = 0, run_ms = 0, download_ms = 0;  // its batch's breakdown
  bool in_flight = false;  // the graph fits what the GPU holds in flight (fast mode's schedule class)
  bool picked = false;     // taken into the batch being formed
  louvain_status status = LOUVAIN_OK;
  louvain_graph_result result{};
  bool done = false;
};

// Upper bound of the device bytes a batched call holds for n vertices and a arcs: the handle's
// per-vertex state (~220 B), ping-pong super-graph arcs and union targets (20 B/arc), the giant-row
// table pool (<= 40 B per arc in giant rows), plus the lane's union input (offsets, targets,
// weights, membership).
size_t estimate_bytes(int64_t n, int64_t a) {
  return (size_t)(256 * (n + 1) + 72 * a) + ((size_t)64 << 20);
}

struct Lane {
  std::thread th;
  louvain_handle h = nullptr;
  cudaStream_t s = nullptr;
  int64_t cap_n = -1, cap_a = -1;
  // largest batch dimensions since the lane's caches were last dropped: the handle's workspace and
  // the union buffers only grow, so what the lane holds is bounded by estimate_bytes(hn, ha)
  int64_t hn = 0, ha = 0;
  int64_t* d_offs = nullptr;
  int32_t* d_tg = nullptr;
  int32_t* d_w = nullptr;
  int32_t* d_mem = nullptr;
  size_t reserved = 0;
  cudaEvent_t ev[4] = {};  // batch phase boundaries on the lane's stream
  double prep_ms = 0;      // the last batch's host preparation and device phases
  float up_ms = 0, run_ms = 0, down_ms = 0;
};

}  // namespace

struct louvain_server_s {
  int device = 0;
  size_t budget = 0;
  int32_t max_graphs = 256;
  int64_t max_arcs = 0;
  int64_t window = 0;  // vertices the GPU holds in flight (SMs x kInFlightPerSm)
  louvain_params p{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  size_t reserved_total = 0;
  bool stopping = false;
  bool want_memory = false;  // the queue head waits for memory: idle lanes drop their caches
  std::vector<Lane> lanes;
  std::string err;
};

namespace {

void lane_free_buffers(Lane& L) {
  if (L.d_offs) cudaFree(L.d_offs);
  if (L.d_tg) cudaFree(L.d_tg);
  if (L.d_w) cudaFree(L.d_w);
  if (L.d_mem) cudaFree(L.d_mem);
  L.d_offs = nullptr; L.d_tg = nullptr; L.d_w = nullptr; L.d_mem = nullptr;
  L.cap_n = L.cap_a = -1;
}

bool lane_buffers(Lane& L, int64_t n, int64_t a) {
  if (L.cap_n >= n && L.cap_a >= a) return true;
  n = n > L.cap_n ? n : L.cap_n;  // grow in both dimensions, never shrink one
  a = a > L.cap_a ? a : L.cap_a;
  lane_free_buffers(L);
  const int64_t nn = n + 1, aa = a > 0 ? a : 1;
  if (cudaMalloc(&L.d_offs, sizeof(int64_t) * nn) != cudaSuccess || cudaMalloc(&L.d_tg, sizeof(int32_t) * aa) != cudaSuccess ||
      cudaMalloc(&L.d_w, sizeof(int32_t) * aa) != cudaSuccess || cudaMalloc(&L.d_mem, sizeof(int32_t) * nn) != cudaSuccess) {
    cudaGetLastError();
    lane_free_buffers(L);
    return false;
  }
  L.cap_n = n;
  L.cap_a = a;
  return true;
}

void finish(louvain_server_s* S, std::vector<Request*>& batch, louvain_status st, const louvain_graph_result* res,
            const double times[4]) {
  const double t = now_ms();
  std::lock_guard<std::mutex> lk(S->mu);
  for (size_t k = 0; k < batch.size(); k++) {
    Request* r = batch[k];
    r->status = st;
    if (res) r->result = res[k];
    r->t_done = t;
    r->batch_graphs = (int32_t)batch.size();
    r->prep_ms = times[0];
    r->upload_ms = times[1];
    r->run_ms = times[2];
    r->download_ms = times[3];
    r->done = true;
  }
  S->cv_done.notify_all();
}

// Runs one batch on a lane: union upload, louvain_run_batch, memberships back to the callers.
louvain_status run_lane_batch(louvain_server_s* S, Lane& L, std::vector<Request*>& batch,
                              std::vector<louvain_graph_result>& res) {
  const int32_t G = (int32_t)batch.size();
  std::vector<int64_t> vo(G + 1, 0);
  int64_t a_tot = 0;
  for (int32_t k = 0; k < G; k++) {
    vo[k + 1] = vo[k] + batch[k]->n;
    a_tot += batch[k]->a;
  }
  const int64_t n = vo[G];
  L.prep_ms = 0;
  L.up_ms = L.run_ms = L.down_ms = 0;
  if (!lane_buffers(L, n, a_tot)) return LOUVAIN_ERR_OOM;
  const double t0 = now_ms();
  // union offsets: each graph's offsets shifted by its arc base (built on the host)
  std::vector<int64_t> offs(n + 1);
  int64_t ab = 0;
  for (int32_t k = 0; k < G; k++) {
    const Request* r = batch[k];
    for (int64_t i = 0; i < r->n; i++) offs[vo[k] + i] = r->offs[i] + ab;
    ab += r->a;
  }
  offs[n] = ab;
  L.prep_ms = now_ms() - t0;
  cudaEventRecord(L.ev[0], L.s);
  cudaMemcpyAsync(L.d_offs, offs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, L.s);
  ab = 0;
  for (int32_t k = 0; k < G; k++) {
    const Request* r = batch[k];
    if (r->a > 0) {
      cudaMemcpyAsync(L.d_tg + ab, r->tg, sizeof(int32_t) * r->a, cudaMemcpyHostToDevice, L.s);
      cudaMemcpyAsync(L.d_w + ab, r->w, 4 * (size_t)r->a, cudaMemcpyHostToDevice, L.s);
    }
    ab += r->a;
  }
  cudaEventRecord(L.ev[1], L.s);
  res.assign(G, louvain_graph_result{});
  louvain_result tot;
  louvain_status st = louvain_run_batch(L.h, G, vo.data(), a_tot, L.d_offs, L.d_tg, L.d_w, batch[0]->wtype, &S->p,
                                        L.s, L.d_mem, res.data(), &tot);
  if (st != LOUVAIN_OK) return st;
  cudaEventRecord(L.ev[2], L.s);
  for (int32_t k = 0; k < G; k++)
    if (batch[k]->n > 0)
      cudaMemcpyAsync(batch[k]->out, L.d_mem + vo[k], sizeof(int32_t) * batch[k]->n, cudaMemcpyDeviceToHost, L.s);
  cudaEventRecord(L.ev[3], L.s);
  if (cudaStreamSynchronize(L.s) != cudaSuccess) {
    cudaGetLastError();
    return LOUVAIN_ERR_CUDA;
  }
  if (cudaEventElapsedTime(&L.up_ms, L.ev[0], L.ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&L.run_ms, L.ev[1], L.ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(&L.down_ms, L.ev[2], L.ev[3]) != cudaSuccess) {
    cudaGetLastError();
    L.up_ms = L.run_ms = L.down_ms = 0;
  }
  return LOUVAIN_OK;
}

void lane_main(louvain_server_s* S, int idx) {
  Lane& L = S->lanes[idx];
  cudaSetDevice(S->device);
  std::vector<Request*> batch;
  std::vector<louvain_graph_result> res;
  while (true) {
    batch.clear();
    size_t need = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stopping && S->queue.empty()) return;
        if (!S->queue.empty()) {
          // the head request first (FIFO), then the queued requests of its class -- weight type,
          // and whether the graph fits what the GPU holds in flight, which decides fast mode's
          // schedule for a batch by its mean graph -- in queue order while they fit; the lane's
          // caches grow to the largest dimensions they have served, which its need covers
          const size_t others = S->reserved_total - L.reserved;
          int64_t n = 0, a = 0;
          for (Request* r : S->queue) {
            if ((int32_t)batch.size() >= S->max_graphs) break;
            if (!batch.empty() && (r->wtype != batch[0]->wtype || r->in_flight != batch[0]->in_flight)) continue;
            if (!batch.empty() && S->max_arcs > 0 && a + r->a > S->max_arcs) break;
            const size_t e = std::max(estimate_bytes(std::max(L.hn, n + r->n), std::max(L.ha, a + r->a)), L.reserved);
            if (others + e > S->budget) break;
            batch.push_back(r);
            r->picked = true;
            n += r->n;
            a += r->a;
            need = e;
          }
          if (!batch.empty()) {
            S->queue.erase(std::remove_if(S->queue.begin(), S->queue.end(), [](const Request* r) { return r->picked; }),
                           S->queue.end());
            S->reserved_total = others + need;
            L.reserved = need;
            L.hn = std::max(L.hn, n);
            L.ha = std::max(L.ha, a);
            S->want_memory = false;
            break;
          }
          if (L.hn > 0 || L.reserved > 0) {
            // the lane's own caches stand in the way: drop them and size the batch afresh
            const size_t mine = L.reserved;
            lk.unlock();
            handle_trim(L.h);
            lane_free_buffers(L);
            lk.lock();
            S->reserved_total -= mine;
            L.reserved = 0;
            L.hn = L.ha = 0;
            continue;
          }
          // the head does not fit now (it fits an empty device: checked at submit): ask the idle
          // lanes to drop their caches and wait for running batches to finish
          S->want_memory = true;
          S->cv_work.notify_all();
        }
        if (S->want_memory && L.reserved > 0) {
          const size_t mine = L.reserved;
          lk.unlock();
          handle_trim(L.h);
          lane_free_buffers(L);
          lk.lock();
          S->reserved_total -= mine;
          L.reserved = 0;
          L.hn = L.ha = 0;
          S->cv_work.notify_all();
          continue;
        }
        S->cv_work.wait(lk);
      }
    }
    const double t0 = now_ms();
    for (Request* r : batch) r->t_start = t0;
    {
      // the handle may use the reservation minus the lane's own union buffers (their largest size)
      const size_t lane_bytes = (size_t)(12 * (L.hn + 1) + 8 * L.ha);
      handle_set_budget(L.h, need > lane_bytes ? need - lane_bytes : 1);
    }
    louvain_status st = run_lane_batch(S, L, batch, res);
    if (st != LOUVAIN_OK) {
      // the reservation is an upper bound, so an OOM here means the estimate was too small for this
      // input: fail the batch, free the lane's caches and go on
      cudaStreamSynchronize(L.s);
      cudaGetLastError();
    }
    const double times[4] = {L.prep_ms, L.up_ms, L.run_ms, L.down_ms};
    finish(S, batch, st, st == LOUVAIN_OK ? res.data() : nullptr, times);
    // keep the caches only while they fit the budget share of an idle lane
    const size_t held = handle_device_bytes(L.h) +
                        (L.cap_n >= 0 ? (size_t)(8 * (L.cap_n + 1) + 4 * (L.cap_n + 1) + 8 * L.cap_a) : 0);
    const size_t share = S->budget / (S->lanes.size() ? S->lanes.size() : 1);
    if (st != LOUVAIN_OK || held > share) {
      handle_trim(L.h);
      lane_free_buffers(L);
      L.hn = L.ha = 0;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const size_t keep = (st == LOUVAIN_OK && held <= share) ? held : 0;
      S->reserved_total = S->reserved_total - L.reserved + keep;
      L.reserved = keep;
    }
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

louvain_status louvain_serve_create(louvain_server* out, int device, size_t hbm_budget_bytes, int32_t lanes,
                                    int32_t max_batch_graphs, int64_t max_batch_arcs, const louvain_params* p) {
  if (!out || !p || lanes < 1 || lanes > 64 || max_batch_graphs < 1 || max_batch_arcs < 0 || hbm_budget_bytes == 0)
    return LOUVAIN_ERR_INVALID;
  *out = nullptr;
  louvain_server_s* S = new (std::nothrow) louvain_server_s();
  if (!S) return LOUVAIN_ERR_OOM;
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->max_graphs = max_batch_graphs;
  S->max_arcs = max_batch_arcs;
  S->p = *p;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    delete S;
    return LOUVAIN_ERR_CUDA;
  }
  S->window = (int64_t)sms * kInFlightPerSm;
  S->lanes.resize(lanes);
  for (Lane& L : S->lanes) {
    louvain_status st = louvain_create(&L.h, device, 0);
    if (st == LOUVAIN_OK && cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      st = LOUVAIN_ERR_CUDA;
    }
    for (int e = 0; e < 4 && st == LOUVAIN_OK; e++)
      if (cudaEventCreate(&L.ev[e]) != cudaSuccess) {
        cudaGetLastError();
        st = LOUVAIN_ERR_CUDA;
      }
    if (st != LOUVAIN_OK) {
      for (Lane& M : S->lanes) {
        for (cudaEvent_t& e : M.ev)
          if (e) cudaEventDestroy(e);
        if (M.s) cudaStreamDestroy(M.s);
        louvain_destroy(M.h);
      }
      delete S;
      return st;
    }
  }
  for (int k = 0; k < lanes; k++) S->lanes[k].th = std::thread(lane_main, S, k);
  *out = S;
  return LOUVAIN_OK;
}

louvain_status louvain_serve_submit(louvain_server S, int64_t n, int64_t n_arcs, const int64_t* h_offsets,
                                    const int32_t* h_targets, const void* h_weights, louvain_wtype wtype,
                                    int32_t* h_membership, uint64_t* ticket) {
  if (!S || !ticket || n < 0 || n >= 0x7fffffffLL || n_arcs < 0 || !h_offsets || (n > 0 && !h_membership) ||
      (n_arcs > 0 && (!h_targets || !h_weights)) || (wtype != LOUVAIN_W_INT32 && wtype != LOUVAIN_W_FP32))
    return LOUVAIN_ERR_INVALID;
  if (h_offsets[0] != 0 || h_offsets[n] != n_arcs) return LOUVAIN_ERR_INVALID;
  const size_t est = estimate_bytes(n, n_arcs);
  if (est > S->budget) return LOUVAIN_ERR_OOM;
  Request* r = new (std::nothrow) Request();
  if (!r) return LOUVAIN_ERR_OOM;
  r->n = n; r->a = n_arcs; r->offs = h_offsets; r->tg = h_targets; r->w = h_weights; r->wtype = wtype;
  r->out = h_membership; r->est = est;
  r->in_flight = n <= S->window;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) {
      delete r;
      return LOUVAIN_ERR_BUSY;
    }
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
  }
  S->cv_work.notify_one();
  return LOUVAIN_OK;
}

louvain_status louvain_serve_poll(louvain_server S, uint64_t ticket, int32_t wait_ms, louvain_serve_result* out) {
  if (!S || !out || wait_ms < 0) return LOUVAIN_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return LOUVAIN_ERR_INVALID;
  Request* r = it->second;
  if (!r->done && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [r] { return r->done; });
  if (!r->done) return LOUVAIN_OK;  // out->ready = 0
  out->ready = 1;
  out->status = r->status;
  out->result = r->result;
  out->latency_ms = r->t_done - r->t_submit;
  out->queue_ms = r->t_start - r->t_submit;
  out->batch_graphs = r->batch_graphs;
  out->prep_ms = r->prep_ms;
  out->upload_ms = r->upload_ms;
  out->run_ms = r->run_ms;
  out->download_ms = r->download_ms;
  S->reqs.erase(it);
  delete r;
  return LOUVAIN_OK;
}

void louvain_serve_destroy(louvain_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (Lane& L : S->lanes)
    if (L.th.joinable()) L.th.join();
  cudaSetDevice(S->device);
  for (Lane& L : S->lanes) {
    lane_free_buffers(L);
    for (cudaEvent_t& e : L.ev)
      if (e) cudaEventDestroy(e);
    if (L.s) cudaStreamDestroy(L.s);
    louvain_destroy(L.h);
  }
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}

}  // extern "C"
