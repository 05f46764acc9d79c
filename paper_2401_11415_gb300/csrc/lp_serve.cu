// lp_serve.cu -- continuous batching of per-source queries (lp_serve_*).
//
// Requests (per-source top-k queries of uneven size) are queued from any
// thread.  Each of `slots` workers owns a shadow view of the graph (shared
// device arrays, its own stream and scratch) plus device and pinned host
// buffers sized for max_batch_sources sources.  A worker takes the oldest
// pending request and every other pending request with the same (measure,
// hub limit, k) up to the source budget, runs them as one per-source batch
// (lp_predict_sources semantics), and scatters the rows back.  Requests that
// arrive while batches run are admitted by the next free slot, so batches of
// different slots overlap on the device.  Row i of a request depends only on
// its own source (the per-source scan has no cross-source state), so a result
// is identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lp_internal.cuh"

namespace {

struct Request {
  uint64_t id = 0;
  int measure = 0, cap = -1, k = 1;
  std::vector<int32_t> sources;
  std::vector<lp_link> out;
  std::vector<int32_t> counts;
  lp_status status = LP_OK;
  std::string error;  // the worker's error text when status != LP_OK
  bool done = false;
};

struct Slot {
  lp::Graph* shadow = nullptr;
  int* d_src = nullptr;
  lp_link* d_out = nullptr;
  int* d_cnt = nullptr;
  int* h_src = nullptr;
  lp_link* h_out = nullptr;
  int* h_cnt = nullptr;
};

}  // namespace

struct lp_server {
  const lp_graph* g = nullptr;
  lp::Graph* base = nullptr;
  lp_serve_opts opts{};
  std::vector<Slot> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> live;
  uint64_t next_id = 1;
  bool closing = false;
  bool paused = false;
  lp_serve_stats stats{};
};

namespace {

void free_slot(Slot& s) {
  cudaFree(s.d_src);
  cudaFree(s.d_out);
  cudaFree(s.d_cnt);
  cudaFreeHost(s.h_src);
  cudaFreeHost(s.h_out);
  cudaFreeHost(s.h_cnt);
  if (s.shadow) lp::destroy_shadow(s.shadow);
  s = Slot{};
}

void worker_main(lp_server* S, int si) {
  Slot& slot = S->slots[si];
  cudaSetDevice(S->base->device);
  std::vector<Request*> batch;
  for (;;) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] { return S->closing || (!S->paused && !S->pending.empty()); });
      if (S->pending.empty()) return;  // closing and drained
      Request* first = S->pending.front();
      int64_t budget = S->opts.max_batch_sources;
      for (auto it = S->pending.begin(); it != S->pending.end();) {
        Request* r = *it;
        if (r->measure == first->measure && r->cap == first->cap && r->k == first->k &&
            (int64_t)r->sources.size() <= budget) {
          budget -= (int64_t)r->sources.size();
          batch.push_back(r);
          it = S->pending.erase(it);
          if (budget == 0) break;
        } else {
          ++it;
        }
      }
    }
    // one device batch: concatenated sources
    const int k = batch[0]->k;
    int n = 0;
    for (Request* r : batch) {
      std::memcpy(slot.h_src + n, r->sources.data(), sizeof(int32_t) * r->sources.size());
      n += (int)r->sources.size();
    }
    cudaStream_t st = slot.shadow->stream;
    lp_status status = LP_OK;
    cudaError_t e = cudaMemcpyAsync(slot.d_src, slot.h_src, sizeof(int) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) status = lp::report_cuda(e, "serving: source upload");
    if (status == LP_OK)
      status = lp::run_sources_dev(*slot.shadow, batch[0]->measure, batch[0]->cap, slot.d_src, n, k,
                                   0.0, slot.d_out, slot.d_cnt);
    if (status == LP_OK) {
      e = cudaMemcpyAsync(slot.h_out, slot.d_out, sizeof(lp_link) * (size_t)n * k,
                          cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(slot.h_cnt, slot.d_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) status = lp::report_cuda(e, "serving: result download");
    }
    const std::string error = status == LP_OK ? std::string() : std::string(lp_last_error());
    int off = 0;
    for (Request* r : batch) {
      const size_t m = r->sources.size();
      if (status == LP_OK) {
        r->out.assign(slot.h_out + (size_t)off * k, slot.h_out + (size_t)(off + m) * k);
        r->counts.assign(slot.h_cnt + off, slot.h_cnt + off + m);
      }
      r->status = status;
      r->error = error;
      off += (int)m;
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (Request* r : batch) r->done = true;
      S->stats.completed += (int64_t)batch.size();
      S->stats.batches += 1;
      S->stats.batched_sources += n;
      S->stats.max_batch_requests = std::max<int64_t>(S->stats.max_batch_requests, (int64_t)batch.size());
    }
    S->cv_done.notify_all();
  }
}

lp_status serve_fail(lp_status s, const char* msg) { return lp::report_error(s, msg); }

}  // namespace

extern "C" {

lp_status lp_serve_open(const lp_graph* g, const lp_serve_opts* opts, lp_server** out) {
  if (!g || !out) return serve_fail(LP_EINVAL, "lp_serve_open: null argument");
  *out = nullptr;
  lp_serve_opts o{};
  if (opts) o = *opts;
  if (o.slots == 0) o.slots = 2;
  if (o.max_batch_sources == 0) o.max_batch_sources = 65536;
  if (o.max_pending == 0) o.max_pending = 65536;
  if (o.max_k == 0) o.max_k = 16;
  if (o.slots < 1 || o.slots > 8 || o.max_batch_sources < 1 || o.max_pending < 1 || o.max_k < 1 ||
      o.max_k > LP_MAX_TOPK_PER_SOURCE)
    return serve_fail(LP_EINVAL, "lp_serve_open: option out of range");
  lp_server* S = new (std::nothrow) lp_server();
  if (!S) return serve_fail(LP_ENOMEM, "lp_serve_open: host allocation");
  S->g = g;
  S->base = &lp::graph_of(g);
  S->opts = o;
  S->paused = o.paused != 0;
  S->slots.resize(o.slots);
  cudaError_t e = cudaSetDevice(S->base->device);
  const size_t ns = (size_t)o.max_batch_sources;
  for (int i = 0; i < o.slots && e == cudaSuccess; ++i) {
    Slot& sl = S->slots[i];
    if (lp::make_shadow(*S->base, &sl.shadow) != LP_OK) {
      e = cudaErrorMemoryAllocation;
      break;
    }
    e = cudaMalloc(&sl.d_src, sizeof(int) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, sizeof(lp_link) * ns * o.max_k);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_cnt, sizeof(int) * ns);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_src, sizeof(int) * ns);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, sizeof(lp_link) * ns * o.max_k);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_cnt, sizeof(int) * ns);
  }
  if (e != cudaSuccess) {
    for (auto& sl : S->slots) free_slot(sl);
    delete S;
    return lp::report_cuda(e, "lp_serve_open");
  }
  for (int i = 0; i < o.slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return LP_OK;
}

lp_status lp_serve_submit(lp_server* S, const int32_t* sources, int32_t n_src, lp_measure measure,
                          int32_t degree_cap, int32_t k, uint64_t* req_id) {
  if (!S || !req_id || !sources) return serve_fail(LP_EINVAL, "lp_serve_submit: null argument");
  if ((int)measure < 0 || (int)measure > LP_RA) return serve_fail(LP_EINVAL, "lp_serve_submit: bad measure");
  if (n_src < 1 || n_src > S->opts.max_batch_sources)
    return serve_fail(LP_EINVAL, "lp_serve_submit: n_src outside [1, max_batch_sources]");
  if (k < 1 || k > S->opts.max_k) return serve_fail(LP_EINVAL, "lp_serve_submit: k outside [1, max_k]");
  const int32_t n = S->base->n;
  for (int32_t i = 0; i < n_src; ++i)
    if (sources[i] < 0 || sources[i] >= n)
      return serve_fail(LP_EINVAL, "lp_serve_submit: source id out of range");
  Request* r = new (std::nothrow) Request();
  if (!r) return serve_fail(LP_ENOMEM, "lp_serve_submit: host allocation");
  r->measure = (int)measure;
  r->cap = degree_cap < 0 ? -1 : degree_cap;
  r->k = k;
  r->sources.assign(sources, sources + n_src);
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->closing) {
      delete r;
      return serve_fail(LP_EINVAL, "lp_serve_submit: server is closing");
    }
    if ((int64_t)S->pending.size() >= S->opts.max_pending) {
      delete r;
      return serve_fail(LP_EBUSY, "lp_serve_submit: queue full");
    }
    r->id = S->next_id++;
    S->pending.push_back(r);
    S->live[r->id] = r;
    S->stats.submitted += 1;
    *req_id = r->id;
  }
  S->cv_work.notify_one();
  return LP_OK;
}

lp_status lp_serve_wait(lp_server* S, uint64_t req_id, int64_t timeout_us, lp_link* out,
                        int32_t* counts) {
  if (!S) return serve_fail(LP_EINVAL, "lp_serve_wait: null server");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->live.find(req_id);
  if (it == S->live.end()) return serve_fail(LP_EINVAL, "lp_serve_wait: unknown request id");
  Request* r = it->second;
  if (timeout_us < 0) {
    S->cv_done.wait(lock, [&] { return r->done; });
  } else if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
    return serve_fail(LP_ETIMEOUT, "lp_serve_wait: request not finished in time");
  }
  S->live.erase(req_id);
  lock.unlock();
  const lp_status st = r->status;
  if (st == LP_OK) {
    if (out) std::memcpy(out, r->out.data(), sizeof(lp_link) * r->out.size());
    if (counts) std::memcpy(counts, r->counts.data(), sizeof(int32_t) * r->counts.size());
  }
  const std::string msg = "lp_serve_wait: the request's batch failed: " + r->error;
  delete r;
  if (st != LP_OK) return serve_fail(st, msg.c_str());
  return LP_OK;
}

lp_status lp_serve_resume(lp_server* S) {
  if (!S) return serve_fail(LP_EINVAL, "lp_serve_resume: null server");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->paused = false;
  }
  S->cv_work.notify_all();
  return LP_OK;
}

lp_status lp_serve_poll(lp_server* S, uint64_t req_id, int32_t* done) {
  if (!S || !done) return serve_fail(LP_EINVAL, "lp_serve_poll: null argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->live.find(req_id);
  if (it == S->live.end()) return serve_fail(LP_EINVAL, "lp_serve_poll: unknown request id");
  *done = it->second->done ? 1 : 0;
  return LP_OK;
}

lp_status lp_serve_get_stats(lp_server* S, lp_serve_stats* out) {
  if (!S || !out) return serve_fail(LP_EINVAL, "lp_serve_get_stats: null argument");
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  return LP_OK;
}

lp_status lp_serve_close(lp_server* S) {
  if (!S) return LP_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->closing = true;
    S->paused = false;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->live) delete kv.second;
  S->live.clear();
  for (auto& sl : S->slots) free_slot(sl);
  delete S;
  return LP_OK;
}

}  // extern "C"
