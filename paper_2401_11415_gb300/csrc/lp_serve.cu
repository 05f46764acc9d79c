// lp_serve.cu -- continuous batching of per-source queries (lp_serve_*).
//
// Mode 0 (the default): requests (per-source top-k queries of uneven size)
// are queued from any thread.  Each of `slots` workers owns a shadow view of
// the graph (shared device arrays, its own stream and scratch) plus device
// and pinned host buffers sized for max_batch_sources sources.  A worker
// takes the oldest pending request and every other pending request with the
// same (measure, hub limit, k) up to the source budget, runs them as one
// per-source batch (lp_predict_sources semantics, the tiered kernels), and
// scatters the rows back.  Requests that arrive while batches run are
// admitted by the next free slot, so batches of different slots overlap on
// the device.  Row i of a request depends only on its own source (the
// per-source scan has no cross-source state), so a result is identical alone
// and in any mix.
//
// Mode 1: a resident kernel (lp_serve_dev.cu) serves the requests.  An
// admitted request gets a request slot and room in two pools of pinned host
// memory the GPU reads and writes directly: its sources and its result rows.
// The host writes them, one work item per source into a ring, and then
// advances the ring's published count; the kernel's CTAs claim the items and
// raise the slot's completion word after the last source.  Admission is by
// that memory: a request waits on the host until its sources and rows
// (4 + 16 k bytes per source) fit in the pools, a slot is free and the ring
// has room.  Finished requests are collected by any call that polls (submit,
// wait, poll): their rows are copied out and their memory freed, so waiting
// requests are admitted as memory frees up.  The kernel leaves as a whole:
// once no work has been outstanding for idle_polls x 4 us, a polling call sets
// the stop word, and clears it when the kernel has ended; a call that sees
// published work and no kernel running launches it again.  Sources with more
// than defer_wedges wedges are left by the kernel to a host thread that runs
// them through the tiered pipeline in batches; while such rows wait, the
// kernel is asked to leave, so the pipeline has the whole GPU, and it is
// launched again after them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
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
  // mode 1: where the admitted request lives
  bool admitted = false;
  int slot = -1;
  long long off = 0;  // first source in the pools
  unsigned seq = 0;
  std::vector<int> deferred;  // rows left to the tiered pipeline
};

// First-fit allocator of [0, cap) ranges (pool entries).
struct RangeAlloc {
  std::map<long long, long long> free_;  // start -> length
  void init(long long cap) {
    free_.clear();
    free_[0] = cap;
  }
  long long take(long long n) {
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        const long long at = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[at + n] = len - n;
        return at;
      }
    return -1;
  }
  void give(long long at, long long n) {
    auto nx = free_.lower_bound(at);
    if (nx != free_.end() && at + n == nx->first) {
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == at) {
        pv->second += n;
        return;
      }
    }
    free_[at] = n;
  }
};

// Mode 1 state: pools and ring in pinned host memory the GPU maps, claim and
// finish counters on the device.
struct DevLoop {
  cudaStream_t stream = nullptr;  // the resident kernel's stream
  lp::SrvArgs args{};
  int2* ring = nullptr;
  unsigned long long* tail = nullptr;
  lp::SrvReq* reqs = nullptr;
  int* src_pool = nullptr;
  lp_link* out_pool = nullptr;
  unsigned* done = nullptr;
  unsigned* status = nullptr;
  unsigned* stop = nullptr;
  unsigned char* defer = nullptr;  // per pool source: left to the host
  lp::Graph* shadow = nullptr;     // the tiered pipeline for deferred sources
  int* d_dsrc = nullptr;
  lp_link* d_dout = nullptr;
  int* d_dcnt = nullptr;
  std::vector<int> h_dsrc;
  std::vector<lp_link> h_dout;
  std::vector<int> h_dcnt;
  unsigned long long* d_head = nullptr;
  unsigned long long* d_finished = nullptr;
  long long pool_cap = 0;        // sources the pools hold
  long long ring_cap = 0;
  int nslots = 0;                // request slots
  unsigned long long published = 0, retired = 0;  // work items
  std::vector<long long> slot_total;  // sources ever assigned to each slot
  std::vector<int> free_slots;
  RangeAlloc pool;
  std::deque<Request*> waiting;  // submitted, not admitted yet
  std::vector<Request*> inflight;
  std::deque<Request*> dq;        // waiting for their deferred rows
  bool dbusy = false;             // dthread is running a batch of them
  std::chrono::steady_clock::time_point launched_at;
  std::thread dthread;            // runs the deferred rows in batches
  bool dstop = false;             // ends dthread (set after the last request)
  bool running = false;
  bool stopping = false;  // the stop word is set for lack of work (not by close)
  bool idle_seen = false; // no outstanding work since idle_since
  std::chrono::steady_clock::time_point idle_since;
  unsigned next_seq = 1;
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
  DevLoop dev;
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

// ------------------------------------------------------------ mode 1 ----

constexpr int kResident = 1;  // lp_serve_opts.mode of the resident kernel

int first_k(const std::vector<Request*>& batch) { return batch.empty() ? 1 : batch[0]->k; }

void dev_free(DevLoop& D) {
  if (D.stream) {
    cudaStreamSynchronize(D.stream);
    cudaStreamDestroy(D.stream);
  }
  cudaFreeHost(D.ring);
  cudaFreeHost(D.tail);
  cudaFreeHost(D.reqs);
  cudaFreeHost(D.src_pool);
  cudaFreeHost(D.out_pool);
  cudaFreeHost(D.done);
  cudaFreeHost(D.status);
  cudaFreeHost(D.stop);
  cudaFreeHost(D.defer);
  cudaFree(D.d_dsrc);
  cudaFree(D.d_dout);
  cudaFree(D.d_dcnt);
  if (D.shadow) lp::destroy_shadow(D.shadow);
  cudaFree(D.d_head);
  cudaFree(D.d_finished);
  D = DevLoop();
}

template <typename T>
cudaError_t mapped(T** host, size_t count, T** dev) {
  cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(host), sizeof(T) * (count ? count : 1),
                                cudaHostAllocMapped);
  if (e != cudaSuccess) return e;
  std::memset(*host, 0, sizeof(T) * (count ? count : 1));
  return cudaHostGetDevicePointer(reinterpret_cast<void**>(dev), *host, 0);
}

cudaError_t dev_open(lp_server* S) {
  DevLoop& D = S->dev;
  const lp::Graph& g = *S->base;
  D.pool_cap = (long long)S->opts.max_batch_sources * S->opts.slots;
  D.ring_cap = D.pool_cap;
  D.nslots = std::min(S->opts.max_pending, 65536);
  lp::SrvArgs& A = D.args;
  int2* ring_d = nullptr;
  unsigned long long* tail_d = nullptr;
  lp::SrvReq* reqs_d = nullptr;
  int* src_d = nullptr;
  lp_link* out_d = nullptr;
  unsigned *done_d = nullptr, *status_d = nullptr, *stop_d = nullptr;
  unsigned char* defer_d = nullptr;
  cudaError_t e = mapped(&D.ring, (size_t)D.ring_cap, &ring_d);
  if (e == cudaSuccess) e = mapped(&D.tail, 1, &tail_d);
  if (e == cudaSuccess) e = mapped(&D.reqs, (size_t)D.nslots, &reqs_d);
  if (e == cudaSuccess) e = mapped(&D.src_pool, (size_t)D.pool_cap, &src_d);
  if (e == cudaSuccess) e = mapped(&D.out_pool, (size_t)D.pool_cap * S->opts.max_k, &out_d);
  if (e == cudaSuccess) e = mapped(&D.done, (size_t)D.nslots, &done_d);
  if (e == cudaSuccess) e = mapped(&D.status, 1, &status_d);
  if (e == cudaSuccess) e = mapped(&D.stop, 1, &stop_d);
  if (e == cudaSuccess) e = mapped(&D.defer, (size_t)D.pool_cap, &defer_d);
  const size_t nd = (size_t)S->opts.max_batch_sources;
  if (e == cudaSuccess) e = cudaMalloc(&D.d_dsrc, sizeof(int) * nd);
  if (e == cudaSuccess) e = cudaMalloc(&D.d_dout, sizeof(lp_link) * nd * S->opts.max_k);
  if (e == cudaSuccess) e = cudaMalloc(&D.d_dcnt, sizeof(int) * nd);
  if (e == cudaSuccess && lp::make_shadow(g, &D.shadow) != LP_OK) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMalloc(&D.d_head, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&D.d_finished, sizeof(unsigned long long) * D.nslots);
  if (e == cudaSuccess) e = cudaMemset(D.d_head, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(D.d_finished, 0, sizeof(unsigned long long) * D.nslots);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&D.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  A.off = g.d_off;
  A.idx = g.d_idx;
  A.deg = g.d_deg;
  A.arc = g.d_arc;
  A.wt = g.d_wt;
  A.n = g.n;
  A.dmax = g.dmax;
  A.fixbits = g.fixbits;
  A.idle_polls = S->opts.idle_polls;
  A.ring = ring_d;
  A.ring_cap = (unsigned long long)D.ring_cap;
  A.tail = tail_d;
  A.head = D.d_head;
  A.reqs = reqs_d;
  A.src_pool = src_d;
  A.out_pool = out_d;
  A.finished = D.d_finished;
  A.done = done_d;
  A.status = status_d;
  A.stop = stop_d;
  A.defer = defer_d;
  A.defer_wedges = (unsigned long long)S->opts.defer_wedges;
  D.slot_total.assign(D.nslots, 0);
  D.free_slots.clear();
  for (int i = D.nslots - 1; i >= 0; --i) D.free_slots.push_back(i);
  D.pool.init(D.pool_cap);
  return cudaSuccess;
}

// S->mu held in every helper below.

// Launch the resident kernel if work is outstanding and it is not running.
// The longest the resident kernel runs while deferred rows wait.
constexpr std::chrono::milliseconds kDeferPeriod(10);

void dev_ensure_running(lp_server* S) {
  DevLoop& D = S->dev;
  const bool work = D.published != D.retired;
  const auto now = std::chrono::steady_clock::now();
  if (D.running) {
    const cudaError_t q = cudaStreamQuery(D.stream);
    if (q == cudaErrorNotReady) {
      // deferred sources waiting for the tiered pipeline: once the kernel
      // has run for kDeferPeriod it gives the GPU up to them (its CTAs leave
      // after their current source); the pipeline runs while no kernel does
      if (!D.dq.empty() && !D.stopping && now - D.launched_at >= kDeferPeriod) {
        __atomic_store_n(D.stop, 1u, __ATOMIC_RELEASE);
        D.stopping = true;
        return;
      }
      // the kernel leaves as a whole: after idle_polls x 4 us with no work
      // outstanding the host sets the stop word, and clears it only once the
      // kernel has ended (new work waits for the next launch)
      if (work) {
        D.idle_seen = false;
      } else if (!D.stopping) {
        if (!D.idle_seen) {
          D.idle_seen = true;
          D.idle_since = now;
        } else if (now - D.idle_since >
                   std::chrono::microseconds(4ll * S->opts.idle_polls)) {
          __atomic_store_n(D.stop, 1u, __ATOMIC_RELEASE);
          D.stopping = true;
        }
      }
      return;
    }
    D.running = false;
    D.idle_seen = false;
    if (D.stopping) {
      __atomic_store_n(D.stop, 0u, __ATOMIC_RELEASE);
      D.stopping = false;
    }
    S->cv_work.notify_all();  // the deferred thread waits for the kernel to end
    if (q != cudaSuccess) {
      cudaGetLastError();
      __atomic_store_n(D.status, 2u, __ATOMIC_RELEASE);  // the kernel failed
      return;
    }
  }
  // no launch while the deferred thread runs a batch or is about to start one
  if (!work || D.dbusy || !D.dq.empty() || __atomic_load_n(D.status, __ATOMIC_ACQUIRE) != 0)
    return;
  if (lp::launch_serve(D.args, S->opts.max_k, D.stream) == cudaSuccess) {
    D.running = true;
    D.launched_at = now;
    S->stats.kernel_launches += 1;
  } else {
    cudaGetLastError();
    __atomic_store_n(D.status, 2u, __ATOMIC_RELEASE);
  }
}

// Admit r if a slot, its pool room and ring room are free: write its
// parameters, sources and work items, then publish.
bool dev_admit(lp_server* S, Request* r) {
  DevLoop& D = S->dev;
  const long long n = (long long)r->sources.size();
  if (D.free_slots.empty()) return false;
  if ((long long)(D.published - D.retired) + n > D.ring_cap) return false;
  const long long off = D.pool.take(n);
  if (off < 0) return false;
  const int slot = D.free_slots.back();
  D.free_slots.pop_back();
  r->slot = slot;
  r->off = off;
  r->seq = D.next_seq++;
  if (D.next_seq == 0) D.next_seq = 1;
  std::memcpy(D.src_pool + off, r->sources.data(), sizeof(int32_t) * n);
  D.slot_total[slot] += n;
  lp::SrvReq q;
  q.measure = r->measure;
  q.cap = r->cap;
  q.k = r->k;
  q.n_src = (int)n;
  q.src_off = off;
  q.out_off = off * S->opts.max_k;
  q.target = D.slot_total[slot];
  q.seq = r->seq;
  q.pad = 0;
  D.reqs[slot] = q;
  for (long long i = 0; i < n; ++i)
    D.ring[(D.published + (unsigned long long)i) % (unsigned long long)D.ring_cap] =
        make_int2(slot, (int)i);
  D.published += (unsigned long long)n;
  __atomic_store_n(D.tail, D.published, __ATOMIC_RELEASE);  // everything above first
  r->admitted = true;
  D.inflight.push_back(r);
  S->stats.batches += 1;
  S->stats.batched_sources += n;
  S->stats.max_batch_requests =
      std::max<int64_t>(S->stats.max_batch_requests, (int64_t)D.inflight.size());
  return true;
}

// The deferred rows: requests whose device part is collected wait in D.dq;
// this thread takes every waiting request of the first one's (measure, hub
// limit, k), up to max_batch_sources deferred sources, runs them as one
// tiered per-source batch (lp_predict_sources semantics) and completes them.
void dev_deferred_main(lp_server* S) {
  DevLoop& D = S->dev;
  cudaSetDevice(S->base->device);
  std::vector<Request*> batch;
  std::vector<int> srcs;
  for (;;) {
    batch.clear();
    srcs.clear();
    {
      std::unique_lock<std::mutex> lock(S->mu);
      // a batch starts when no resident kernel runs (it gives the GPU up)
      S->cv_work.wait(lock, [&] { return D.dstop || (!D.dq.empty() && !D.running); });
      if (D.dq.empty()) return;  // stopped and drained
      Request* first = D.dq.front();
      for (auto it = D.dq.begin(); it != D.dq.end();) {
        Request* r = *it;
        if (r->measure == first->measure && r->cap == first->cap && r->k == first->k &&
            (batch.empty() || srcs.size() + r->deferred.size() <=
                                  (size_t)S->opts.max_batch_sources)) {
          for (int j : r->deferred) srcs.push_back(r->sources[j]);
          batch.push_back(r);
          it = D.dq.erase(it);
        } else {
          ++it;
        }
      }
      D.dbusy = true;
    }
    const int nd = (int)srcs.size(), k = first_k(batch);
    D.h_dout.resize((size_t)nd * k);
    D.h_dcnt.resize(nd);
    cudaStream_t ds = D.shadow->stream;
    lp_status ps = LP_OK;
    for (int at = 0; at < nd && ps == LP_OK; at += S->opts.max_batch_sources) {
      const int m = std::min(nd - at, S->opts.max_batch_sources);
      cudaError_t e = cudaMemcpyAsync(D.d_dsrc, srcs.data() + at, sizeof(int) * m,
                                      cudaMemcpyHostToDevice, ds);
      if (e != cudaSuccess) ps = lp::report_cuda(e, "serving: deferred sources");
      if (ps == LP_OK)
        ps = lp::run_sources_dev(*D.shadow, batch[0]->measure, batch[0]->cap, D.d_dsrc, m, k, 0.0,
                                 D.d_dout, D.d_dcnt);
      if (ps == LP_OK) {
        e = cudaMemcpyAsync(D.h_dout.data() + (size_t)at * k, D.d_dout, sizeof(lp_link) * m * k,
                            cudaMemcpyDeviceToHost, ds);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(D.h_dcnt.data() + at, D.d_dcnt, sizeof(int) * m,
                              cudaMemcpyDeviceToHost, ds);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ds);
        if (e != cudaSuccess) ps = lp::report_cuda(e, "serving: deferred rows");
      }
    }
    const std::string error = ps == LP_OK ? std::string() : std::string(lp_last_error());
    {
      std::lock_guard<std::mutex> lock(S->mu);
      int q = 0;
      for (Request* r : batch) {
        for (int j : r->deferred) {
          if (ps == LP_OK) {
            std::memcpy(r->out.data() + (size_t)j * k, D.h_dout.data() + (size_t)q * k,
                        sizeof(lp_link) * k);
            r->counts[j] = D.h_dcnt[q];
          }
          ++q;
        }
        if (ps != LP_OK) {
          r->status = ps;
          r->error = error;
        }
        r->done = true;
        S->stats.completed += 1;
      }
      S->stats.deferred_sources += nd;
      D.dbusy = false;
    }
    S->cv_done.notify_all();
  }
}

// Collect finished requests (copy their rows out, free their memory), then
// admit waiting requests in arrival order while they fit.
void dev_harvest(lp_server* S) {
  DevLoop& D = S->dev;
  const unsigned st = __atomic_load_n(D.status, __ATOMIC_ACQUIRE);
  bool any = false;
  for (size_t i = 0; i < D.inflight.size();) {
    Request* r = D.inflight[i];
    const bool fin = __atomic_load_n(D.done + r->slot, __ATOMIC_ACQUIRE) == r->seq;
    if (!fin && st == 0) {
      ++i;
      continue;
    }
    const size_t n = r->sources.size(), k = (size_t)r->k;
    if (fin && st == 0) {
      r->out.resize(n * k);
      r->counts.resize(n);
      const lp_link* base = D.out_pool + (size_t)r->off * S->opts.max_k;
      r->deferred.clear();
      for (size_t j = 0; j < n; ++j) {
        if (D.defer[r->off + j]) {  // left to the tiered pipeline (dev_deferred_main)
          D.defer[r->off + j] = 0;
          r->deferred.push_back((int)j);
          continue;
        }
        std::memcpy(r->out.data() + j * k, base + j * k, sizeof(lp_link) * k);
        int c = 0;
        while (c < (int)k && r->out[j * k + c].v >= 0) ++c;
        r->counts[j] = c;
      }
      r->status = LP_OK;
    } else {
      r->status = st == 2 ? LP_ECUDA : LP_EINTERNAL;
      r->error = st == 2 ? "the resident serving kernel failed" : "serving: device check failed";
    }
    if (r->deferred.empty()) {
      r->done = true;
      S->stats.completed += 1;
    } else {
      D.dq.push_back(r);  // done when the deferred rows are in
      S->cv_work.notify_all();
    }
    if (fin) {  // the slot and the pool room are free again
      D.pool.give(r->off, (long long)n);
      D.free_slots.push_back(r->slot);
      D.retired += (unsigned long long)n;
    }
    D.inflight[i] = D.inflight.back();
    D.inflight.pop_back();
    any = true;
  }
  while (!S->paused && st == 0 && !D.waiting.empty() && dev_admit(S, D.waiting.front()))
    D.waiting.pop_front();
  dev_ensure_running(S);
  if (any) S->cv_done.notify_all();
}

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
  if (o.idle_polls == 0) o.idle_polls = 2500;
  if (o.defer_wedges == 0) o.defer_wedges = 65536;
  if (o.slots < 1 || o.slots > 8 || o.max_batch_sources < 1 || o.max_pending < 1 || o.max_k < 1 ||
      o.max_k > LP_MAX_TOPK_PER_SOURCE || o.mode < 0 || o.mode > 1 || o.idle_polls < 1 ||
      o.defer_wedges < 1)
    return serve_fail(LP_EINVAL, "lp_serve_open: option out of range");
  lp_server* S = new (std::nothrow) lp_server();
  if (!S) return serve_fail(LP_ENOMEM, "lp_serve_open: host allocation");
  S->g = g;
  S->base = &lp::graph_of(g);
  S->opts = o;
  S->paused = o.paused != 0;
  if (o.mode == kResident) {
    cudaError_t e = cudaSetDevice(S->base->device);
    if (e == cudaSuccess) e = dev_open(S);
    if (e != cudaSuccess) {
      dev_free(S->dev);
      delete S;
      return lp::report_cuda(e, "lp_serve_open");
    }
    S->dev.dthread = std::thread(dev_deferred_main, S);
    *out = S;
    return LP_OK;
  }
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
  if (S->opts.mode == kResident) {
    std::lock_guard<std::mutex> lock(S->mu);
    DevLoop& D = S->dev;
    if (S->closing) {
      delete r;
      return serve_fail(LP_EINVAL, "lp_serve_submit: server is closing");
    }
    if ((int64_t)(D.waiting.size() + D.inflight.size()) >= S->opts.max_pending) {
      delete r;
      return serve_fail(LP_EBUSY, "lp_serve_submit: queue full");
    }
    cudaSetDevice(S->base->device);
    r->id = S->next_id++;
    S->live[r->id] = r;
    S->stats.submitted += 1;
    *req_id = r->id;
    D.waiting.push_back(r);
    dev_harvest(S);  // frees finished requests' memory, admits in arrival order
    return LP_OK;
  }
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
  if (S->opts.mode == kResident) {
    // poll: collect finished requests and keep the resident kernel running
    cudaSetDevice(S->base->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      dev_harvest(S);
      if (r->done) break;
      if (timeout_us >= 0 &&
          std::chrono::steady_clock::now() - t0 >= std::chrono::microseconds(timeout_us))
        return serve_fail(LP_ETIMEOUT, "lp_serve_wait: request not finished in time");
      S->cv_done.wait_for(lock, std::chrono::microseconds(20), [&] { return r->done; });
    }
  } else if (timeout_us < 0) {
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
    if (S->opts.mode == kResident) {
      cudaSetDevice(S->base->device);
      dev_harvest(S);
    }
  }
  S->cv_work.notify_all();
  return LP_OK;
}

lp_status lp_serve_poll(lp_server* S, uint64_t req_id, int32_t* done) {
  if (!S || !done) return serve_fail(LP_EINVAL, "lp_serve_poll: null argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->live.find(req_id);
  if (it == S->live.end()) return serve_fail(LP_EINVAL, "lp_serve_poll: unknown request id");
  if (S->opts.mode == kResident) {
    cudaSetDevice(S->base->device);
    dev_harvest(S);
  }
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
  if (S->opts.mode == kResident) {
    std::unique_lock<std::mutex> lock(S->mu);
    cudaSetDevice(S->base->device);
    S->closing = true;
    S->paused = false;
    DevLoop& D = S->dev;
    for (;;) {  // finish every queued request, deferred rows included
      dev_harvest(S);
      bool all_done = true;
      for (auto& kv : S->live) all_done = all_done && kv.second->done;
      if (all_done || (D.inflight.empty() && D.dq.empty() &&
                       __atomic_load_n(D.status, __ATOMIC_ACQUIRE) != 0))
        break;
      S->cv_done.wait_for(lock, std::chrono::microseconds(50));
    }
    __atomic_store_n(D.stop, 1u, __ATOMIC_RELEASE);  // idle CTAs leave at once
    D.dstop = true;
    lock.unlock();
    S->cv_work.notify_all();
    if (D.dthread.joinable()) D.dthread.join();
    dev_free(D);
    for (auto& kv : S->live) delete kv.second;
    S->live.clear();
    delete S;
    return LP_OK;
  }
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
