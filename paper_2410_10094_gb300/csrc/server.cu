// A contraction server: requests (each one stc_contract's arguments) are queued, counted, admitted
// against a device-memory budget by their exact bound (the product count of Section 4.3
// gives the output bound before any product is formed), and run in batches by worker
// threads, each on its own stream, so that batches overlap on the device. Submission only
// queues a request: a counting thread runs the counting pass of each request in arrival order
// on its own stream and hands it to the admission queue (one counting thread per worker,
// taking requests in arrival order). Requests that arrive while batches
// are running join the next batch of a free worker (continuous batching). With `plain` set the
// server runs one request at a time with stc_contract on one worker: the one-at-a-time
// baseline on the same arrival trace.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "launch.h"

namespace stc {
stc_status report_error(stc_status s, const char* msg);
int ctx_device(const stc_ctx* ctx);
void result_release_on_default_stream(stc_result* r);
}
using namespace stc;

namespace {

using Clock = std::chrono::steady_clock;

// Requests with more products than this run as plain contractions even in batched mode.
constexpr uint64_t kServerAloneProducts = 1ull << 24;

struct Ticket {
  stc_problem req{};
  std::vector<int64_t> xshape, yshape;
  std::vector<int32_t> cx, cy, oo;
  bool has_oo = false;
  uint64_t bytes = 0;  // admission bound
  uint64_t products = 0;  // exact product count
  bool alone = false;     // runs as a plain contraction (its contract keys need renumbering)
  bool counting = false;  // its counting pass is running
  bool cancel = false;    // cancelled during its counting pass: finished when that pass ends
  bool done = false;
  stc_status status = STC_OK;
  std::string error;
  stc_result* result = nullptr;
  double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct stc_server {
  stc_ctx* ctx = nullptr;
  stc_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;     // counted, waiting for admission
  std::deque<uint64_t> pending;   // submitted, waiting for the counting pass
  std::condition_variable cv_count;
  std::vector<std::thread> counters;  // counting threads, one per worker
  std::map<uint64_t, Ticket> tickets;
  uint64_t next_ticket = 1;
  uint64_t reserved = 0;
  int running_batches = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::vector<cudaStream_t> count_streams;
  Clock::time_point epoch;
  double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }
};

namespace {

// Copies the host-side parts of a request (shapes, mode lists) so the caller's arrays may go.
void own_request(Ticket& t, const stc_problem& r) {
  t.req = r;
  t.xshape.assign(r.X.shape, r.X.shape + r.X.order);
  t.yshape.assign(r.Y.shape, r.Y.shape + r.Y.order);
  t.cx.assign(r.cx, r.cx + r.ncontract);
  t.cy.assign(r.cy, r.cy + r.ncontract);
  t.req.X.shape = t.xshape.data();
  t.req.Y.shape = t.yshape.data();
  t.req.cx = t.cx.data();
  t.req.cy = t.cy.data();
  if (r.out_order) {
    const int oz = (r.X.order - r.ncontract) + (r.Y.order - r.ncontract);
    t.oo.assign(r.out_order, r.out_order + (oz > 0 ? oz : 0));
    t.req.out_order = t.oo.data();
    t.has_oo = true;
  }
}

// A counting thread: the exact product count and memory bound of the submitted requests it
// takes (in arrival order), then admission.
void counter_main(stc_server* sv, int c) {
  cudaStream_t cs = sv->count_streams[c];
  cudaSetDevice(ctx_device(sv->ctx));
  for (;;) {
    uint64_t id = 0;
    stc_problem req{};
    // The request's host arrays are copied: a cancelled ticket may be consumed by its wait
    // while its counting pass still runs.
    std::vector<int64_t> xs, ys;
    std::vector<int32_t> cx, cy;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_count.wait(lk, [&] { return sv->stopping || !sv->pending.empty(); });
      if (sv->pending.empty()) return;  // stopping and drained
      id = sv->pending.front();
      sv->pending.pop_front();
      Ticket& t = sv->tickets[id];
      t.counting = true;
      req = t.req;
      xs = t.xshape;
      ys = t.yshape;
      cx = t.cx;
      cy = t.cy;
      req.X.shape = xs.data();
      req.Y.shape = ys.data();
      req.cx = cx.data();
      req.cy = cy.data();
      req.out_order = nullptr;
    }
    uint64_t P = 0, bytes = 0;
    const stc_status st = stc_count(sv->ctx, &req.X, &req.Y, req.ncontract, req.cx, req.cy, cs, &P,
                                     &bytes);
    const std::string err = st == STC_OK ? std::string() : std::string(stc_last_error());
    // The batched launch groups Y by contract key directly; a key space above 2^26 is
    // renumbered to dense ids by the plain path only.
    unsigned __int128 K = 1;
    for (int32_t i = 0; i < req.ncontract; i++) {
      K *= (unsigned __int128)req.X.shape[req.cx[i]];
      if (K > ((unsigned __int128)1 << 26)) break;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      auto it = sv->tickets.find(id);
      if (it == sv->tickets.end() || it->second.done) continue;
      Ticket& t = it->second;
      t.counting = false;
      if (t.cancel) {  // cancelled while it was counted: its arrays are no longer read
        t.done = true;
        t.status = STC_ERR_CANCELLED;
        t.error = "the request was cancelled before it ran";
        t.t_start = t.t_done = sv->now();
      } else if (st != STC_OK) {
        t.done = true;
        t.status = st;
        t.error = err;
        t.t_start = t.t_done = sv->now();
      } else {
        t.bytes = bytes;
        t.products = P;
        t.alone = K > ((unsigned __int128)1 << 26);
        sv->queue.push_back(id);
      }
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_one();
  }
}

void worker_main(stc_server* sv, int w) {
  cudaStream_t s = sv->streams[w];
  cudaSetDevice(ctx_device(sv->ctx));
  for (;;) {
    std::vector<uint64_t> batch;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] { return sv->stopping || !sv->queue.empty(); });
      if (sv->queue.empty()) return;  // stopping and drained
      // Take queued requests in arrival order while they fit the budget; a request larger
      // than the whole budget runs alone once nothing else is reserved.
      const uint64_t budget = sv->opts.mem_budget_bytes;
      const int maxb = sv->opts.plain ? 1 : (sv->opts.max_batch > 0 ? sv->opts.max_batch : 1 << 30);
      while (!sv->queue.empty() && (int)batch.size() < maxb) {
        Ticket& t = sv->tickets[sv->queue.front()];
        const bool fits = budget == 0 || sv->reserved + t.bytes <= budget || (sv->reserved == 0 && batch.empty());
        if (!fits) break;
        sv->reserved += t.bytes;
        batch.push_back(sv->queue.front());
        sv->queue.pop_front();
      }
      if (batch.empty()) {
        // Nothing fits until memory is released: wait for a batch to finish.
        sv->cv_work.wait(lk, [&] { return sv->stopping || sv->running_batches == 0 || sv->reserved == 0; });
        continue;
      }
      sv->running_batches++;
      const double t0 = sv->now();
      for (uint64_t id : batch) sv->tickets[id].t_start = t0;
    }
    // Run the batch (outside the lock).
    std::vector<stc_problem> probs;
    probs.reserve(batch.size());
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (uint64_t id : batch) probs.push_back(sv->tickets[id].req);
    }
    std::vector<stc_result*> outs(batch.size(), nullptr);
    stc_status st = STC_OK;
    std::string err;
    // Requests large enough to fill the GPU alone (and a request that is alone in its batch)
    // run as plain contractions; the others share one batched launch sequence.
    std::vector<uint64_t> prods(batch.size());
    std::vector<char> lone(batch.size());
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (size_t k = 0; k < batch.size(); k++) {
        prods[k] = sv->tickets[batch[k]].products;
        lone[k] = sv->tickets[batch[k]].alone;
      }
    }
    std::vector<size_t> small, alone;
    for (size_t k = 0; k < batch.size(); k++)
      (sv->opts.plain || lone[k] || prods[k] > kServerAloneProducts ? alone : small).push_back(k);
    if (small.size() == 1) {
      alone.insert(alone.begin(), small[0]);
      small.clear();
    }
    if (!small.empty()) {
      std::vector<stc_problem> sp;
      std::vector<stc_result*> so(small.size(), nullptr);
      for (size_t k : small) sp.push_back(probs[k]);
      stc_opts o{};
      o.strategy = STC_STRATEGY_GROUPED;
      st = stc_contract_batch(sv->ctx, (int32_t)sp.size(), sp.data(), &o, s, so.data());
      for (size_t i = 0; i < small.size(); i++) outs[small[i]] = so[i];
    }
    for (size_t k : alone) {
      if (st != STC_OK) break;
      const stc_problem& q = probs[k];
      st = stc_contract(sv->ctx, &q.X, &q.Y, q.ncontract, q.cx, q.cy, q.out_order, nullptr, s, &outs[k]);
    }
    if (st != STC_OK) {
      // The whole take fails together; results already made are returned.
      err = stc_last_error();
      for (stc_result*& r : outs) {
        if (r) stc_result_free(r);
        r = nullptr;
      }
    }
    for (stc_result* r : outs) result_release_on_default_stream(r);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      const double t1 = sv->now();
      for (size_t k = 0; k < batch.size(); k++) {
        Ticket& t = sv->tickets[batch[k]];
        t.done = true;
        t.status = st;
        t.error = err;
        t.result = outs[k];
        t.t_done = t1;
        sv->reserved -= t.bytes;
      }
      sv->running_batches--;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

stc_status stc_server_create(stc_ctx* ctx, const stc_server_opts* opts, stc_server** out) {
  if (!ctx || !out) return report_error(STC_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  stc_server* sv = new stc_server;
  sv->ctx = ctx;
  if (opts) sv->opts = *opts;
  if (sv->opts.workers <= 0) sv->opts.workers = sv->opts.plain ? 1 : 2;
  if (sv->opts.plain) sv->opts.workers = 1;
  sv->epoch = Clock::now();
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx_device(ctx)) {
    delete sv;
    return report_error(STC_ERR_INVALID_ARG, "the current device is not the context's device");
  }
  for (int w = 0; w < 2 * sv->opts.workers; w++) {
    cudaStream_t s = nullptr;
    const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto x : sv->streams) cudaStreamDestroy(x);
      for (auto x : sv->count_streams) cudaStreamDestroy(x);
      delete sv;
      return report_error(STC_ERR_CUDA, cudaGetErrorString(e));
    }
    (w < sv->opts.workers ? sv->streams : sv->count_streams).push_back(s);
  }
  for (int w = 0; w < sv->opts.workers; w++) sv->workers.emplace_back(worker_main, sv, w);
  for (int c = 0; c < sv->opts.workers; c++) sv->counters.emplace_back(counter_main, sv, c);
  *out = sv;
  return STC_OK;
}

stc_status stc_server_submit(stc_server* sv, const stc_problem* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return report_error(STC_ERR_INVALID_ARG, "NULL argument");
  const double t_arrive = sv->now();
  Ticket t;
  own_request(t, *req);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stopping) return report_error(STC_ERR_INVALID_ARG, "server is shutting down");
  const uint64_t id = sv->next_ticket++;
  t.t_submit = t_arrive;
  sv->tickets.emplace(id, std::move(t));
  // Re-point the copied host arrays at the map's copy.
  Ticket& tt = sv->tickets[id];
  tt.req.X.shape = tt.xshape.data();
  tt.req.Y.shape = tt.yshape.data();
  tt.req.cx = tt.cx.data();
  tt.req.cy = tt.cy.data();
  tt.req.out_order = tt.has_oo ? tt.oo.data() : nullptr;
  sv->pending.push_back(id);
  *ticket = id;
  sv->cv_count.notify_one();
  return STC_OK;
}

stc_status stc_server_poll(stc_server* sv, uint64_t ticket, int32_t* done) {
  if (!sv || !done) return report_error(STC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return report_error(STC_ERR_INVALID_ARG, "unknown ticket");
  *done = it->second.done ? 1 : 0;
  return STC_OK;
}

stc_status stc_server_wait(stc_server* sv, uint64_t ticket, int64_t timeout_ms, stc_result** out,
                           double* times) {
  if (!sv || !out) return report_error(STC_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->tickets.find(ticket);
  if (it == sv->tickets.end()) return report_error(STC_ERR_INVALID_ARG, "unknown ticket");
  const auto pred = [&] { return sv->tickets[ticket].done; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, pred);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    return report_error(STC_ERR_TIMEOUT, "request not finished within the timeout");
  }
  Ticket t = std::move(sv->tickets[ticket]);
  sv->tickets.erase(ticket);
  if (times) {
    times[0] = t.t_submit;
    times[1] = t.t_start;
    times[2] = t.t_done;
  }
  if (t.status != STC_OK) return report_error(t.status, t.error.c_str());
  *out = t.result;
  return STC_OK;
}

stc_status stc_server_cancel(stc_server* sv, uint64_t ticket, int32_t* cancelled) {
  if (!sv || !cancelled) return report_error(STC_ERR_INVALID_ARG, "NULL argument");
  *cancelled = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return report_error(STC_ERR_INVALID_ARG, "unknown ticket");
    Ticket& t = it->second;
    if (t.done) return STC_OK;
    // Only a request no worker has taken is still queued (it holds no reservation yet): in the
    // admission queue or in the counting queue; one being counted is finished by the counting
    // thread when its pass ends (its wait returns only then, its arrays no longer in use).
    if (t.counting) {
      t.cancel = true;
      *cancelled = 1;
      return STC_OK;
    }
    bool taken = true;
    for (auto* dq : {&sv->queue, &sv->pending}) {
      for (auto q = dq->begin(); q != dq->end(); ++q) {
        if (*q != ticket) continue;
        dq->erase(q);
        taken = false;
        break;
      }
    }
    if (!taken) {
      t.done = true;
      t.status = STC_ERR_CANCELLED;
      t.error = "the request was cancelled before it ran";
      t.t_start = t.t_done = sv->now();
      *cancelled = 1;
    }
  }
  if (*cancelled) sv->cv_done.notify_all();
  return STC_OK;
}

stc_status stc_server_destroy(stc_server* sv) {
  if (!sv) return STC_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  // The counting threads drain the counting queue first, then the workers drain the rest.
  sv->cv_count.notify_all();
  for (auto& th : sv->counters) th.join();
  sv->cv_work.notify_all();
  for (auto& th : sv->workers) th.join();
  // Results nobody collected are freed here.
  for (auto& kv : sv->tickets)
    if (kv.second.result) stc_result_free(kv.second.result);
  for (auto s : sv->streams) cudaStreamDestroy(s);
  for (auto s : sv->count_streams) cudaStreamDestroy(s);
  delete sv;
  return STC_OK;
}

}  // extern "C"
