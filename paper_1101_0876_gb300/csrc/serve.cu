// Serving loop: continuous batching of simulation requests on one GPU.
//
// A host thread owns an Engine.  Each iteration it (1) admits queued
// requests, oldest first, while a slot is free and the device bytes in use
// plus the request's planes fit the budget, allocating and initialising
// their lattices; (2) drops cancelled requests; (3) runs one batched step of
// up to sweeps_per_step sweeps over every active lattice; (4) appends each
// lattice's new per-sweep records to its request's outbox and retires the
// lattices that are done, freeing their slot and memory.  Clients talk to
// the loop only through the mutex-protected queue and outboxes
// (potts_serve_submit / poll / cancel), which never block on the GPU.
#include <atomic>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "engine.cuh"

using namespace potts;

namespace {

enum class ReqState { Queued, Active, Done, Cancelled, Failed };

struct Request {
  uint64_t id = 0;
  potts_req r{};
  ReqState state = ReqState::Queued;
  Member m;
  int64_t remaining = 0;       // sweeps still to run
  std::vector<uint64_t> outbox;  // ready records, flattened
  size_t outbox_head = 0;      // first record not yet polled (in u64)
  bool cancel_requested = false;
  int error = POTTS_OK;
};

}  // namespace

struct potts_server {
  potts_serve_cfg cfg{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, Request *> all;
  std::vector<Request *> active;
  Engine eng;
  cudaStream_t st = nullptr;
  int device = 0;
  uint64_t next_id = 1;
  potts_serve_stats stats{};
  int loop_error = POTTS_OK;
  std::string loop_msg;

  static uint64_t bytes_of(const potts_req &r) {
    return (uint64_t)r.L * (uint64_t)r.L;
  }

  void retire(Request *q, ReqState s) {
    eng.free_member(&q->m);
    stats.bytes_in_use -= bytes_of(q->r);
    q->state = s;
  }

  void run() {
    cudaSetDevice(device);
    std::vector<Member *> members;
    for (;;) {
      std::vector<Request *> admit;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait_for(lk, std::chrono::milliseconds(50), [&] {
          return stop || !queue.empty() || !active.empty();
        });
        if (stop) break;
        // cancellations of queued and active requests
        for (auto it = queue.begin(); it != queue.end();) {
          if ((*it)->cancel_requested) {
            (*it)->state = ReqState::Cancelled;
            stats.cancelled += 1;
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
        // admission: FIFO, by slot and by HBM budget
        while (!queue.empty() &&
               (int32_t)(active.size() + admit.size()) < cfg.max_slots) {
          Request *q = queue.front();
          const uint64_t b = bytes_of(q->r);
          if (stats.bytes_in_use + b > cfg.hbm_budget_bytes) break;
          queue.pop_front();
          stats.bytes_in_use += b;
          admit.push_back(q);
        }
      }
      // allocate + initialise outside the lock
      for (Request *q : admit) {
        q->m.L = q->r.L;
        q->m.q = q->r.q;
        q->m.start = q->r.start;
        q->m.seed = q->r.seed;
        q->m.beta = q->r.beta;
        q->remaining = q->r.nsweeps;
        int rc = eng.create_member(&q->m);
        std::lock_guard<std::mutex> lk(mu);
        if (rc != POTTS_OK) {
          q->error = rc;
          stats.bytes_in_use -= bytes_of(q->r);
          q->state = ReqState::Failed;
          continue;
        }
        q->state = ReqState::Active;
        stats.admitted += 1;
        active.push_back(q);
      }
      bool changed = !admit.empty();
      {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < active.size();) {
          Request *q = active[i];
          if (q->cancel_requested || q->remaining == 0) {
            if (q->cancel_requested) stats.cancelled += 1;
            else stats.completed += 1;
            retire(q, q->cancel_requested ? ReqState::Cancelled
                                          : ReqState::Done);
            active.erase(active.begin() + (int64_t)i);
            changed = true;
          } else {
            ++i;
          }
        }
        stats.active = (int32_t)active.size();
        stats.queued = (int32_t)queue.size();
      }
      if (active.empty()) continue;
      const int32_t k = std::max(1, cfg.sweeps_per_step);
      if (changed) {
        members.clear();
        for (Request *q : active) members.push_back(&q->m);
        eng.set_members(members);
      }
      for (Request *q : active)
        q->m.nsweeps_step = (int32_t)std::min<int64_t>(q->remaining, k);
      const int rc = eng.step(k);
      std::lock_guard<std::mutex> lk(mu);
      if (rc != POTTS_OK) {
        loop_error = rc;
        loop_msg = potts_last_error();
        for (Request *q : active) {
          q->error = rc;
          retire(q, ReqState::Failed);
        }
        active.clear();
        members.clear();
        eng.set_members(members);
        continue;
      }
      stats.steps += 1;
      for (Request *q : active) {
        const int32_t n = q->m.nsweeps_step;
        const uint64_t *rec = eng.records(&q->m);
        q->outbox.insert(q->outbox.end(), rec, rec + (size_t)n * (1 + q->r.q));
        q->remaining -= n;
        stats.sweeps_done += (uint64_t)n;
        stats.updates_done += (uint64_t)n * (uint64_t)q->r.L * (uint64_t)q->r.L;
      }
      cv.notify_all();
    }
    // shutdown: free everything still held
    std::lock_guard<std::mutex> lk(mu);
    for (Request *q : active) retire(q, ReqState::Cancelled);
    active.clear();
  }
};

extern "C" {

int potts_serve_start(const potts_serve_cfg *cfg, potts_server_h *out) {
  if (!cfg || !out) return fail(POTTS_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots <= 0 || cfg->sweeps_per_step <= 0 ||
      cfg->hbm_budget_bytes == 0 || cfg->queue_capacity < 0)
    return fail(POTTS_EINVAL, "max_slots, sweeps_per_step and the budget "
                              "must be positive");
  potts_server *s = new (std::nothrow) potts_server();
  if (!s) return fail(POTTS_ENOMEM, "host allocation failed");
  s->cfg = *cfg;
  if (s->cfg.queue_capacity == 0) s->cfg.queue_capacity = 65536;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return fail(POTTS_ECUDA, "server stream: %s", cudaGetErrorString(e));
  }
  int rc = s->eng.init(s->st);
  if (rc != POTTS_OK) {
    cudaStreamDestroy(s->st);
    delete s;
    return rc;
  }
  s->eng.initial_counts = false;
  try {
    s->th = std::thread([s] { s->run(); });
  } catch (...) {
    cudaStreamDestroy(s->st);
    delete s;
    return fail(POTTS_ENOMEM, "could not start the server thread");
  }
  *out = s;
  return POTTS_OK;
}

int potts_serve_submit(potts_server_h s, const potts_req *req,
                       uint64_t *req_id) {
  if (!s || !req || !req_id) return fail(POTTS_EINVAL, "NULL argument");
  const potts_req &r = *req;
  if (r.L < 32 || r.L > 65536 || r.L % 32 != 0)
    return fail(POTTS_EINVAL, "L must be a multiple of 32 in [32, 65536]");
  if (r.q < 2 || r.q > 256) return fail(POTTS_EINVAL, "q must be in [2, 256]");
  if (r.start != POTTS_START_ORDERED && r.start != POTTS_START_RANDOM)
    return fail(POTTS_EINVAL, "start must be 0 or 1");
  if (r.nsweeps < 1) return fail(POTTS_EINVAL, "nsweeps must be >= 1");
  uint64_t thr[5];
  if (!threshold_table(r.beta, thr))
    return fail(POTTS_EINVAL, "beta must be finite and >= 0");
  if (potts_server::bytes_of(r) > s->cfg.hbm_budget_bytes)
    return fail(POTTS_EINVAL, "request needs %llu bytes, over the budget",
                (unsigned long long)potts_server::bytes_of(r));
  Request *q = new (std::nothrow) Request();
  if (!q) return fail(POTTS_ENOMEM, "host allocation failed");
  q->r = r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int32_t)s->queue.size() >= s->cfg.queue_capacity) {
      delete q;
      return fail(POTTS_EBUSY, "request queue is full");
    }
    q->id = s->next_id++;
    s->queue.push_back(q);
    s->all[q->id] = q;
    s->stats.submitted += 1;
    *req_id = q->id;
  }
  s->cv.notify_all();
  return POTTS_OK;
}

int potts_serve_poll(potts_server_h s, uint64_t req_id, uint64_t *out_counts,
                     int64_t max_sweeps, int64_t *n_ready, int *done) {
  if (!s || !n_ready || !done) return fail(POTTS_EINVAL, "NULL argument");
  if (max_sweeps > 0 && !out_counts)
    return fail(POTTS_EINVAL, "out_counts is NULL");
  *n_ready = 0;
  *done = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(req_id);
  if (it == s->all.end()) return fail(POTTS_ENOTFOUND, "unknown request");
  Request *q = it->second;
  const size_t rl = (size_t)(1 + q->r.q);
  const size_t avail = (q->outbox.size() - q->outbox_head) / rl;
  const size_t n = std::min<size_t>(avail, (size_t)std::max<int64_t>(0, max_sweeps));
  if (n) {
    std::memcpy(out_counts, q->outbox.data() + q->outbox_head, n * rl * 8);
    q->outbox_head += n * rl;
    if (q->outbox_head > (1u << 20) && q->outbox_head * 2 > q->outbox.size()) {
      q->outbox.erase(q->outbox.begin(),
                      q->outbox.begin() + (int64_t)q->outbox_head);
      q->outbox_head = 0;
    }
  }
  *n_ready = (int64_t)n;
  const bool drained = q->outbox_head == q->outbox.size();
  int rc = POTTS_OK;
  if (q->state == ReqState::Done && drained) {
    *done = 1;
  } else if (q->state == ReqState::Cancelled) {
    *done = 1;
    rc = fail(POTTS_ECANCELLED, "request was cancelled");
  } else if (q->state == ReqState::Failed) {
    *done = 1;
    rc = fail(q->error ? q->error : POTTS_ECUDA, "request failed: %s",
              s->loop_msg.c_str());
  }
  if (*done) {
    s->all.erase(it);
    delete q;
  }
  return rc;
}

int potts_serve_cancel(potts_server_h s, uint64_t req_id) {
  if (!s) return fail(POTTS_EINVAL, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(req_id);
    if (it == s->all.end()) return fail(POTTS_ENOTFOUND, "unknown request");
    it->second->cancel_requested = true;
  }
  s->cv.notify_all();
  return POTTS_OK;
}

int potts_serve_stats_get(potts_server_h s, potts_serve_stats *out) {
  if (!s || !out) return fail(POTTS_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->active = (int32_t)s->active.size();
  out->queued = (int32_t)s->queue.size();
  return POTTS_OK;
}

int potts_serve_stop(potts_server_h s) {
  if (!s) return fail(POTTS_EINVAL, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  for (auto &kv : s->all) delete kv.second;
  s->all.clear();
  if (s->st) {
    cudaStreamSynchronize(s->st);
    cudaStreamDestroy(s->st);
  }
  int rc = s->loop_error;
  delete s;
  return rc == POTTS_OK ? POTTS_OK : fail(rc, "server loop had failed");
}

}  // extern "C"
