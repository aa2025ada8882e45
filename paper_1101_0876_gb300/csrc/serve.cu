// Serving loop: continuous batching of simulation requests on one GPU.
//
// A host thread owns an Engine.  Each iteration it (1) admits queued
// requests (oldest first, or smallest work first) while a slot is free and
// the device bytes in use plus the request's planes fit the budget,
// allocating and initialising their lattices; (2) drops cancelled
// requests; (3) runs one batched step of up to sweeps_per_step sweeps over
// every active lattice; (4) appends each lattice's new per-sweep records to
// its request's outbox and retires the lattices that are done, freeing
// their slot and memory.  Clients talk to
// the loop only through the mutex-protected queue and outboxes
// (potts_serve_submit / poll / cancel), which never block on the GPU.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "engine.cuh"

using namespace potts;

namespace {

enum class ReqState { Queued, Active, Done, Cancelled, Failed };

struct Request {
  uint64_t id = 0;
  potts_req r{};
  ReqState state = ReqState::Queued;
  Member m;
  int64_t to_launch = 0;       // sweeps not yet launched
  int64_t to_deliver = 0;      // sweeps whose records have not arrived
  bool in_engine = false;      // holds planes and a slot
  std::vector<uint64_t> outbox;  // ready records, flattened
  size_t outbox_head = 0;      // first record not yet polled (in u64)
  bool cancel_requested = false;
  bool forgotten = false;      // the client has seen the final state
  uint64_t last_seq = 0;       // last launch that may reference it
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
  std::vector<Request *> active;   // admitted, in the engine
  std::vector<Request *> retired;  // out of the engine, records in flight
  Engine eng;
  cudaStream_t st = nullptr;
  int device = 0;
  uint64_t next_id = 1;
  uint64_t launch_seq = 0, complete_seq = 0;
  potts_serve_stats stats{};
  int loop_error = POTTS_OK;
  std::string loop_msg;

  static uint64_t bytes_of(const potts_req &r) {
    return (uint64_t)r.L * (uint64_t)r.L;
  }
  // spin updates a request asks for
  static uint64_t work_of(const potts_req &r) {
    return (uint64_t)r.L * (uint64_t)r.L * (uint64_t)r.nsweeps;
  }

  // Leaves the engine: slot and memory are free for the next admission
  // (the stream-ordered free runs after the steps already queued).
  void leave_engine(Request *q) {
    if (!q->in_engine) return;
    eng.free_member(&q->m);
    stats.bytes_in_use -= bytes_of(q->r);
    q->in_engine = false;
    q->last_seq = launch_seq;
  }

  // Deletes retired requests that the client has finished with and that no
  // in-flight step can still reference.
  void reap() {
    retired.erase(std::remove_if(retired.begin(), retired.end(),
                                 [&](Request *q) {
                                   if (q->forgotten &&
                                       complete_seq >= q->last_seq) {
                                     delete q;
                                     return true;
                                   }
                                   return false;
                                 }),
                  retired.end());
  }

  void deliver() {
    const StepRecords &r = eng.last();
    std::lock_guard<std::mutex> lk(mu);
    stats.steps += 1;
    for (size_t i = 0; i < r.mem.size(); ++i) {
      Request *q = static_cast<Request *>(r.mem[i]->user);
      const int32_t n = r.nsw[i];
      if (n <= 0) continue;
      if (q->state == ReqState::Active) {
        const uint64_t *rec = r.base + r.off[i];
        q->outbox.insert(q->outbox.end(), rec, rec + (size_t)n * (1 + q->r.q));
      }
      q->to_deliver -= n;
      stats.sweeps_done += (uint64_t)n;
      stats.updates_done += (uint64_t)n * (uint64_t)q->r.L * (uint64_t)q->r.L;
      if (q->to_deliver == 0 && q->state == ReqState::Active) {
        q->state = ReqState::Done;
        stats.completed += 1;
      }
    }
    reap();
  }

  void run() {
    cudaSetDevice(device);
    std::vector<Member *> members;
    bool changed = true;
    for (;;) {
      std::vector<Request *> admit;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (active.empty() && eng.in_flight() == 0)
          cv.wait_for(lk, std::chrono::milliseconds(50),
                      [&] { return stop || !queue.empty(); });
        if (stop) break;
        for (auto it = queue.begin(); it != queue.end();) {
          if ((*it)->cancel_requested) {
            (*it)->state = ReqState::Cancelled;
            stats.cancelled += 1;
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
        // admission by slot and by HBM budget, in the configured order
        while (!queue.empty() &&
               (int32_t)(active.size() + admit.size()) < cfg.max_slots) {
          auto pick = queue.end();
          if (cfg.policy == POTTS_ADMIT_SMALLEST) {
            for (auto it = queue.begin(); it != queue.end(); ++it) {
              if (stats.bytes_in_use + bytes_of((*it)->r) >
                  cfg.hbm_budget_bytes)
                continue;
              if (pick == queue.end() || work_of((*it)->r) < work_of((*pick)->r))
                pick = it;
            }
          } else if (stats.bytes_in_use + bytes_of(queue.front()->r) <=
                     cfg.hbm_budget_bytes) {
            pick = queue.begin();
          }
          if (pick == queue.end()) break;
          Request *q = *pick;
          queue.erase(pick);
          stats.bytes_in_use += bytes_of(q->r);
          admit.push_back(q);
        }
        // cancellations of admitted requests
        for (size_t i = 0; i < active.size();) {
          Request *q = active[i];
          if (q->cancel_requested) {
            q->state = ReqState::Cancelled;
            stats.cancelled += 1;
            leave_engine(q);
            retired.push_back(q);
            active.erase(active.begin() + (int64_t)i);
            changed = true;
          } else {
            ++i;
          }
        }
      }
      for (Request *q : admit) {  // allocation + init are stream-ordered
        q->m.L = q->r.L;
        q->m.q = q->r.q;
        q->m.start = q->r.start;
        q->m.seed = q->r.seed;
        q->m.beta = q->r.beta;
        q->m.update = q->r.update;
        q->m.user = q;
        q->to_launch = q->r.nsweeps;
        q->to_deliver = q->r.nsweeps;
        const int rc = eng.create_member(&q->m);
        std::lock_guard<std::mutex> lk(mu);
        if (rc != POTTS_OK) {
          q->error = rc;
          stats.bytes_in_use -= bytes_of(q->r);
          q->state = ReqState::Failed;
          continue;
        }
        q->in_engine = true;
        q->state = ReqState::Active;
        stats.admitted += 1;
        active.push_back(q);
        changed = true;
      }
      const int32_t k = std::max(1, cfg.sweeps_per_step);
      bool launched = false;
      if (!active.empty()) {
        if (changed) {
          members.clear();
          for (Request *q : active) members.push_back(&q->m);
          eng.set_members(members);
          changed = false;
        }
        for (Request *q : active) {
          q->m.nsweeps_step = (int32_t)std::min<int64_t>(q->to_launch, k);
          q->to_launch -= q->m.nsweeps_step;
        }
        int rc = eng.launch(k);
        if (rc == POTTS_OK) {
          launched = true;
          std::lock_guard<std::mutex> lk(mu);
          launch_seq += 1;
          for (size_t i = 0; i < active.size();) {
            Request *q = active[i];
            if (q->to_launch == 0) {  // all its sweeps are queued
              leave_engine(q);
              retired.push_back(q);
              active.erase(active.begin() + (int64_t)i);
              changed = true;
            } else {
              ++i;
            }
          }
        } else {
          fail_all(rc);
          members.clear();
          eng.set_members(members);
          continue;
        }
      }
      if (eng.in_flight() == 2 || (!launched && eng.in_flight() > 0)) {
        const int rc = eng.complete();
        if (rc != POTTS_OK) {
          fail_all(rc);
          continue;
        }
        complete_seq += 1;
        deliver();
        cv.notify_all();
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        stats.active = (int32_t)active.size();
        stats.queued = (int32_t)queue.size();
      }
    }
    // shutdown: finish what is in flight, free everything still held
    eng.drain();
    std::lock_guard<std::mutex> lk(mu);
    for (Request *q : active) {
      leave_engine(q);
      q->state = ReqState::Cancelled;
    }
    active.clear();
  }

  void fail_all(int rc) {
    eng.drain();
    std::lock_guard<std::mutex> lk(mu);
    complete_seq = launch_seq;
    loop_error = rc;
    loop_msg = potts_last_error();
    for (Request *q : active) {
      q->error = rc;
      q->state = ReqState::Failed;
      leave_engine(q);
      retired.push_back(q);
    }
    active.clear();
  }
};

extern "C" {

int potts_serve_start(const potts_serve_cfg *cfg, potts_server_h *out) {
  if (!cfg || !out) return fail(POTTS_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->max_slots <= 0 || cfg->sweeps_per_step <= 0 ||
      cfg->hbm_budget_bytes == 0 || cfg->queue_capacity < 0 ||
      (cfg->policy != POTTS_ADMIT_FIFO && cfg->policy != POTTS_ADMIT_SMALLEST))
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
    s->eng.release();
    cudaStreamDestroy(s->st);
    delete s;
    return rc;
  }
  s->eng.initial_counts = false;
  try {
    s->th = std::thread([s] { s->run(); });
  } catch (...) {
    s->eng.release();
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
  if (r.update != POTTS_UPDATE_METROPOLIS && r.update != POTTS_UPDATE_HEATBATH)
    return fail(POTTS_EINVAL, "unknown update rule %d", r.update);
  if (r.update == POTTS_UPDATE_HEATBATH) {
    uint64_t W[5];
    int32_t e = 0;
    if (!heatbath_table(r.beta, r.q, W, &e))
      return fail(POTTS_EINVAL,
                  "beta=%g is outside the heat-bath weights' range for q=%d",
                  r.beta, r.q);
  }
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
    // a request that went through the engine stays on the retired list
    // until no in-flight step can reference it; the loop deletes it then
    const bool held = std::find(s->retired.begin(), s->retired.end(), q) !=
                          s->retired.end() ||
                      std::find(s->active.begin(), s->active.end(), q) !=
                          s->active.end();
    if (held) q->forgotten = true;
    else delete q;
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
  {
    std::unordered_set<Request *> owned;
    for (auto &kv : s->all) owned.insert(kv.second);
    for (Request *q : s->retired) owned.insert(q);
    for (Request *q : owned) delete q;
    s->all.clear();
    s->retired.clear();
  }
  s->eng.release();  // uses the stream: before it is destroyed
  if (s->st) cudaStreamDestroy(s->st);
  int rc = s->loop_error;
  delete s;
  return rc == POTTS_OK ? POTTS_OK : fail(rc, "server loop had failed");
}

}  // extern "C"
