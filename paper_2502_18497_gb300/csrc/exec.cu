// Execution forms around the plain batch update.
//
// Batched form: many independent graphs (contexts), each on its own CUDA
// stream, updated concurrently by a pool of host threads, so that the
// device overlaps the kernels of different graphs while each graph's update
// keeps its own order.  Served form: a request server with a worker pool;
// requests on one context run in submission order, requests on different
// contexts overlap on the device; new contexts are admitted only when the
// device's free memory covers their estimated footprint, and each batch only
// when the free memory covers its estimated growth (otherwise it waits).
//
// Neither form changes the arithmetic: every context's result is the one
// it would reach alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "kern.cuh"

// ---------------------------------------------------------------- batched form
extern "C" ldl_status ldl_apply_batches(ldl_ctx* const* ctxs, const ldl_update* const* updates,
                                        const int64_t* counts, int32_t g, int32_t updates_on_device,
                                        int32_t threads, ldl_status* statuses, ldl_result* results) {
  if (g < 0 || (g > 0 && (!ctxs || !counts))) return LDL_E_INVALID;
  if (g == 0) return LDL_OK;
  int nt = threads > 0 ? threads : (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  nt = std::min(nt, (int)g);
  std::vector<ldl_status> st((size_t)g, LDL_OK);
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= g) return;
      st[(size_t)i] = ldl_apply_batch(ctxs[i], updates ? updates[i] : nullptr, counts[i], updates_on_device,
                                      results ? &results[i] : nullptr);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  ldl_status first = LDL_OK;
  for (int32_t i = 0; i < g; ++i) {
    if (statuses) statuses[i] = st[(size_t)i];
    if (first == LDL_OK && st[(size_t)i] != LDL_OK) first = st[(size_t)i];
  }
  return first;
}

// ---------------------------------------------------------------- admission
// Device bytes a context of n vertices and nnz stored entries needs: per-node
// arrays of every level, the level-0 adjacency with its slack, a working
// reserve for aggregate levels and record buffers.
extern "C" ldl_status ldl_estimate_bytes(const ldl_params* p, int64_t n, int64_t nnz, int64_t* bytes) {
  if (!p || !bytes || n <= 0 || nnz < 0) return LDL_E_INVALID;
  const int64_t levels = (int64_t)p->L + 1;
  const int64_t per_node_global = 64 * 4 + 10 * 8;                 // stamps, lists, candidates, scratch
  const int64_t per_node_level = 3 * 4 + 2 * 8 + 1 + 2 * 4 + 3 * 8; // lab/par/cnt, k, alive, frontier, CSRs
  const int64_t dir = p->directed ? 2 : 1;
  const int64_t adj0 = dir * nnz * 8 * 5 / 2;  // level 0: 25% slack, doubled by a pool compaction
  const int64_t upper = dir * nnz * 12 * 2;     // aggregate levels (bounded by level 0), same headroom
  const int64_t records = dir * nnz * 16 * 6;   // sort ping-pong, reduce and CSR update scratch
  *bytes = n * (per_node_global + levels * per_node_level) + adj0 + upper + records + (64 << 20);
  return LDL_OK;
}

// ---------------------------------------------------------------- served form
namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket;
  ldl_ctx* ctx;
  std::vector<ldl_update> upd;
  int64_t need = 0;  // estimated new device bytes of this batch
  bool counted_deferral = false;
  int64_t wait_done = 0;  // after a rollback: run again once this many requests completed
  Clock::time_point submit, start, end;
  ldl_status status = LDL_OK;
  ldl_result res{};
  bool done = false;
};

}  // namespace

// Requests wait in one queue.  A worker takes the oldest request whose
// context is idle and whose estimated memory need fits the device's free
// memory minus what running requests have reserved; a request that does not
// fit is deferred (it keeps its place, and later requests of its context wait
// behind it) until a running request finishes.  Batches are atomic, so a
// request that still runs out of memory while others run is rolled back and
// queued again at the front instead of failing; with nothing else running it
// fails with LDL_E_NOMEM.
struct ldl_server {
  std::mutex mu;
  std::mutex admit_mu;  // serialises admission checks with the creation they guard
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<int64_t, Job*> jobs;
  std::set<ldl_ctx*> busy;
  std::vector<std::thread> workers;
  int64_t next_ticket = 0;
  bool stop = false;
  double margin = 1.10;
  int64_t free_override = -1;  // test hook: the device's free bytes (-1: ask CUDA)
  int64_t reserved = 0;        // bytes reserved by running requests
  int running = 0;
  int64_t deferred = 0, retried = 0, completed = 0;

  int64_t free_bytes() {
    if (free_override >= 0) return free_override;
    size_t f = 0, t = 0;
    if (cudaMemGetInfo(&f, &t) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return (int64_t)f;
  }

  // the oldest runnable request (context idle, memory available), or null;
  // caller holds mu
  Job* take() {
    std::set<ldl_ctx*> blocked;  // contexts with an earlier deferred request
    int64_t avail = -1;
    for (auto it = pending.begin(); it != pending.end(); ++it) {
      Job* j = *it;
      if (busy.count(j->ctx) || blocked.count(j->ctx)) continue;
      if (completed < j->wait_done && running > 0) {
        blocked.insert(j->ctx);
        continue;
      }
      if (running > 0) {
        if (avail < 0) avail = free_bytes() - reserved;
        if ((double)j->need * margin > (double)avail) {
          if (!j->counted_deferral) {
            j->counted_deferral = true;
            ++deferred;
          }
          blocked.insert(j->ctx);
          continue;
        }
      }
      pending.erase(it);
      return j;
    }
    return nullptr;
  }

  void run() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      Job* job = take();
      if (!job) {
        if (stop && pending.empty() && running == 0) return;
        cv_work.wait(lk);
        continue;
      }
      busy.insert(job->ctx);
      reserved += job->need;
      ++running;
      const bool others = running > 1;
      lk.unlock();
      if (job->start == Clock::time_point()) job->start = Clock::now();
      const ldl_status st = ldl_apply_batch(job->ctx, job->upd.data(), (int64_t)job->upd.size(), 0, &job->res);
      const Clock::time_point end = Clock::now();
      lk.lock();
      busy.erase(job->ctx);
      reserved -= job->need;
      --running;
      if (st == LDL_E_NOMEM && (others || running > 0) && !stop) {
        // rolled back: try again once memory held by other requests is free
        ++retried;
        job->wait_done = completed + 1;
        pending.push_front(job);
      } else {
        job->status = st;
        job->end = end;
        job->done = true;
        ++completed;
        cv_done.notify_all();
      }
      cv_work.notify_all();
    }
  }
};

extern "C" {

ldl_status ldl_server_create(int32_t workers, ldl_server** out) {
  if (!out || workers < 1 || workers > 256) return LDL_E_INVALID;
  ldl_server* s = new ldl_server();
  for (int i = 0; i < workers; ++i) s->workers.emplace_back([s]() { s->run(); });
  *out = s;
  return LDL_OK;
}

ldl_status ldl_server_admit(ldl_server* s, const ldl_params* params, int64_t n, int64_t nnz, const int64_t* row_ptr,
                            const int32_t* col, const int32_t* w, ldl_ctx** out) {
  if (!s || !out) return LDL_E_INVALID;
  int64_t need = 0;
  ldl_status st = ldl_estimate_bytes(params, n, nnz, &need);
  if (st != LDL_OK) return st;
  // one admission at a time: the free memory seen here is what the creation
  // below gets (running requests' reservations are subtracted)
  std::lock_guard<std::mutex> ak(s->admit_mu);
  int64_t avail = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    avail = s->free_bytes() - s->reserved;
  }
  if ((double)avail < (double)need * s->margin) return LDL_E_NOMEM;
  return ldl_create(params, n, nnz, row_ptr, col, w, out);
}

ldl_status ldl_server_submit(ldl_server* s, ldl_ctx* ctx, const ldl_update* updates, int64_t count, int64_t* ticket) {
  if (!s || !ctx || count < 0 || (count > 0 && !updates) || !ticket) return LDL_E_INVALID;
  Job* j = new Job();
  j->ctx = ctx;
  j->upd.assign(updates, updates + count);
  if (ldl_batch_estimate_bytes(ctx, count, &j->need) != LDL_OK) j->need = 0;
  j->submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete j;
      return LDL_E_INVALID;
    }
    j->ticket = s->next_ticket++;
    s->jobs[j->ticket] = j;
    s->pending.push_back(j);
    *ticket = j->ticket;
  }
  s->cv_work.notify_one();
  return LDL_OK;
}

ldl_status ldl_server_wait(ldl_server* s, int64_t ticket, int32_t timeout_ms, ldl_status* status, ldl_result* result,
                           double* queue_us, double* service_us) {
  if (!s) return LDL_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return LDL_E_INVALID;
  Job* j = it->second;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, [j]() { return j->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [j]() { return j->done; })) {
    return LDL_E_TIMEOUT;
  }
  if (status) *status = j->status;
  if (result) *result = j->res;
  if (queue_us) *queue_us = std::chrono::duration<double, std::micro>(j->start - j->submit).count();
  if (service_us) *service_us = std::chrono::duration<double, std::micro>(j->end - j->start).count();
  s->jobs.erase(it);
  delete j;
  return LDL_OK;
}

ldl_status ldl_server_stats(ldl_server* s, int64_t* deferred, int64_t* retried) {
  if (!s) return LDL_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (deferred) *deferred = s->deferred;
  if (retried) *retried = s->retried;
  return LDL_OK;
}

ldl_status ldl_server_debug_free_bytes(ldl_server* s, int64_t bytes) {
  if (!s) return LDL_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  s->free_override = bytes < 0 ? -1 : bytes;
  s->cv_work.notify_all();
  return LDL_OK;
}

void ldl_server_destroy(ldl_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
}

}  // extern "C"
