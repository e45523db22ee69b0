// Execution forms around the plain batch update.
//
// Batched form: many independent graphs (contexts), each on its own CUDA
// stream, updated concurrently by a pool of host threads, so that the
// device overlaps the kernels of different graphs while each graph's update
// keeps its own order.  Served form: a request server with a worker pool;
// requests on one context run in submission order, requests on different
// contexts overlap on the device; new contexts are admitted only when the
// device's free memory covers their estimated footprint.
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
  Clock::time_point submit, start, end;
  ldl_status status = LDL_OK;
  ldl_result res{};
  bool done = false;
};

}  // namespace

struct ldl_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<int64_t, Job*> jobs;
  std::set<ldl_ctx*> busy;
  std::vector<std::thread> workers;
  int64_t next_ticket = 0;
  bool stop = false;
  double margin = 1.10;

  void run() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      Job* job = nullptr;
      for (auto it = pending.begin(); it != pending.end(); ++it)
        if (!busy.count((*it)->ctx)) {
          job = *it;
          pending.erase(it);
          break;
        }
      if (!job) {
        if (stop && pending.empty()) return;
        cv_work.wait(lk);
        continue;
      }
      busy.insert(job->ctx);
      lk.unlock();
      job->start = Clock::now();
      job->status = ldl_apply_batch(job->ctx, job->upd.data(), (int64_t)job->upd.size(), 0, &job->res);
      job->end = Clock::now();
      lk.lock();
      busy.erase(job->ctx);
      job->done = true;
      cv_done.notify_all();
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
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return LDL_E_CUDA;
  }
  if ((double)free_b < (double)need * s->margin) return LDL_E_NOMEM;
  return ldl_create(params, n, nnz, row_ptr, col, w, out);
}

ldl_status ldl_server_submit(ldl_server* s, ldl_ctx* ctx, const ldl_update* updates, int64_t count, int64_t* ticket) {
  if (!s || !ctx || count < 0 || (count > 0 && !updates) || !ticket) return LDL_E_INVALID;
  Job* j = new Job();
  j->ctx = ctx;
  j->upd.assign(updates, updates + count);
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
