// Layout-query server: continuous admission of top-k requests onto a pool of worker slots.
//
// Each slot owns a context (its own CUDA stream, arena and copies of the device graphs) and a
// host thread, so requests on different slots run concurrently on the GPU. A request is
// planned by the slot that takes it; its projected join memory (the planner's row estimates
// times the row widths, for the two largest consecutive tables) is reserved from a pool
// shared by all slots before it runs and released when it finishes. Requests are taken in
// arrival order as slots and pool memory free up; a request whose projection alone exceeds
// the pool, or whose projected or actual candidate rows exceed the work cap, is answered
// with DM_E_CAPACITY.
//
// Overlap on the device is measured, not assumed: every slot runs on a stream of its own and
// brackets each request's device work with two CUDA events; their times against one reference
// event give each request's interval on the GPU timeline, and a request whose interval
// intersects that of another request counts as overlapped.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/dm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  dm_graph g;
  int32_t n_p, k;
  std::vector<int32_t> rp, ci;
  Clock::time_point arrival;
};

struct Result {
  int32_t status = 0;
  std::vector<int32_t> rows;
  std::vector<float> scores;
  int32_t n = 0;
  double latency_ms = 0, queue_ms = 0;
  bool done = false;
};

}  // namespace

struct dm_server {
  int device = 0;
  dm_server_opts opts{};
  std::vector<int32_t> motifs;
  std::vector<dm_ctx *> slots;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::map<uint64_t, Result> results;
  uint64_t next_id = 1;
  uint64_t pool_total = 0, pool_used = 0;
  bool stop = false;
  int64_t in_flight = 0;
  int64_t running = 0;  // requests inside their device work right now
  dm_server_stats st{};
  // device timeline: one stream and two events per slot, one reference event for all
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_start, ev_end;
  cudaEvent_t ev_ref = nullptr;
  std::deque<std::pair<double, double>> recent;  // device intervals of the latest requests (ms)
};

namespace {

// Projected device bytes of a plan: the largest pair of consecutive tables it materialises,
// from the rows the plan predicts after each step (the trained model's for plans made in the
// learned order, the independence heuristic's otherwise) and the tables' widths.
uint64_t projected_bytes(const dm_plan_t *pl, int64_t *max_rows_est) {
  int32_t nwords = dm_plan_describe(pl, nullptr, 0);
  std::vector<int32_t> d(nwords > 0 ? nwords : 1);
  dm_plan_describe(pl, d.data(), nwords);
  int32_t n_steps = d[0];
  std::vector<double> rows_after(n_steps > 0 ? n_steps : 1, 0.0);
  dm_plan_predicted_rows(pl, rows_after.data(), n_steps);
  double prev_bytes = 0.0, best = 0.0, maxr = 0.0;
  int32_t pos = 1, w = 0;
  for (int32_t j = 0; j < n_steps; j++) {  // walk the steps for the widths
    int32_t k = d[pos + 1];
    int32_t n_keys = d[pos + 2 + k];
    int32_t n_be = d[pos + 3 + k];
    w += k - n_keys;
    pos += 4 + k + 2 * n_be;
    double rows = rows_after[j];
    maxr = std::max(maxr, rows);
    double bytes = rows * (4.0 * w + 4.0);
    best = std::max(best, bytes + prev_bytes);
    prev_bytes = bytes;
  }
  if (max_rows_est) *max_rows_est = (int64_t)std::min(maxr, 9.0e18);
  return (uint64_t)std::min(best, 1.8e19);
}

void worker(dm_server *s, int slot) {
  dm_ctx *c = s->slots[slot];
  while (true) {
    Request rq;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop && s->queue.empty()) return;
      rq = std::move(s->queue.front());
      s->queue.pop_front();
      s->in_flight++;
    }
    Result res;
    dm_plan_opts po{};
    po.motifs = s->motifs.empty() ? nullptr : s->motifs.data();
    po.n_motifs = (int32_t)s->motifs.size();
    po.order = s->opts.order;
    po.max_rows = s->opts.max_rows;
    dm_plan_t *pl = nullptr;
    int rc = dm_plan(c, rq.g, rq.n_p, rq.rp.data(), rq.ci.data(), &po, &pl);
    uint64_t need = 0;
    bool reserved = false;
    if (rc == DM_OK) {
      int64_t est_rows = 0;
      need = std::max<uint64_t>(projected_bytes(pl, &est_rows), 1);
      if (need > s->pool_total || (s->opts.max_rows > 0 && est_rows > s->opts.max_rows)) rc = DM_E_CAPACITY;
    }
    if (rc == DM_OK) {  // admission: wait until the projected memory fits the shared pool
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_done.wait(lk, [&] { return s->pool_used + need <= s->pool_total; });
      s->pool_used += need;
      reserved = true;
    }
    auto start = Clock::now();
    double dev_a = -1, dev_b = -1;
    if (rc == DM_OK) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->running++;
        s->st.max_running = std::max(s->st.max_running, s->running);
      }
      res.rows.assign((size_t)rq.k * rq.n_p, 0);
      res.scores.assign(rq.k, 0.f);
      const bool timed = cudaEventRecord(s->ev_start[slot], s->streams[slot]) == cudaSuccess;
      rc = dm_score_topk(c, pl, rq.k, res.rows.data(), res.scores.data(), &res.n);
      float a = 0.f, b = 0.f;
      if (timed && cudaEventRecord(s->ev_end[slot], s->streams[slot]) == cudaSuccess &&
          cudaEventSynchronize(s->ev_end[slot]) == cudaSuccess &&
          cudaEventElapsedTime(&a, s->ev_ref, s->ev_start[slot]) == cudaSuccess &&
          cudaEventElapsedTime(&b, s->ev_ref, s->ev_end[slot]) == cudaSuccess) {
        dev_a = a;
        dev_b = b;
      }
      cudaGetLastError();
    }
    auto end = Clock::now();
    if (pl) dm_plan_free(pl);
    res.status = rc;
    res.latency_ms = std::chrono::duration<double, std::milli>(end - rq.arrival).count();
    res.queue_ms = std::chrono::duration<double, std::milli>(start - rq.arrival).count();
    res.done = true;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (reserved) s->pool_used -= need;
      if (reserved) s->running--;
      if (dev_b > dev_a && dev_a >= 0) {
        bool ov = false;
        for (auto &iv : s->recent) ov |= iv.first < dev_b && dev_a < iv.second;
        if (ov) s->st.overlapped++;
        s->recent.emplace_back(dev_a, dev_b);
        if (s->recent.size() > 4 * s->slots.size()) s->recent.pop_front();
      }
      s->in_flight--;
      if (rc == DM_OK) s->st.completed++;
      else if (rc == DM_E_CAPACITY) s->st.rejected++;
      else s->st.failed++;
      s->results[rq.id] = std::move(res);
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int dm_server_create(dm_server **out, int device, const dm_server_opts *opts) {
  if (!out) return DM_E_INVAL;
  dm_server_opts o{};
  if (opts) o = *opts;
  if (o.n_slots <= 0) o.n_slots = 4;
  if (o.n_slots > 64) return DM_E_INVAL;
  dm_server *s = new dm_server();
  s->device = device;
  s->opts = o;
  if (o.motifs && o.n_motifs > 0) s->motifs.assign(o.motifs, o.motifs + o.n_motifs);
  s->opts.motifs = nullptr;
  cudaSetDevice(device);
  if (cudaEventCreate(&s->ev_ref) != cudaSuccess) {
    cudaGetLastError();
    s->ev_ref = nullptr;
    dm_server_destroy(s);
    return DM_E_CUDA;
  }
  for (int i = 0; i < o.n_slots; i++) {
    dm_ctx *c = nullptr;
    int rc = dm_create(&c, device, 0);
    if (rc != DM_OK) {
      dm_server_destroy(s);
      return rc;
    }
    s->slots.push_back(c);
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      if (st) cudaStreamDestroy(st);
      if (a) cudaEventDestroy(a);
      dm_server_destroy(s);
      return DM_E_CUDA;
    }
    s->streams.push_back(st);
    s->ev_start.push_back(a);
    s->ev_end.push_back(b);
    dm_set_stream(c, st);
  }
  if (cudaEventRecord(s->ev_ref, s->streams[0]) != cudaSuccess || cudaEventSynchronize(s->ev_ref) != cudaSuccess) {
    cudaGetLastError();
    dm_server_destroy(s);
    return DM_E_CUDA;
  }
  uint64_t budget = o.mem_budget_bytes;
  if (budget == 0) budget = 16ull << 30;
  s->pool_total = budget;
  for (int i = 0; i < o.n_slots; i++) s->threads.emplace_back(worker, s, i);
  *out = s;
  return DM_OK;
}

int dm_server_load_graph(dm_server *s, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const float *edge_err, const float *qubit_err, dm_graph *out) {
  if (!s || !out) return DM_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->in_flight || !s->queue.empty()) return DM_E_INVAL;
  dm_graph first = -1;
  for (dm_ctx *c : s->slots) {
    dm_graph g;
    int rc = dm_load_data_graph(c, n, row_ptr, col_idx, edge_err, qubit_err, &g);
    if (rc != DM_OK) return rc;
    if (first < 0) first = g;
    else if (g != first) return DM_E_INVAL;
  }
  *out = first;
  return DM_OK;
}

int dm_server_set_model(dm_server *s, const float *w, int64_t n) {
  if (!s) return DM_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  for (dm_ctx *c : s->slots) {
    int rc = dm_model_set_weights(c, w, n);
    if (rc != DM_OK) return rc;
  }
  return DM_OK;
}

int dm_server_submit(dm_server *s, dm_graph g, int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx,
                     int32_t k, uint64_t *out_id) {
  if (!s || !p_row_ptr || (n_p > 0 && !p_col_idx) || n_p < 1 || k < 1) return DM_E_INVAL;
  Request rq;
  rq.g = g;
  rq.n_p = n_p;
  rq.k = k;
  rq.rp.assign(p_row_ptr, p_row_ptr + n_p + 1);
  rq.ci.assign(p_col_idx, p_col_idx + p_row_ptr[n_p]);
  rq.arrival = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rq.id = s->next_id++;
    if (out_id) *out_id = rq.id;
    s->queue.push_back(std::move(rq));
    s->st.submitted++;
  }
  s->cv_work.notify_one();
  return DM_OK;
}

int dm_server_wait(dm_server *s, uint64_t id, int32_t *rows, float *scores, int32_t *n_out, int32_t *status,
                   double *latency_ms, double *queue_ms) {
  if (!s) return DM_E_INVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (id == 0 || id >= s->next_id) return DM_E_NOTFOUND;
  s->cv_done.wait(lk, [&] { return s->results.count(id) && s->results[id].done; });
  Result &r = s->results[id];
  if (rows && !r.rows.empty()) memcpy(rows, r.rows.data(), sizeof(int32_t) * r.rows.size());
  if (scores && !r.scores.empty()) memcpy(scores, r.scores.data(), sizeof(float) * r.scores.size());
  if (n_out) *n_out = r.n;
  if (status) *status = r.status;
  if (latency_ms) *latency_ms = r.latency_ms;
  if (queue_ms) *queue_ms = r.queue_ms;
  s->results.erase(id);
  return DM_OK;
}

int dm_server_stats_get(dm_server *s, dm_server_stats *out) {
  if (!s || !out) return DM_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = (int64_t)s->queue.size();
  out->in_flight = s->in_flight;
  out->pool_used = s->pool_used;
  out->pool_total = s->pool_total;
  return DM_OK;
}

int dm_server_destroy(dm_server *s) {
  if (!s) return DM_E_INVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (auto &t : s->threads) t.join();
  for (dm_ctx *c : s->slots) dm_destroy(c);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->ev_start) cudaEventDestroy(e);
  for (cudaEvent_t e : s->ev_end) cudaEventDestroy(e);
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  delete s;
  return DM_OK;
}

}  // extern "C"
