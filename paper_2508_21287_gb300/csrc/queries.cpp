// Host-side runner for a batch of independent layout queries: one thread per context, each
// planning and answering queries (dm_plan + dm_match_topk) in index order as it frees up, so
// the dependent launches of one query overlap on the GPU with those of the others. No state
// is shared between the threads but the next-query counter and the per-query output slots.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>

#include "../../include/dm.h"

namespace {

struct QueryTap {  // forwards dm_match_topk's chunk callback with the query index
  dm_query_cb cb;
  void *user;
  int32_t query;
};

int tap_cb(void *u, const int32_t *rows, const float *scores, int64_t nrows, int32_t n_cols) {
  const QueryTap *t = (const QueryTap *)u;
  return t->cb(t->user, t->query, rows, scores, nrows, n_cols);
}

struct StatSum {
  int64_t chunks = 0, join_launches = 0, kernel_launches = 0, max_rows = 0;
  double join_ms = 0.0, join_bytes = 0.0;
};

}  // namespace

extern "C" int dm_match_topk_queries(dm_ctx *const *ctxs, const dm_graph *gids, int32_t n_ctx, int32_t n_q,
                                     const int32_t *n_p, const int32_t *const *p_row_ptr,
                                     const int32_t *const *p_col_idx, const dm_plan_opts *opts, int mode,
                                     dm_query_cb cb, void *user, int32_t k, int32_t *const *out_rows,
                                     float *const *out_scores, int32_t *out_n, uint64_t *out_counts,
                                     uint64_t *out_checksums, int32_t *out_status, dm_stats *out_stats) {
  if (!ctxs || !gids || n_ctx < 1 || n_q < 0 || k < 1 || (mode & 0xF) != DM_ALL) return DM_E_INVAL;
  if (n_q > 0 && (!n_p || !p_row_ptr || !p_col_idx || !out_rows || !out_n)) return DM_E_INVAL;
  for (int32_t t = 0; t < n_ctx; t++) {
    if (!ctxs[t]) return DM_E_INVAL;
    for (int32_t u = 0; u < t; u++)
      if (ctxs[u] == ctxs[t]) return DM_E_INVAL;  // a context serves one thread at a time
  }
  for (int32_t i = 0; i < n_q; i++)
    if (!out_rows[i]) return DM_E_INVAL;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int32_t> status(n_q, DM_OK);
  std::vector<StatSum> sums(n_ctx);
  std::atomic<int32_t> next{0};
  auto work = [&](int32_t t) {
    dm_ctx *c = ctxs[t];
    StatSum &sm = sums[t];
    for (int32_t i; (i = next.fetch_add(1)) < n_q;) {
      dm_plan_t *pl = nullptr;
      int32_t n = 0;
      uint64_t cnt = 0, cs = 0;
      int rc = dm_plan(c, gids[t], n_p[i], p_row_ptr[i], p_col_idx[i], opts, &pl);
      if (rc == DM_OK) {
        QueryTap tap{cb, user, i};
        rc = dm_match_topk(c, pl, mode, cb ? tap_cb : nullptr, cb ? &tap : nullptr, k, out_rows[i],
                           out_scores ? out_scores[i] : nullptr, &n, &cnt, &cs);
        dm_stats st;
        if (dm_get_stats(c, &st) == DM_OK) {
          sm.chunks += st.chunks;
          sm.join_launches += st.join_launches;
          sm.kernel_launches += st.kernel_launches;
          sm.max_rows = std::max(sm.max_rows, st.max_rows);
          sm.join_ms += st.join_ms;
          sm.join_bytes += st.join_bytes;
        }
      }
      if (pl) dm_plan_free(pl);
      out_n[i] = rc == DM_OK ? n : 0;
      if (out_counts) out_counts[i] = rc == DM_OK ? cnt : 0;
      if (out_checksums) out_checksums[i] = rc == DM_OK ? cs : 0;
      status[i] = rc;
    }
  };
  std::vector<std::thread> th;
  for (int32_t t = 1; t < n_ctx && t < n_q; t++) th.emplace_back(work, t);
  work(0);
  for (auto &x : th) x.join();
  if (out_status)
    for (int32_t i = 0; i < n_q; i++) out_status[i] = status[i];
  if (out_stats) {
    memset(out_stats, 0, sizeof(*out_stats));
    for (auto &sm : sums) {
      out_stats->chunks += sm.chunks;
      out_stats->join_launches += sm.join_launches;
      out_stats->kernel_launches += sm.kernel_launches;
      out_stats->max_rows = std::max(out_stats->max_rows, sm.max_rows);
      out_stats->join_ms += sm.join_ms;
      out_stats->join_bytes += sm.join_bytes;
    }
    out_stats->total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  for (int32_t i = 0; i < n_q; i++)
    if (status[i] != DM_OK) return status[i];
  return DM_OK;
}
