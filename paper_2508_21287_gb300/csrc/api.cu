// C ABI of the Delta-Motif library: context, data-graph store, motif database (Alg. 2),
// plans (Sec. 3.2), the chunked join executor (Alg. 1), canonical output, top-k scoring.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <set>
#include <memory>
#include <string>
#include <tuple>
#include <atomic>
#include <thread>
#include <vector>

#include "../../include/dm.h"
#include "dm_internal.h"
#include "kernels.h"

using namespace dmi;

namespace {

struct DevTable {
  int32_t *rows = nullptr;
  float *score = nullptr;
  int64_t n = 0;
  int32_t w = 0;
  bool borrowed = false;  // lives in the context's arena: never freed by its holder
  int64_t held = 0;       // bytes counted against the memory budget while it lives
};

struct Index {
  IndexView v{};
  int32_t *rows = nullptr;
  float *score = nullptr;
  int32_t *offsets = nullptr;
  HashSlot *slots = nullptr;
  unsigned long long *keys = nullptr;  // sort-merge join: sorted packed keys
  int64_t distinct = 0;
  int64_t max_group = 0;
  int64_t bytes = 0;
};

struct DevGraph {
  int32_t V = 0;
  int64_t nnz = 0;
  int32_t *row_ptr = nullptr, *col_idx = nullptr;
  float *eerr = nullptr, *qerr = nullptr;
  float *edir = nullptr;  // per-direction gate costs aligned with col_idx (direction-aware scores)
  unsigned long long *adj = nullptr;
  int32_t adj_words = 0;
  double avg_deg = 0;
  int32_t max_deg = 0;
  // every edge and vertex weight is >= 0, so a partial score never exceeds a full one and
  // top-k may drop rows whose partial score is above the current k-th best
  bool nonneg_weights = true;
  std::map<int, DevTable> motifs;
  std::map<std::tuple<int, int, int, int>, Index> indices;  // (motif, key position 0, 1, sort-merge)
};

}  // namespace

struct dm_ctx {
  int device = 0;
  cudaStream_t own = nullptr, stream = nullptr;
  int num_sms = 1;
  uint64_t budget = 0;
  std::vector<DevGraph *> graphs;
  unsigned long long *d_ctr = nullptr, *h_ctr = nullptr;
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  dm_stats stats{};
  int64_t inflight = 0;
  std::string last_error;
  void *h_stage = nullptr;
  size_t h_stage_bytes = 0;
  // arena of the device-driven path: two halves alternate as the input and output of a step
  unsigned char *arena = nullptr;
  size_t arena_bytes = 0;
  unsigned long long *d_ctr_steps = nullptr;  // CTR_N counters per step
  unsigned long long *h_ctr_steps = nullptr;
  struct BatchState *batch = nullptr;  // cached device image of the last batch of plans
  // cardinality model (DM_ORDER_LEARNED) and the step log it is trained on
  float *m_params = nullptr, *m_grads = nullptr, *m_m = nullptr, *m_v = nullptr;
  int m_step = 0;
  bool m_trained = false;
  float m_mean[NFEAT] = {}, m_std[NFEAT] = {};
  bool log_steps = true;
  std::vector<float> log_feat, log_target;
  int autotune = 1;
  double hash_lf = 0.5;               // load factor of two-key hash indices
  double heavy_rows = 1e300;          // plans predicted to hold more rows run step by step
  int batch_threads = 256, batch_ctas = 0;  // block shape of dm_match_batch without autotuning
  bool fuse_last = false;  // counted plans: the last two joins in one launch when they qualify
  std::vector<double> batch_latency;  // per plan, ms from the start of the last dm_match_batch
};

struct dm_plan_s {
  Plan p;
};

namespace {

#define CK(x)                                              \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #x);    \
  } while (0)
#define RET(x)                     \
  do {                             \
    int r_ = (x);                  \
    if (r_ != DM_OK) return r_;    \
  } while (0)

int cuda_fail(dm_ctx *c, cudaError_t e, const char *what) {
  if (c) c->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DM_E_NOMEM;
  }
  return DM_E_CUDA;
}

// Device allocations come from the stream-ordered pool (fast reuse of the large blocks that
// streaming allocates and frees chunk after chunk); when an allocation fails, the pool's
// cached free memory is returned to the device and the allocation is tried once more.
static void trim_pool(dm_ctx *c) {
  cudaStreamSynchronize(c->stream);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
  cudaGetLastError();
}

int dalloc(dm_ctx *c, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  for (int attempt = 0; attempt < 2; attempt++) {
    if (cudaMallocAsync(p, bytes, c->stream) == cudaSuccess) return DM_OK;
    cudaGetLastError();
    *p = nullptr;
    if (attempt == 0) trim_pool(c);
  }
  c->last_error = "cudaMallocAsync of " + std::to_string(bytes) + " bytes failed (budget " +
                  std::to_string(c->budget) + ", held by the current plan " + std::to_string(c->inflight) + ")";
  return DM_E_NOMEM;
}
template <class T>
int dalloc_t(dm_ctx *c, T **p, size_t count) {
  return dalloc(c, (void **)p, count * sizeof(T));
}
void dfree(dm_ctx *c, void *p) {
  if (p) cudaFreeAsync(p, c->stream);
}
void free_table(dm_ctx *c, DevTable &t) {
  if (!t.borrowed) {
    dfree(c, t.rows);
    dfree(c, t.score);
  }
  t.rows = nullptr;
  t.score = nullptr;
  t.n = 0;
}

int bit_length(int64_t x) {
  int b = 0;
  while (x > 0) {
    b++;
    x >>= 1;
  }
  return b;
}

// ------------------------------------------------------------------ host CSR checks ----
struct HostCSR {
  std::vector<int32_t> rp, ci;
  std::vector<float> ee;
};

int validate_csr(int32_t n, const int32_t *rp, const int32_t *ci, const float *ee, HostCSR *out) {
  if (n < 0 || !rp || (n > 0 && !ci && rp[n] > 0)) return DM_E_INVAL;
  if (rp[0] != 0) return DM_E_INVAL;
  out->rp.assign(n + 1, 0);
  for (int32_t u = 0; u < n; u++) {
    if (rp[u + 1] < rp[u]) return DM_E_INVAL;
    int32_t prev = -1;
    for (int32_t k = rp[u]; k < rp[u + 1]; k++) {
      int32_t v = ci[k];
      if (v < 0 || v >= n) return DM_E_INVAL;
      if (v <= prev) return DM_E_INVAL;  // unsorted or duplicate
      prev = v;
      if (v == u) continue;              // self-loops are dropped (Res(M2) excludes them)
      out->ci.push_back(v);
      if (ee) out->ee.push_back(ee[k]);
    }
    out->rp[u + 1] = (int32_t)out->ci.size();
  }
  // symmetry (and equal weights on both directions)
  for (int32_t u = 0; u < n; u++)
    for (int32_t k = out->rp[u]; k < out->rp[u + 1]; k++) {
      int32_t v = out->ci[k];
      auto b = out->ci.begin() + out->rp[v], e = out->ci.begin() + out->rp[v + 1];
      auto it = std::lower_bound(b, e, u);
      if (it == e || *it != u) return DM_E_INVAL;
      if (ee && out->ee[it - out->ci.begin()] != out->ee[k]) return DM_E_INVAL;
    }
  return DM_OK;
}

bool connected(const HostCSR &g, int32_t n) {
  if (n <= 1) return true;
  std::vector<char> seen(n, 0);
  std::vector<int32_t> st{0};
  seen[0] = 1;
  int32_t cnt = 1;
  while (!st.empty()) {
    int32_t u = st.back();
    st.pop_back();
    for (int32_t k = g.rp[u]; k < g.rp[u + 1]; k++)
      if (!seen[g.ci[k]]) {
        seen[g.ci[k]] = 1;
        cnt++;
        st.push_back(g.ci[k]);
      }
  }
  return cnt == n;
}

// ------------------------------------------------------------------ sorting ------------
// Sort a table's rows lexicographically (column 0 most significant); ids < 2^bits.
int sort_perm_by_columns(dm_ctx *c, const DevTable &t, const std::vector<int> &cols_msb_first, int bits,
                         int32_t **perm_out) {
  int64_t n = t.n;
  int32_t *A = nullptr, *B = nullptr;
  int64_t *hist = nullptr, *hscan = nullptr, *tmp = nullptr;
  int64_t he = dmk::radix_hist_elems(n);
  RET(dalloc_t(c, &A, n));
  RET(dalloc_t(c, &B, n));
  RET(dalloc_t(c, &hist, he));
  RET(dalloc_t(c, &hscan, he + 1));
  RET(dalloc_t(c, &tmp, dmk::scan_tmp_elems(he)));
  CK(dmk::launch_iota(A, n, c->stream));
  if (bits < 1) bits = 1;
  for (int ci = (int)cols_msb_first.size() - 1; ci >= 0; ci--) {
    int col = cols_msb_first[ci];
    for (int shift = 0; shift < bits; shift += 8) {
      CK(dmk::radix_pass((const uint32_t *)t.rows + col, t.w, A, B, n, shift, hist, hscan, tmp, c->stream));
      std::swap(A, B);
    }
  }
  dfree(c, B);
  dfree(c, hist);
  dfree(c, hscan);
  dfree(c, tmp);
  *perm_out = A;
  return DM_OK;
}

int stable_sort_perm_by_score(dm_ctx *c, const DevTable &t, int32_t *&perm) {
  int64_t n = t.n;
  int32_t *B = nullptr;
  int64_t *hist = nullptr, *hscan = nullptr, *tmp = nullptr;
  uint32_t *keys = nullptr;  // scores as order-preserving unsigned keys (negative scores too)
  int64_t he = dmk::radix_hist_elems(n);
  RET(dalloc_t(c, &keys, std::max<int64_t>(1, n)));
  RET(dalloc_t(c, &B, n));
  RET(dalloc_t(c, &hist, he));
  RET(dalloc_t(c, &hscan, he + 1));
  RET(dalloc_t(c, &tmp, dmk::scan_tmp_elems(he)));
  CK(dmk::launch_score_keys(t.score, n, keys, c->stream));
  for (int shift = 0; shift < 32; shift += 8) {
    CK(dmk::radix_pass(keys, 1, perm, B, n, shift, hist, hscan, tmp, c->stream));
    std::swap(perm, B);
  }
  dfree(c, keys);
  dfree(c, B);
  dfree(c, hist);
  dfree(c, hscan);
  dfree(c, tmp);
  return DM_OK;
}

int gather_table(dm_ctx *c, const DevTable &t, const int32_t *perm, int64_t n, DevTable *out) {
  DevTable o;
  o.n = n;
  o.w = t.w;
  RET(dalloc_t(c, &o.rows, (size_t)n * t.w));
  if (t.score) RET(dalloc_t(c, &o.score, n));
  CK(dmk::launch_gather_rows(t.rows, t.score, perm, n, t.w, o.rows, o.score, c->stream));
  *out = o;
  return DM_OK;
}

// Replace t by its rows in canonical (lexicographic) order.
// Sort a table into canonical order; when ctr is set, the rows' checksum is added to
// ctr[CTR_SUM] on the way.
int sort_canonical(dm_ctx *c, DevTable &t, int bits, unsigned long long *ctr = nullptr) {
  if (t.n <= 1) {
    if (ctr && t.n == 1) CK(dmk::launch_hash_rows(t.rows, 1, t.w, ctr, c->stream));
    if (t.borrowed && t.n == 1) {  // take a private copy so the holder may free it
      DevTable o;
      int32_t *one = nullptr;
      RET(dalloc_t(c, &one, 1));
      CK(dmk::launch_iota(one, 1, c->stream));
      RET(gather_table(c, t, one, 1, &o));
      dfree(c, one);
      t = o;
    }
    return DM_OK;
  }
  void *tmp = nullptr;
  RET(dalloc(c, &tmp, (size_t)dmk::msort_tmp_bytes(t.n)));
  DevTable o;
  if (t.n <= dmk::msort_into_max_rows()) {  // small tables: rows go straight to their positions
    o.n = t.n;
    o.w = t.w;
    int r = dalloc_t(c, &o.rows, (size_t)t.n * t.w);
    if (r == DM_OK && t.score) r = dalloc_t(c, &o.score, t.n);
    if (r != DM_OK) {
      free_table(c, o);
      dfree(c, tmp);
      return r;
    }
    CK(dmk::msort_rows_into(t.rows, t.score, t.n, t.w, bits, tmp, o.rows, o.score, ctr ? ctr + CTR_SUM : nullptr,
                            c->num_sms, c->stream));
  } else {
    int32_t *perm = nullptr;
    CK(dmk::msort_rows(t.rows, t.n, t.w, bits, tmp, &perm, ctr ? ctr + CTR_SUM : nullptr, c->stream));
    RET(gather_table(c, t, perm, t.n, &o));
  }
  dfree(c, tmp);
  free_table(c, t);
  t = o;
  return DM_OK;
}

// ------------------------------------------------------------------ motif database -----
int graph_bits(const DevGraph *g) { return std::max(1, bit_length((int64_t)g->V - 1)); }

int read_ctr(dm_ctx *c) {
  CK(cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(unsigned long long) * CTR_N, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DM_OK;
}

// Index of a motif table on its key positions: the table sorted by the key columns, plus
// direct offsets (one key) or an open-addressing hash of the packed key (two keys), or, for the
// sort-merge join, the sorted packed keys themselves (groups found by binary search).
int ensure_index(dm_ctx *c, DevGraph *g, int motif, int kp0, int kp1, bool sortmerge, Index **out) {
  auto key = std::make_tuple(motif, kp0, kp1, sortmerge ? 1 : 0);
  auto it = g->indices.find(key);
  if (it != g->indices.end()) {
    *out = &it->second;
    return DM_OK;
  }
  DevTable &T = g->motifs.at(motif);
  Index ix;
  ix.v.nkeys = kp1 >= 0 ? 2 : 1;
  ix.v.kpos[0] = kp0;
  ix.v.kpos[1] = kp1;
  ix.v.mw = T.w;
  ix.v.n = T.n;
  DevTable sorted = T;
  int32_t *perm = nullptr;
  std::vector<int> cols{kp0};
  if (kp1 >= 0) cols.push_back(kp1);
  if (T.n > 0) {
    RET(sort_perm_by_columns(c, T, cols, graph_bits(g), &perm));
    RET(gather_table(c, T, perm, T.n, &sorted));
    dfree(c, perm);
  } else {
    RET(dalloc_t(c, &sorted.rows, 1));
    sorted.score = nullptr;
  }
  ix.rows = sorted.rows;
  ix.score = sorted.score;
  ix.v.rows = sorted.rows;
  ix.v.score = sorted.score;
  ix.bytes = T.n * (4 * T.w + (sorted.score ? 4 : 0));
  if (sortmerge) {
    RET(dalloc_t(c, &ix.keys, (size_t)std::max<int64_t>(1, T.n)));
    CK(dmk::launch_join_keys(sorted.rows, T.w, kp0, kp1, T.n, ix.keys, c->stream));
    std::vector<unsigned long long> hk((size_t)T.n);
    if (T.n > 0)
      CK(cudaMemcpyAsync(hk.data(), ix.keys, sizeof(unsigned long long) * T.n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int64_t i = 0, run = 0; i < T.n; i++) {  // runs of equal keys: distinct keys, largest group
      run = (i > 0 && hk[i] == hk[i - 1]) ? run + 1 : 1;
      ix.distinct += run == 1;
      ix.max_group = std::max(ix.max_group, run);
    }
    ix.v.keys = ix.keys;
    ix.bytes += 8 * T.n;
  } else if (kp1 < 0) {
    RET(dalloc_t(c, &ix.offsets, (size_t)g->V + 1));
    CK(dmk::launch_offsets_direct(sorted.rows, T.w, kp0, T.n, g->V, ix.offsets, c->stream));
    std::vector<int32_t> off(g->V + 1);
    CK(cudaMemcpyAsync(off.data(), ix.offsets, sizeof(int32_t) * (g->V + 1), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int32_t v = 0; v < g->V; v++) {
      int64_t l = off[v + 1] - off[v];
      ix.distinct += l > 0;
      ix.max_group = std::max(ix.max_group, l);
    }
    ix.v.offsets = ix.offsets;
    ix.bytes += 4 * ((int64_t)g->V + 1);
  } else {
    uint32_t lg = 1;
    while ((double)(1ll << lg) * c->hash_lf < (double)std::max<int64_t>(1, T.n)) lg++;
    RET(dalloc_t(c, &ix.slots, (size_t)1 << lg));
    CK(cudaMemsetAsync(ix.slots, 0xFF, sizeof(HashSlot) << lg, c->stream));
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * CTR_N, c->stream));
    CK(dmk::launch_hash_build(sorted.rows, T.w, kp0, kp1, T.n, ix.slots, lg, c->d_ctr, c->stream));
    RET(read_ctr(c));
    ix.distinct = (int64_t)c->h_ctr[0];
    ix.max_group = (int64_t)c->h_ctr[1];
    ix.v.slots = ix.slots;
    ix.v.log2cap = lg;
    ix.bytes += (int64_t)sizeof(HashSlot) << lg;
  }
  auto res = g->indices.emplace(key, ix);
  *out = &res.first->second;
  return DM_OK;
}

// ------------------------------------------------------------------ executor -----------
struct Sink {
  virtual ~Sink() {}
  // Takes ownership of a table of final rows (pattern-vertex order, unsorted).
  virtual int take(dm_ctx *c, DevTable t) = 0;
};

struct StepRT {
  JoinArgs base{};
  Index *ix = nullptr;
  DevTable *seed_table = nullptr;
  int64_t max_group = 1;
  int64_t motif_bytes = 0;
};

struct Exec {
  dm_ctx *c;
  DevGraph *g;
  const Plan *p;
  int mode;          // DM_ALL / DM_COUNT
  bool use_qerr;
  int32_t shard = 0, n_shards = 1;  // one shard of R_0 (count runs over several GPUs)
  float prune = INFINITY;
  Sink *sink = nullptr;
  int64_t chunk_rows = 0, max_rows = 0;
  bool fused = false;  // the last run_fast ran the plan's last two joins as one kernel
  std::vector<StepRT> st;
  uint64_t count = 0, checksum = 0;

  int setup() {
    const int S = (int)p->steps.size();
    st.assign(S, StepRT());
    for (int j = 0; j < S; j++) {
      const StepSpec &s = p->steps[j];
      StepRT &r = st[j];
      JoinArgs &a = r.base;
      memset(&a, 0, sizeof(a));
      if (j == 0) {
        auto it = g->motifs.find(s.motif);
        if (it == g->motifs.end()) return DM_E_NOTFOUND;
        r.seed_table = &it->second;
        a.ix.nkeys = 0;
        a.ix.rows = it->second.rows;
        a.ix.score = it->second.score;
        a.ix.n = it->second.n;
        a.ix.mw = it->second.w;
        r.motif_bytes = it->second.n * (4 * it->second.w + (it->second.score ? 4 : 0));
      } else {
        if (s.n_keys < 1) return DM_E_INVAL;
        RET(ensure_index(c, g, s.motif, s.key_mpos[0], s.n_keys >= 2 ? s.key_mpos[1] : -1,
                         p->join_algo == DM_JOIN_SORTMERGE, &r.ix));
        a.ix = r.ix->v;
        r.max_group = std::max<int64_t>(1, r.ix->max_group);
        r.motif_bytes = r.ix->bytes;
      }
      a.key_col[0] = s.n_keys > 0 ? s.key_col[0] : 0;
      a.key_col[1] = s.n_keys > 1 ? s.key_col[1] : 0;
      a.n_chk = std::max(0, s.n_keys - 2);
      for (int i = 2; i < s.n_keys; i++) {
        a.chk_mpos[i - 2] = (int8_t)s.key_mpos[i];
        a.chk_col[i - 2] = (int8_t)s.key_col[i];
      }
      a.n_new = s.n_new;
      for (int i = 0; i < s.n_new; i++) a.new_mpos[i] = (int8_t)s.new_mpos[i];
      a.n_be = s.n_be;
      for (int i = 0; i < s.n_be; i++) {
        a.be_a[i] = (int8_t)s.be_col[i][0];
        a.be_b[i] = (int8_t)s.be_col[i][1];
      }
      a.w = s.w_in;
      a.wo = s.w_out;
      a.induced = p->induced;
      for (int i = 0; i < s.n_new; i++)
        for (int h = 0; h < 2; h++) a.nonadj[i][h] = p->induced ? s.nonadj[i][h] : 0ull;
      for (int cc = 0; cc < a.wo; cc++) a.src_col[cc] = (int8_t)cc;
      if (j == S - 1)  // the last step writes rows in pattern-vertex order
        for (int cc = 0; cc < a.wo; cc++) a.src_col[p->col_vertex[cc]] = (int8_t)cc;
      a.adj = g->adj;
      a.adj_words = g->adj_words;
      a.row_ptr = g->row_ptr;
      a.col_idx = g->col_idx;
      a.eerr = g->eerr;
      a.qerr = use_qerr ? g->qerr : nullptr;
      a.scored = g->eerr != nullptr && mode != DM_COUNT;  // a count needs no scores
      a.prune = prune;
      a.mode = (j == S - 1 && mode == DM_COUNT) ? 1 : 0;
      a.nx.nkeys = -1;
      if (j == 0 && n_shards > 1) {
        a.shard = shard;
        a.n_shards = n_shards;
      }
    }
    for (int j = 0; j + 1 < S; j++) {
      st[j].base.nx = st[j + 1].base.ix;
      st[j].base.nx_key_col[0] = st[j + 1].base.key_col[0];
      st[j].base.nx_key_col[1] = st[j + 1].base.key_col[1];
    }
    return DM_OK;
  }

  int64_t row_bytes(int j) const {
    const JoinArgs &a = st[j].base;
    return 4ll * a.wo + (a.scored ? 4 : 0) + (j + 1 < (int)st.size() ? 4 : 0);
  }

  // One join launch over `in` (or over seed rows [lo, hi) of the motif table at step 0).
  int launch(int j, const DevTable &in, int64_t lo, int64_t hi, int64_t cap, DevTable *out, int32_t **out_next,
             int64_t *next_total) {
    const int S = (int)st.size();
    JoinArgs a = st[j].base;
    a.prune = prune;
    DevTable o;
    o.w = a.wo;
    int32_t *nxt = nullptr;
    if (a.mode == 0) {
      int r = dalloc_t(c, &o.rows, (size_t)std::max<int64_t>(1, cap) * a.wo);
      if (r == DM_OK && a.scored) r = dalloc_t(c, &o.score, std::max<int64_t>(1, cap));
      if (r == DM_OK && j + 1 < S) r = dalloc_t(c, &nxt, std::max<int64_t>(1, cap));
      if (r != DM_OK) {  // nothing of a failed launch stays allocated
        free_table(c, o);
        dfree(c, nxt);
        return r;
      }
    }
    a.out = o.rows;
    a.outs = o.score;
    a.out_next = nxt;
    a.out_cap = cap;
    a.ctr = c->d_ctr;
    if (j == 0) {
      a.R = nullptr;
      a.Rs = nullptr;
      a.N = 0;
      a.seed_lo = lo;
      a.seed_hi = hi;
    } else {
      a.R = in.rows;
      a.Rs = in.score;
      a.N = in.n;
    }
    DevTable sorted_in;  // sort-merge join: R ordered by its key columns, so that consecutive
                         // rows probe the same or neighbouring runs of the sorted motif keys
    if (j > 0 && p->join_algo == DM_JOIN_SORTMERGE && in.n > 1) {
      std::vector<int> kc{a.key_col[0]};
      if (a.ix.nkeys == 2) kc.push_back(a.key_col[1]);
      int32_t *perm = nullptr;
      RET(sort_perm_by_columns(c, in, kc, graph_bits(g), &perm));
      RET(gather_table(c, in, perm, in.n, &sorted_in));
      dfree(c, perm);
      a.R = sorted_in.rows;
      a.Rs = sorted_in.score;
    }
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * CTR_N, c->stream));
    int grid = dmk::wjoin_grid(a, c->num_sms);
    if (c->timing) CK(cudaEventRecord(c->ev0, c->stream));
    CK(dmk::launch_wjoin(a, grid, c->stream));
    if (c->timing) CK(cudaEventRecord(c->ev1, c->stream));
    RET(read_ctr(c));
    if (sorted_in.rows) free_table(c, sorted_in);
    if (c->h_ctr[CTR_OVF]) {
      c->last_error = "join output overflow";
      free_table(c, o);
      dfree(c, nxt);
      return DM_E_CAPACITY;
    }
    int64_t rows = (int64_t)c->h_ctr[CTR_ROWS];
    int64_t nin = j == 0 ? hi - lo : in.n;
    if (c->timing) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      c->stats.join_ms += ms;
    }
    c->stats.join_launches++;
    c->stats.chunks++;
    double bytes = (double)st[j].motif_bytes + (double)nin * (4.0 * a.w + (a.Rs ? 4 : 0));
    if (a.mode == 0) bytes += (double)rows * row_bytes(j);
    c->stats.join_bytes += bytes;
    if (j < DM_MAX_STEPS) {
      c->stats.rows[j] += rows;
      c->stats.candidates[j] += (int64_t)c->h_ctr[CTR_CAND];
    }
    if (a.mode == 1) {
      count += (uint64_t)rows;
      checksum += c->h_ctr[CTR_SUM];
    }
    o.n = rows;
    *out = o;
    if (out_next) *out_next = nxt;
    if (next_total) *next_total = (int64_t)c->h_ctr[CTR_NEXT];
    return DM_OK;
  }

  int64_t limit_rows(int j) const {
    int64_t avail = (int64_t)c->budget - c->inflight;
    int64_t lim = std::max<int64_t>(1, avail / row_bytes(j));
    if (chunk_rows > 0) lim = std::min(lim, chunk_rows);
    return lim;
  }

  // After a step-j output (or the seed) exists: run steps j+1.. on it.
  int descend(int j, DevTable &t, int32_t *t_next, int64_t next_total) {
    const int S = (int)st.size();
    if (j == S - 1) {
      if (mode == DM_COUNT) {  // counted inside the last launch
        free_table(c, t);
        dfree(c, t_next);
        return DM_OK;
      }
      c->inflight -= t.held;
      int r = sink->take(c, t);
      dfree(c, t_next);
      return r;
    }
    c->stats.max_rows = std::max(c->stats.max_rows, t.n);
    int r = process(j + 1, t, t_next, next_total);
    c->inflight -= t.held;
    free_table(c, t);
    dfree(c, t_next);
    return r;
  }

  // A table was allocated for `cap` rows (its candidates) and counts against the budget with
  // the rows that survived. When the unused part of its allocation is large (the candidates
  // of a step can be several times its rows, and tables stay alive along the depth-first
  // path), the rows move into an allocation of their own size, so that memory held beyond the
  // budget stays bounded.
  int shrink(int j, DevTable &o, int32_t *&onext, int64_t cap) {
    const int64_t rb = row_bytes(j), alloc = std::max<int64_t>(1, cap) * rb;
    o.held = std::max<int64_t>(1, o.n) * rb;
    const int64_t slack_limit = std::max<int64_t>((int64_t)64 << 20, (int64_t)(c->budget / 32));
    if (alloc - o.held < slack_limit) return DM_OK;
    DevTable t;
    t.n = o.n;
    t.w = o.w;
    int32_t *tn = nullptr;
    int r = dalloc_t(c, &t.rows, (size_t)std::max<int64_t>(1, o.n) * o.w);
    if (r == DM_OK && o.score) r = dalloc_t(c, &t.score, std::max<int64_t>(1, o.n));
    if (r == DM_OK && onext) r = dalloc_t(c, &tn, std::max<int64_t>(1, o.n));
    if (r != DM_OK) {  // keep the original allocation
      free_table(c, t);
      dfree(c, tn);
      return DM_OK;
    }
    if (o.n > 0) {
      CK(cudaMemcpyAsync(t.rows, o.rows, sizeof(int32_t) * o.n * o.w, cudaMemcpyDeviceToDevice, c->stream));
      if (o.score) CK(cudaMemcpyAsync(t.score, o.score, sizeof(float) * o.n, cudaMemcpyDeviceToDevice, c->stream));
      if (onext) CK(cudaMemcpyAsync(tn, onext, sizeof(int32_t) * o.n, cudaMemcpyDeviceToDevice, c->stream));
    }
    free_table(c, o);
    dfree(c, onext);
    o = t;
    o.held = std::max<int64_t>(1, o.n) * rb;
    onext = tn;
    return DM_OK;
  }

  int run_one(int j, const DevTable &in, int64_t lo, int64_t hi, int64_t cap) {
    DevTable o;
    int32_t *onext = nullptr;
    int64_t ntot = 0;
    RET(launch(j, in, lo, hi, cap, &o, &onext, &ntot));
    if (st[j].base.mode == 1) return DM_OK;
    RET(shrink(j, o, onext, cap));
    c->inflight += o.held;
    return descend(j, o, onext, ntot);
  }

  // Process step j over the rows of `in`; in_next[i] is the candidate count of row i.
  int process(int j, const DevTable &in, const int32_t *in_next, int64_t cand_total) {
    if (in.n == 0) return DM_OK;
    if (max_rows > 0 && cand_total > max_rows) return DM_E_CAPACITY;
    const bool count_last = st[j].base.mode == 1;
    int64_t lim = limit_rows(j);
    if (count_last || cand_total <= lim || in.n == 1) return run_one(j, in, 0, 0, std::max<int64_t>(1, cand_total));
    // chunked streaming: split the input so that each chunk's candidates fit the budget
    int64_t *pre = nullptr, *tmp = nullptr;
    int64_t step = std::max<int64_t>(1, lim - st[j].max_group);
    int64_t nch = (cand_total + step - 1) / step;
    // boundaries (the last row index whose prefix is <= i * step) found on the device; only
    // the nch + 1 boundaries and their prefixes come back
    int64_t *dbound = nullptr;
    {
      int r = dalloc_t(c, &pre, in.n + 1);
      if (r == DM_OK) r = dalloc_t(c, &tmp, dmk::scan_tmp_elems(in.n));
      if (r == DM_OK) r = dalloc_t(c, &dbound, 2 * (nch + 2));
      if (r != DM_OK) {
        dfree(c, pre);
        dfree(c, tmp);
        dfree(c, dbound);
        return r;
      }
    }
    CK(dmk::scan_i32(in_next, pre, in.n, tmp, c->stream));
    CK(dmk::launch_chunk_bounds(pre, in.n, step, nch, dbound, dbound + nch + 1, c->stream));
    std::vector<int64_t> hb(2 * (nch + 1) + 1);
    CK(cudaMemcpyAsync(hb.data(), dbound, sizeof(int64_t) * 2 * (nch + 1), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(hb.data() + 2 * (nch + 1), pre + in.n / 2, sizeof(int64_t), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, dbound);
    dfree(c, pre);
    dfree(c, tmp);
    std::vector<int64_t> b{0}, bp{hb[nch + 1]};  // boundaries and the prefix at each
    for (int64_t i = 1; i < nch; i++)
      if (hb[i] > b.back()) {
        b.push_back(hb[i]);
        bp.push_back(hb[nch + 1 + i]);
      }
    if (b.size() == 1 && in.n > 1) {  // always make progress
      b.push_back(in.n / 2);
      bp.push_back(hb[2 * (nch + 1)]);
    }
    b.push_back(in.n);
    bp.push_back(hb[nch + 1 + nch]);
    for (size_t i = 0; i + 1 < b.size(); i++) {
      int64_t lo = b[i], hi = b[i + 1];
      if (hi <= lo) continue;
      DevTable sub;
      sub.rows = in.rows + lo * in.w;
      sub.score = in.score ? in.score + lo : nullptr;
      sub.n = hi - lo;
      sub.w = in.w;
      int64_t sc = bp[i + 1] - bp[i];
      if (sc == 0) continue;
      if (sc <= limit_rows(j) || sub.n == 1) RET(run_one(j, sub, 0, 0, sc));
      else RET(process(j, sub, in_next + lo, sc));
    }
    return DM_OK;
  }

  // Device-driven execution: every step's output goes to one half of the arena, each launch
  // reads its input row count from the previous launch's counters, and the host waits once
  // at the end. *fits is false when some step overflowed its half (nothing is delivered then).
  int run_fast(bool *fits) {
    const int S = (int)st.size();
    *fits = false;
    size_t half = (c->arena_bytes / 2) / 256 * 256;
    unsigned char *buf[2] = {c->arena, c->arena + half};
    CK(cudaMemsetAsync(c->d_ctr_steps, 0, sizeof(unsigned long long) * CTR_N * S, c->stream));
    if (c->timing) CK(cudaEventRecord(c->ev0, c->stream));
    int32_t *prev_rows = nullptr;
    float *prev_score = nullptr;
    int64_t prev_cap = 0;
    int32_t prev_rs = 0;
    // a counted plan's last two joins run as one kernel when they qualify: the table between
    // them stays in shared memory
    const bool fuse = c->fuse_last && S >= 2 && st[S - 1].base.mode == 1 &&
                      dmk::fused_ok(st[S - 2].base, st[S - 1].base);
    fused = fuse;
    for (int j = 0; j < S; j++) {
      JoinArgs a = st[j].base;
      a.prune = prune;
      a.ctr = c->d_ctr_steps + (size_t)j * CTR_N;
      a.out_next = nullptr;
      a.nx.nkeys = -1;
      // a table the next launch reads has rows padded to 16 bytes (whole-int4 loads and stores)
      bool identity = true;
      for (int q = 0; q < a.wo; q++) identity &= a.src_col[q] == q;
      const bool pad = a.mode == 0 && j + 1 < S && a.n_new >= 1 && a.n_new <= 4 && a.wo == a.w + a.n_new && identity;
      a.rs_out = pad ? (a.wo + 3) / 4 * 4 : 0;
      const int64_t ows = a.rs_out ? a.rs_out : a.wo;  // output row stride in words
      int64_t rb = 4ll * ows + (a.scored ? 4 : 0);
      int64_t cap = std::max<int64_t>(1, ((int64_t)half - 512) / rb);
      int32_t *orows = (int32_t *)buf[j & 1];
      float *oscore = (float *)(buf[j & 1] + ((size_t)cap * ows * 4 + 255) / 256 * 256);
      a.out = a.mode == 0 ? orows : nullptr;
      a.outs = (a.mode == 0 && a.scored) ? oscore : nullptr;
      a.out_cap = cap;
      if (j == 0) {
        a.R = nullptr;
        a.seed_lo = 0;
        a.seed_hi = st[0].seed_table->n;
      } else {
        a.R = prev_rows;
        a.Rs = prev_score;
        a.N = 0;
        a.n_dev = c->d_ctr_steps + (size_t)(j - 1) * CTR_N + CTR_ROWS;
        a.in_cap = prev_cap;
        a.rs_in = prev_rs;
      }
      if (fuse && j == S - 2) {
        JoinArgs b = st[S - 1].base;
        b.prune = prune;
        b.ctr = c->d_ctr_steps + (size_t)(S - 1) * CTR_N;
        b.out_next = nullptr;
        b.nx.nkeys = -1;
        a.out = nullptr;
        a.outs = nullptr;
        a.out_cap = 0;
        CK(dmk::launch_fused(a, b, c->num_sms, c->stream, j > 0));
        break;
      }
      int grid = dmk::wjoin_grid(a, c->num_sms);
      CK(dmk::launch_wjoin(a, grid, c->stream, j > 0));  // steps chain kernel to kernel
      prev_rows = orows;
      prev_score = a.outs;
      prev_cap = cap;
      prev_rs = a.rs_out;
    }
    if (c->timing) CK(cudaEventRecord(c->ev1, c->stream));
    CK(cudaMemcpyAsync(c->h_ctr_steps, c->d_ctr_steps, sizeof(unsigned long long) * CTR_N * S,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int j = 0; j < S; j++)
      if (c->h_ctr_steps[(size_t)j * CTR_N + CTR_OVF]) return DM_OK;  // does not fit: caller falls back
    *fits = true;
    if (c->timing) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      c->stats.join_ms += ms;
    }
    int64_t nin = st[0].seed_table->n;
    for (int j = 0; j < S; j++) {
      const unsigned long long *h = c->h_ctr_steps + (size_t)j * CTR_N;
      const JoinArgs &a = st[j].base;
      int64_t rows = (int64_t)h[CTR_ROWS];
      // fused last two joins: the table between them is neither written nor read
      const bool in_smem = fused && j == S - 1, out_smem = fused && j == S - 2;
      double bytes = (double)st[j].motif_bytes;
      if (j && !in_smem) bytes += (double)nin * (4.0 * a.w + (a.scored ? 4 : 0));
      if (a.mode == 0 && !out_smem) bytes += (double)rows * (4.0 * a.wo + (a.scored ? 4 : 0));
      c->stats.join_bytes += bytes;
      if (!in_smem) c->stats.join_launches++;
      c->stats.chunks++;
      if (j < DM_MAX_STEPS) {
        c->stats.rows[j] += rows;
        c->stats.candidates[j] += (int64_t)h[CTR_CAND];
      }
      if (j + 1 < S) c->stats.max_rows = std::max(c->stats.max_rows, rows);
      nin = rows;
    }
    const unsigned long long *hl = c->h_ctr_steps + (size_t)(S - 1) * CTR_N;
    if (st[S - 1].base.mode == 1) {
      count += hl[CTR_ROWS];
      checksum += hl[CTR_SUM];
      return DM_OK;
    }
    DevTable t;
    t.rows = prev_rows;
    t.score = prev_score;
    t.n = (int64_t)hl[CTR_ROWS];
    t.w = st[S - 1].base.wo;
    t.borrowed = true;
    return sink->take(c, t);
  }

  int ensure_arena(size_t bytes) {
    if (c->arena_bytes >= bytes) return DM_OK;
    if (c->arena) {
      CK(cudaStreamSynchronize(c->stream));
      cudaFree(c->arena);
      c->arena = nullptr;
      c->arena_bytes = 0;
    }
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      return DM_E_NOMEM;
    }
    c->arena_bytes = bytes;
    return DM_OK;
  }

  int run() {
    RET(setup());
    const int S = (int)st.size();
    c->stats.n_steps = S;
    if (chunk_rows == 0 && max_rows == 0 && p->join_algo != DM_JOIN_SORTMERGE && st[0].seed_table->n > 0) {
      // device-driven path first; grow the arena (up to the budget) while a step overflows
      size_t want = std::max<size_t>(c->arena_bytes, (size_t)4 << 30);
      while (true) {
        want = std::min<size_t>(want, (size_t)c->budget);
        if (ensure_arena(want) != DM_OK) break;
        bool fits = false;
        dm_stats saved = c->stats;
        RET(run_fast(&fits));
        if (fits) return DM_OK;
        c->stats = saved;
        if (want >= (size_t)c->budget) break;
        want *= 4;
      }
      if (c->arena_bytes > ((size_t)4 << 30)) {  // streaming needs the budget the arena holds
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->arena);
        c->arena = nullptr;
        c->arena_bytes = 0;
      }
    }
    DevTable *T = st[0].seed_table;
    int64_t n0 = T->n;
    if (n0 == 0) return DM_OK;
    // the seed step: candidates are the motif-table rows, chunked like any other step
    int64_t lim = st[0].base.mode == 1 ? n0 : limit_rows(0);
    for (int64_t lo = 0; lo < n0; lo += lim) {
      int64_t hi = std::min(n0, lo + lim);
      DevTable none;
      RET(run_one(0, none, lo, hi, hi - lo));
    }
    return DM_OK;
  }
};

struct CollectSink : Sink {
  std::vector<DevTable> parts;
  int take(dm_ctx *, DevTable t) override {
    parts.push_back(t);
    return DM_OK;
  }
  int concat(dm_ctx *c, int32_t w, bool scored, DevTable *out) {
    int64_t n = 0;
    for (auto &p : parts) n += p.n;
    DevTable o;
    o.n = n;
    o.w = w;
    RET(dalloc_t(c, &o.rows, (size_t)std::max<int64_t>(1, n) * w));
    if (scored) RET(dalloc_t(c, &o.score, std::max<int64_t>(1, n)));
    int64_t off = 0;
    for (auto &p : parts) {
      if (p.n) {
        CK(cudaMemcpyAsync(o.rows + off * w, p.rows, sizeof(int32_t) * p.n * w, cudaMemcpyDeviceToDevice, c->stream));
        if (scored && p.score)
          CK(cudaMemcpyAsync(o.score + off, p.score, sizeof(float) * p.n, cudaMemcpyDeviceToDevice, c->stream));
      }
      off += p.n;
      free_table(c, p);
    }
    parts.clear();
    *out = o;
    return DM_OK;
  }
};

// Hand a finished table to the user callback (device pointers, or host copies in staging-sized
// pieces). synced: the caller has just synchronised the stream after the table was produced.
int deliver(dm_ctx *c, const DevTable &t, int flags, dm_chunk_cb cb, void *user, bool synced = false) {
  if (!cb || t.n == 0) return DM_OK;
  if (flags & DM_DEVICE_ROWS) {
    if (!synced) CK(cudaStreamSynchronize(c->stream));
    return cb(user, t.rows, t.score, t.n, t.w) ? DM_E_CANCELLED : DM_OK;
  }
  const int64_t rb = 4ll * t.w + (t.score ? 4 : 0);
  int64_t per = std::max<int64_t>(1, (int64_t)c->h_stage_bytes / rb);
  for (int64_t lo = 0; lo < t.n; lo += per) {
    int64_t m = std::min(per, t.n - lo);
    int32_t *hr = (int32_t *)c->h_stage;
    float *hs = t.score ? (float *)(hr + m * t.w) : nullptr;
    CK(cudaMemcpyAsync(hr, t.rows + lo * t.w, sizeof(int32_t) * m * t.w, cudaMemcpyDeviceToHost, c->stream));
    if (hs) CK(cudaMemcpyAsync(hs, t.score + lo, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (cb(user, hr, hs, m, t.w)) return DM_E_CANCELLED;
  }
  return DM_OK;
}

struct TopkSink;
int topk_take(dm_ctx *c, TopkSink *t, DevTable tab);
bool topk_small_enough(const TopkSink *t);
int topk_into_host(dm_ctx *c, TopkSink *t, const DevTable &sorted, int32_t *rows, float *scores, int64_t *n);

struct AllSink : Sink {
  TopkSink *tap = nullptr;  // also feeds every final chunk to a top-k accumulator
  int flags;
  dm_chunk_cb cb;
  void *user;
  int bits;
  std::vector<DevTable> held;
  int64_t held_bytes = 0;
  bool streaming = false;
  uint64_t count = 0, checksum = 0;
  // host buffers of the caller's top-k: when the whole result is one table, its top-k is
  // copied out under the same synchronisation as the count and checksum
  int32_t *final_rows = nullptr;
  float *final_scores = nullptr;
  bool final_done = false;
  int64_t final_n = 0;
  // sort (checksum fused into the key packing), one synchronisation, delivery, then the top-k
  // tap (which takes the table over). last: no table follows, nothing was flushed before.
  int flush_one(dm_ctx *c, DevTable &t, bool last = false) {
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * CTR_N, c->stream));
    RET(sort_canonical(c, t, bits, c->d_ctr));
    const bool fast_topk = last && tap && final_rows && topk_small_enough(tap);
    if (fast_topk) RET(topk_into_host(c, tap, t, final_rows, final_scores, &final_n));
    RET(read_ctr(c));
    final_done = fast_topk;
    count += (uint64_t)t.n;
    checksum += c->h_ctr[CTR_SUM];
    int r = deliver(c, t, flags, cb, user, true);
    if (r == DM_OK && tap && !fast_topk) return topk_take(c, tap, t);  // the tap takes ownership
    free_table(c, t);
    return r;
  }
  int take(dm_ctx *c, DevTable t) override {
    int64_t tb = t.n * (4ll * t.w + (t.score ? 4 : 0));
    if (!streaming && held_bytes + tb <= (int64_t)c->budget / 2) {
      held.push_back(t);
      held_bytes += tb;
      return DM_OK;
    }
    streaming = true;
    for (auto &h : held) RET(flush_one(c, h));
    held.clear();
    held_bytes = 0;
    return flush_one(c, t);
  }
  int finish(dm_ctx *c, int32_t w, bool scored) {
    if (held.empty()) return DM_OK;
    if (held.size() == 1) {  // sorting makes its own copy: no concatenation needed
      DevTable t = held[0];
      held.clear();
      return flush_one(c, t, !streaming);
    }
    CollectSink cs;
    cs.parts = held;
    held.clear();
    DevTable all;
    RET(cs.concat(c, w, scored, &all));
    return flush_one(c, all, !streaming);
  }
};

// Top-k of a table (rows in pattern order + scores) by (score, row): a new table of
// min(k, n) rows in that order.
int topk_table(dm_ctx *c, DevGraph *g, const DevTable &t, int64_t k, DevTable *out) {
  int64_t n = t.n;
  int32_t *idx = nullptr;
  int64_t m = n;
  if (n > k) {
    uint32_t prefix = 0, pmask = 0;
    int64_t kk = k;
    unsigned long long *hist = nullptr;
    RET(dalloc_t(c, &hist, 256));
    for (int shift = 24; shift >= 0; shift -= 8) {
      CK(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), c->stream));
      CK(dmk::launch_score_hist(t.score, n, prefix, pmask, shift, hist, c->stream));
      unsigned long long h[256];
      CK(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      int64_t cum = 0;
      int d = 0;
      for (; d < 256; d++) {
        if (cum + (int64_t)h[d] >= kk) break;
        cum += (int64_t)h[d];
      }
      kk -= cum;
      prefix |= (uint32_t)d << shift;
      pmask |= 255u << shift;
    }
    dfree(c, hist);
    RET(dalloc_t(c, &idx, n));
    CK(cudaMemsetAsync(c->d_ctr, 0, sizeof(unsigned long long) * CTR_N, c->stream));
    CK(dmk::launch_select_le(t.score, n, prefix, idx, c->d_ctr, c->stream));
    RET(read_ctr(c));
    m = (int64_t)c->h_ctr[0];
  } else {
    RET(dalloc_t(c, &idx, std::max<int64_t>(1, n)));
    CK(dmk::launch_iota(idx, n, c->stream));
  }
  DevTable cand;
  RET(gather_table(c, t, idx, m, &cand));
  dfree(c, idx);
  // (score, row) order: canonical sort by row, then a stable sort by score
  RET(sort_canonical(c, cand, graph_bits(g)));
  int32_t *perm = nullptr;
  RET(dalloc_t(c, &perm, std::max<int64_t>(1, m)));
  CK(dmk::launch_iota(perm, m, c->stream));
  RET(stable_sort_perm_by_score(c, cand, perm));
  DevTable o;
  RET(gather_table(c, cand, perm, std::min(k, m), &o));
  dfree(c, perm);
  free_table(c, cand);
  *out = o;
  return DM_OK;
}

// k best of a canonically sorted table (rows in pattern order + scores), in (score, row)
// order; consumes t.
int topk_of_sorted(dm_ctx *c, DevGraph *g, DevTable &t, int64_t k, DevTable *out) {
  if (k > 1024) {  // large k: select by radix on the order-preserving score keys, then sort the candidates
    RET(topk_table(c, g, t, k, out));
    free_table(c, t);
    return DM_OK;
  }
  DevTable o;
  o.w = t.w;
  o.n = std::min<int64_t>(k, t.n);
  RET(dalloc_t(c, &o.rows, (size_t)std::max<int64_t>(1, o.n) * t.w));
  RET(dalloc_t(c, &o.score, std::max<int64_t>(1, o.n)));
  if (o.n > 0) {
    void *tmp = nullptr;
    RET(dalloc(c, &tmp, (size_t)dmk::topk_tmp_bytes(t.n)));
    CK(dmk::topk_sorted(t.rows, t.score, t.n, t.w, (int32_t)k, tmp, o.rows, o.score, c->stream));
    dfree(c, tmp);
  }
  free_table(c, t);
  *out = o;
  return DM_OK;
}

struct TopkSink : Sink {
  DevGraph *g;
  int64_t k;
  bool input_sorted = false;  // tables arrive in canonical order (from AllSink)
  DevTable best;              // current best min(k, seen) rows, (score, row) order
  bool have = false;
  float *prune_ptr = nullptr;
  int take(dm_ctx *c, DevTable t) override {
    DevTable tk;
    if (!input_sorted && t.n > 16384) {
      // a large unsorted table: select by score first and sort only the candidates, instead
      // of sorting every row into canonical order
      RET(topk_table(c, g, t, k, &tk));
      free_table(c, t);
    } else {
      if (!input_sorted || t.borrowed) RET(sort_canonical(c, t, graph_bits(g)));
      RET(topk_of_sorted(c, g, t, k, &tk));
    }
    if (have) {
      CollectSink cs;
      cs.parts = {best, tk};
      DevTable both;
      RET(cs.concat(c, tk.w, true, &both));
      RET(sort_canonical(c, both, graph_bits(g)));
      RET(topk_of_sorted(c, g, both, k, &best));
    } else {
      best = tk;
      have = true;
    }
    if (prune_ptr && best.n == k) {  // rows scoring above the k-th best can never enter
      float kth;
      CK(cudaMemcpyAsync(&kth, best.score + (k - 1), sizeof(float), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      *prune_ptr = kth;
    }
    return DM_OK;
  }
};

int topk_take(dm_ctx *c, TopkSink *t, DevTable tab) { return t->take(c, tab); }

// Direction-aware post-processing (Sec. 5.4 footnote): every delivered table gets its rows'
// direction-aware scores (k_rescore_directed over the pattern's weighted slots) in place of the
// undirected ones, then goes to the top-k.
struct DirectedSink : Sink {
  DevGraph *g = nullptr;
  TopkSink *tk = nullptr;
  int32_t np = 0, nslots = 0;
  const int32_t *sp = nullptr, *sq = nullptr;
  const float *sw = nullptr;
  int take(dm_ctx *c, DevTable t) override {
    float *dsc = nullptr;
    RET(dalloc_t(c, &dsc, std::max<int64_t>(1, t.n)));
    CK(dmk::launch_rescore_directed(t.rows, t.n, np, sp, sq, sw, nslots, g->row_ptr, g->col_idx, g->edir, g->qerr,
                                    dsc, c->stream));
    if (!t.borrowed) dfree(c, t.score);
    DevTable s = t;
    s.score = dsc;
    const int r = tk->take(c, s);
    if (t.borrowed) dfree(c, dsc);  // the top-k keeps copies; a borrowed table's holder frees nothing
    return r;
  }
};

bool topk_small_enough(const TopkSink *t) { return !t->have && t->k <= 1024; }

// Top-k of a canonically sorted table straight into the caller's host buffers (enqueued on
// the stream; the caller synchronises); the table stays with the caller.
int topk_into_host(dm_ctx *c, TopkSink *t, const DevTable &sorted, int32_t *rows, float *scores, int64_t *n) {
  const int64_t m = std::min<int64_t>(t->k, sorted.n);
  *n = m;
  if (m <= 0) return DM_OK;
  DevTable o;
  o.w = sorted.w;
  o.n = m;
  RET(dalloc_t(c, &o.rows, (size_t)m * sorted.w));
  RET(dalloc_t(c, &o.score, m));
  void *tmp = nullptr;
  RET(dalloc(c, &tmp, (size_t)dmk::topk_tmp_bytes(sorted.n)));
  CK(dmk::topk_sorted(sorted.rows, sorted.score, sorted.n, sorted.w, (int32_t)t->k, tmp, o.rows, o.score, c->stream));
  dfree(c, tmp);
  CK(cudaMemcpyAsync(rows, o.rows, sizeof(int32_t) * m * o.w, cudaMemcpyDeviceToHost, c->stream));
  if (scores) CK(cudaMemcpyAsync(scores, o.score, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
  free_table(c, o);
  return DM_OK;
}

int ensure_motif(dm_ctx *c, DevGraph *g, int id);

int build_motif_by_joins(dm_ctx *c, DevGraph *g, const MotifDef &md) {
  // Alg. 2: Res(M) <- Delta-Motif(M, DB), with DB = Res(M2) plus the smaller motifs built so far
  Plan mp;
  mp.n_p = md.k;
  std::vector<std::vector<int>> adj(md.k);
  for (auto &e : md.edges) {
    adj[e.first].push_back(e.second);
    adj[e.second].push_back(e.first);
  }
  mp.rp.assign(md.k + 1, 0);
  for (int u = 0; u < md.k; u++) {
    std::sort(adj[u].begin(), adj[u].end());
    mp.rp[u + 1] = mp.rp[u] + (int)adj[u].size();
    for (int v : adj[u]) mp.ci.push_back(v);
  }
  std::vector<int32_t> set{2};
  for (auto &kv : g->motifs) {
    MotifDef d;
    if (kv.first >= 2 && motif_def(kv.first, &d) && d.k < md.k) set.push_back(kv.first);
  }
  RET(ensure_motif(c, g, 2));
  GraphStats gs;
  gs.V = g->V;
  int r = decompose(mp, set, DM_ORDER_PAPER, gs, &mp.steps, mp.col_vertex);
  if (r != DM_OK) return r;
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &mp;
  ex.mode = DM_ALL;
  ex.use_qerr = false;
  CollectSink sink;
  ex.sink = &sink;
  dm_stats saved = c->stats;
  r = ex.run();
  c->stats = saved;
  if (r != DM_OK) return r;
  DevTable t;
  RET(sink.concat(c, md.k, g->eerr != nullptr, &t));
  g->motifs[md.id] = t;
  return DM_OK;
}

int ensure_motif(dm_ctx *c, DevGraph *g, int id) {
  if (g->motifs.count(id)) return DM_OK;
  DevTable t;
  if (id == MOTIF_VERTEX) {
    t.n = g->V;
    t.w = 1;
    RET(dalloc_t(c, &t.rows, std::max(1, g->V)));
    if (g->eerr) RET(dalloc_t(c, &t.score, std::max(1, g->V)));
    CK(dmk::launch_vertex_table(g->V, t.rows, t.score, c->stream));
    g->motifs[id] = t;
    return DM_OK;
  }
  if (id == 2) {
    t.n = g->nnz;
    t.w = 2;
    RET(dalloc_t(c, &t.rows, (size_t)std::max<int64_t>(1, g->nnz) * 2));
    if (g->eerr) RET(dalloc_t(c, &t.score, std::max<int64_t>(1, g->nnz)));
    CK(dmk::launch_csr_to_m2(g->row_ptr, g->col_idx, g->eerr, g->V, g->nnz, t.rows, t.score, c->stream));
    g->motifs[id] = t;
    return DM_OK;
  }
  MotifDef md;
  if (!motif_def(id, &md)) return DM_E_NOTFOUND;
  return build_motif_by_joins(c, g, md);
}

}  // namespace

// Device image of a batch of plans for the persistent kernel, with its tuned launch shape
// and the CUDA graph that replays memsets + launch + result copy.
struct BatchState {
  std::vector<const dm_plan_t *> key;
  double hash_lf = 0, heavy_rows = 0;
  std::vector<int32_t> light, heavy;  // plans in the persistent launch / run step by step
  int TR = 64;
  int64_t root_chunk = 16;
  int threads = 256;                  // block shape of the persistent launch: threads per CTA
  int ctas_per_sm = 0;                // ... and resident CTAs per SM (0 = as many as fit)
  void *d_left0 = nullptr;            // items per plan (copied into the live counters each run)
  dmk::BatchParams prm{};
  int grid = 0;
  void *d_args = nullptr, *d_plans = nullptr, *d_items = nullptr, *d_work = nullptr, *scratch = nullptr;
  unsigned long long *h_out = nullptr;
  int32_t n_plans = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool tuned = false;
};

namespace {

void batch_release(dm_ctx *c, BatchState *b) {
  if (!b) return;
  cudaStreamSynchronize(c->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_args);
  cudaFree(b->d_plans);
  cudaFree(b->d_items);
  cudaFree(b->d_work);
  cudaFree(b->d_left0);
  cudaFree(b->scratch);
  if (b->h_out) cudaFreeHost(b->h_out);
  delete b;
}

int batch_build(dm_ctx *c, DevGraph *g, const dm_plan_t *const *plans, int32_t n, int TR, int64_t root_chunk,
                double heavy_rows, int threads, int ctas_per_sm, BatchState **out);

DevGraph *get_graph(dm_ctx *c, dm_graph g) {
  if (!c || g < 0 || g >= (int)c->graphs.size()) return nullptr;
  return c->graphs[g];
}

int batch_build(dm_ctx *c, DevGraph *g, const dm_plan_t *const *plans, int32_t n, int TR, int64_t root_chunk,
                double heavy_rows, int threads, int ctas_per_sm, BatchState **out) {
  std::unique_ptr<BatchState> b(new BatchState());
  b->key.assign(plans, plans + n);
  b->hash_lf = c->hash_lf;
  b->heavy_rows = heavy_rows;
  b->root_chunk = root_chunk;
  const bool walk = threads == 32;  // one depth-first walk per warp (k_batchw): 32-row tiles
  if (walk) TR = 32;
  b->TR = TR;
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  b->n_plans = n;
  std::vector<uint64_t> items_per(n, 0);
  std::vector<JoinArgs> args;
  std::vector<dmk::BatchPlan> bplans(n);
  std::vector<std::pair<double, dmk::BatchItem>> items;
  std::vector<int64_t> cap(MAXSTEPS, 0), maxw(MAXSTEPS, 0);
  int ws_max = 1, max_steps = 1;
  bool wide = false;  // some step maps more than 4 new vertices
  for (int32_t i = 0; i < n; i++) {
    if (plans[i]->p.pred_max_rows > heavy_rows) {  // runs step by step after the launch
      b->heavy.push_back(i);
      continue;
    }
    b->light.push_back(i);
    Exec ex;
    ex.c = c;
    ex.g = g;
    ex.p = &plans[i]->p;
    ex.mode = DM_COUNT;
    ex.use_qerr = false;
    RET(ex.setup());
    const int S = (int)ex.st.size();
    bplans[i].n_steps = S;
    bplans[i].args_off = (int32_t)args.size();
    max_steps = std::max(max_steps, S);
    double cost = 0;
    for (int j = 0; j < S; j++) {
      JoinArgs a = ex.st[j].base;
      a.scored = 0;
      a.qerr = nullptr;
      a.eerr = nullptr;
      a.out_next = nullptr;
      a.nx.nkeys = -1;
      a.prune = INFINITY;
      a.rs_in = 0;
      a.rs_out = 0;
      if (walk && a.mode == 0 && j + 1 < S && a.n_new >= 1 && a.n_new <= 4 && a.wo == a.w + a.n_new) {
        // warp walks keep a level's rows padded to 16 bytes when its columns are in working order
        bool identity = true;
        for (int q = 0; q < a.wo; q++) identity &= a.src_col[q] == q;
        if (identity) a.rs_out = (a.wo + 3) / 4 * 4;
      }
      args.push_back(a);
      ws_max = std::max(ws_max, join_row_stride(a.w));
      wide |= j > 0 && a.n_new > 4;
      maxw[j] = std::max<int64_t>(maxw[j], a.rs_out ? a.rs_out : a.wo);
      if (j > 0) cap[j] = std::max<int64_t>(cap[j], (int64_t)TR * ex.st[j].max_group);
      cost += ex.p->steps[j].est_rows;
    }
    // root chunks: the tuned size, larger for plans whose first table is so long that the
    // tuned size would cut it into many more items than the GPU has CTAs (per-item overhead)
    int64_t n0 = ex.st[0].seed_table->n;
    const int64_t chunk = std::max<int64_t>(root_chunk, (n0 + 4ll * c->num_sms - 1) / (4ll * c->num_sms));
    cap[0] = std::max<int64_t>(cap[0], chunk);
    for (int64_t lo = 0; lo < n0; lo += chunk) {
      dmk::BatchItem it{};
      it.plan = i;
      it.lo = lo;
      it.hi = std::min(n0, lo + chunk);
      items.push_back({cost / std::max<double>(1.0, (double)(n0 + chunk - 1) / chunk), it});
      items_per[i]++;
    }
  }
  // expensive chunks first: the tail of the persistent loop is made of cheap ones
  std::stable_sort(items.begin(), items.end(), [](const std::pair<double, dmk::BatchItem> &x,
                                                  const std::pair<double, dmk::BatchItem> &y) { return x.first > y.first; });
  std::vector<dmk::BatchItem> hitems(items.size());
  for (size_t i = 0; i < items.size(); i++) hitems[i] = items[i].second;
  dmk::BatchParams &P = b->prm;
  int64_t off = 0;
  for (int j = 0; j < MAXSTEPS; j++) {
    P.lvl_off[j] = off;
    P.lvl_cap[j] = cap[j];
    off += (cap[j] * std::max<int64_t>(1, maxw[j]) * 4 + 255) / 256 * 256;
  }
  P.cta_bytes = off;  // per CTA, or per warp for warp walks
  P.TR = TR;
  P.ws_max = ws_max;
  P.max_steps = max_steps;
  // wide steps test injectivity in per-row id bitmaps when the graph is small enough for them
  P.bm_words = 0;
  if (!walk && wide && g->V <= 2048) {
    const int bw = (g->V + 63) / 64;
    if (dmk::batch_smem_bytes(TR, ws_max, bw, threads) <= 160 * 1024) P.bm_words = bw;
  }
  P.n_items = (int64_t)hitems.size();
  const int64_t slices = walk ? dmk::BW_WALK_WARPS : 1;  // scratch slices a CTA holds
  P.tile_words = 32 * std::min(ws_max, dmk::BW_WALK_TILE_STRIDE);  // >= 6 rows of the widest (132 words)
  if (walk) {
    if (dmk::walk_smem_bytes(P.tile_words, max_steps) > 200 * 1024) return DM_E_CAPACITY;
    b->grid = dmk::walk_grid(P.tile_words, max_steps, c->num_sms, ctas_per_sm);
  } else {
    b->grid = dmk::batch_grid(TR, ws_max, P.bm_words, c->num_sms, threads, ctas_per_sm);
  }
  while (b->grid > c->num_sms && (uint64_t)b->grid * slices * P.cta_bytes > c->budget / 2) b->grid /= 2;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return DM_E_NOMEM;
    }
    cudaError_t e = bytes ? cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(c, e, "batch upload");
    return DM_OK;
  };
  RET(up(&b->d_args, args.data(), sizeof(JoinArgs) * args.size()));
  RET(up(&b->d_plans, bplans.data(), sizeof(dmk::BatchPlan) * bplans.size()));
  RET(up(&b->d_items, hitems.data(), sizeof(dmk::BatchItem) * hitems.size()));
  // work counter, overflow flag, (count, checksum) per plan, items left per plan, done times,
  // start time
  if (cudaMalloc(&b->d_work, sizeof(unsigned long long) * (3 + 4 * (size_t)n)) != cudaSuccess) {
    cudaGetLastError();
    return DM_E_NOMEM;
  }
  RET(up(&b->d_left0, items_per.data(), sizeof(uint64_t) * n));
  if (cudaMalloc(&b->scratch, std::max<size_t>(16, (size_t)b->grid * slices * P.cta_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return DM_E_NOMEM;
  }
  if (cudaMallocHost(&b->h_out, sizeof(unsigned long long) * (3 + 4 * (size_t)n)) != cudaSuccess) return DM_E_NOMEM;
  unsigned long long *work = (unsigned long long *)b->d_work;
  P.args = (const JoinArgs *)b->d_args;
  P.plans = (const dmk::BatchPlan *)b->d_plans;
  P.items = (const dmk::BatchItem *)b->d_items;
  P.next_item = work;
  P.ovf = work + 1;
  P.out = work + 2;
  P.plan_left = work + 2 + 2 * n;
  P.plan_done = work + 2 + 3 * n;
  P.start_ns = work + 2 + 4 * n;
  P.scratch = (unsigned char *)b->scratch;
  *out = b.release();
  return DM_OK;
}

// One execution of a built batch: reset counters, run the persistent kernel, copy the results
// back. The sequence is captured once into a CUDA graph and replayed afterwards.
int batch_run(dm_ctx *c, DevGraph *g, BatchState *b) {
  const size_t n = (size_t)b->n_plans;
  size_t wbytes = sizeof(unsigned long long) * (3 + 4 * n);
  auto t0 = std::chrono::steady_clock::now();
  c->batch_latency.assign(n, 0.0);
  if (!b->light.empty()) {
    if (!b->exec) {
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaMemsetAsync(b->d_work, 0, sizeof(unsigned long long) * (2 + 2 * n), cs);
        cudaMemcpyAsync((unsigned long long *)b->d_work + 2 + 2 * n, b->d_left0, sizeof(unsigned long long) * n,
                        cudaMemcpyDeviceToDevice, cs);
        if (b->threads == 32) dmk::launch_batch_walk(b->prm, b->grid, cs);
        else dmk::launch_batch(b->prm, b->grid, b->threads, cs);
        cudaMemcpyAsync(b->h_out, b->d_work, wbytes, cudaMemcpyDeviceToHost, cs);
        e = cudaStreamEndCapture(cs, &b->graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) return cuda_fail(c, e, "batch graph capture");
    } else {
      dmk::g_launches++;  // the replayed graph holds one launch of the batch kernel
    }
    CK(cudaGraphLaunch(b->exec, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (b->h_out[1]) {
      c->last_error = "batch level buffer overflow";
      return DM_E_CAPACITY;
    }
    // GPU global-timer offset of each plan's last item from the start of the launch
    unsigned long long st = b->h_out[2 + 4 * n];
    for (int32_t i : b->light) {
      unsigned long long d = b->h_out[2 + 3 * n + i];
      c->batch_latency[i] = d > st ? (double)(d - st) * 1e-6 : 0.0;
    }
  }
  for (int32_t i : b->heavy) {  // expensive plans: every step over the whole GPU
    Exec ex;
    ex.c = c;
    ex.g = g;
    ex.p = &b->key[i]->p;
    ex.mode = DM_COUNT;
    ex.use_qerr = false;
    c->inflight = 0;
    dm_stats saved = c->stats;
    RET(ex.run());
    c->stats = saved;
    b->h_out[2 + 2 * i] = ex.count;
    b->h_out[3 + 2 * i] = ex.checksum;
    c->batch_latency[i] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return DM_OK;
}

// Model input of a planner feature vector: the model predicts growth, so the absolute
// estimate f[0] is dropped and the heuristic's absolute estimate f[22] becomes its growth.
void model_input(const float *f, float *x) {
  for (int i = 0; i < NFEAT; i++) x[i] = f[i];
  x[22] = f[22] - f[0];
  x[0] = 0.f;
}

// Log (features, observed log growth) of every executed step of a plan (training data).
void log_plan_steps(dm_ctx *c, const Plan &p) {
  if (!c->log_steps || c->log_target.size() > (size_t)4 << 20) return;
  double prev = 0.0;
  for (size_t j = 0; j < p.steps.size() && j < (size_t)DM_MAX_STEPS; j++) {
    double cur = log1p((double)c->stats.rows[j]);
    float x[NFEAT];
    model_input(p.steps[j].feat, x);
    c->log_feat.insert(c->log_feat.end(), x, x + NFEAT);
    c->log_target.push_back((float)(cur - prev));
    prev = cur;
  }
}

int model_alloc(dm_ctx *c) {
  if (c->m_params) return DM_OK;
  size_t b = sizeof(float) * (size_t)dmk::mlp_param_count();
  if (cudaMalloc(&c->m_params, b) != cudaSuccess || cudaMalloc(&c->m_grads, b) != cudaSuccess ||
      cudaMalloc(&c->m_m, b) != cudaSuccess || cudaMalloc(&c->m_v, b) != cudaSuccess) {
    cudaGetLastError();
    return DM_E_NOMEM;
  }
  CK(cudaMemset(c->m_grads, 0, b));
  CK(cudaMemset(c->m_m, 0, b));
  CK(cudaMemset(c->m_v, 0, b));
  return DM_OK;
}

// Forward (and backward when targets and grads are given) over n samples of raw inputs.
int model_run(dm_ctx *c, const float *x_host, const float *t_host, int32_t n, float *y_host, float *grads_dev,
              float *loss_host) {
  int rows = (n + 15) / 16 * 16;
  float *X = nullptr, *T = nullptr, *Y = nullptr, *L = nullptr;
  void *work = nullptr;
  RET(dalloc_t(c, &X, (size_t)rows * NFEAT));
  RET(dalloc_t(c, &Y, rows));
  RET(dalloc_t(c, &L, 1));
  RET(dalloc(c, &work, (size_t)dmk::mlp_work_bytes(rows)));
  CK(cudaMemsetAsync(X, 0, sizeof(float) * rows * NFEAT, c->stream));
  CK(cudaMemcpyAsync(X, x_host, sizeof(float) * n * NFEAT, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(L, 0, sizeof(float), c->stream));
  if (t_host) {
    RET(dalloc_t(c, &T, rows));
    CK(cudaMemsetAsync(T, 0, sizeof(float) * rows, c->stream));
    CK(cudaMemcpyAsync(T, t_host, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
  }
  CK(dmk::mlp_forward_backward(c->m_params, X, T, rows, n, Y, grads_dev, L, work, c->stream));
  if (y_host) CK(cudaMemcpyAsync(y_host, Y, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
  if (loss_host) CK(cudaMemcpyAsync(loss_host, L, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  // the tensor-core timeout flag, into a pinned counter slot that no other call of this
  // context uses while the model runs
  unsigned long long *flag_host = c->h_ctr + CTR_N - 1;
  *flag_host = 0;
  CK(cudaMemcpyAsync(flag_host, dmk::mlp_error_flag(work, rows), sizeof(unsigned), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const unsigned long long timed_out = *flag_host;
  dfree(c, X);
  dfree(c, T);
  dfree(c, Y);
  dfree(c, L);
  dfree(c, work);
  if (timed_out) {
    c->last_error = "a tensor-core wait of the cardinality model timed out";
    return DM_E_TIMEOUT;
  }
  return DM_OK;
}

void normalise(const dm_ctx *c, const float *x, int32_t n, std::vector<float> &out) {
  out.resize((size_t)n * NFEAT);
  for (int32_t i = 0; i < n; i++)
    for (int k = 0; k < NFEAT; k++) out[(size_t)i * NFEAT + k] = (x[(size_t)i * NFEAT + k] - c->m_mean[k]) / c->m_std[k];
}

// Predicted cost of a plan: bytes of every intermediate table it writes (rows from the chain
// of predicted log growths, model or heuristic) plus 64 KiB per step for launch and barrier
// overheads; and its largest predicted table.
// Costs of several plans with one model evaluation over all their steps (see plan_cost).
int plan_costs(dm_ctx *c, const std::vector<const std::vector<StepSpec> *> &plans, std::vector<double> *cost,
               std::vector<double> *max_rows, std::vector<std::vector<float>> *growths) {
  int total = 0;
  for (auto *st : plans) total += (int)st->size();
  std::vector<float> x((size_t)std::max(1, total) * NFEAT), growth(std::max(1, total));
  int k = 0;
  for (auto *st : plans)
    for (auto &s : *st) {
      model_input(s.feat, &x[(size_t)k * NFEAT]);
      growth[k] = x[(size_t)k * NFEAT + 22];
      k++;
    }
  if (total > 0) {
    std::vector<float> xn;
    normalise(c, x.data(), total, xn);
    RET(model_run(c, xn.data(), nullptr, total, growth.data(), nullptr, nullptr));
  }
  cost->assign(plans.size(), 0.0);
  max_rows->assign(plans.size(), 0.0);
  growths->assign(plans.size(), {});
  k = 0;
  for (size_t i = 0; i < plans.size(); i++) {
    double lr = 0, tot = 0, mx = 0;
    for (auto &s : *plans[i]) {
      (*growths)[i].push_back(growth[k]);
      lr += growth[k++];
      double rows = exp(std::min(60.0, std::max(-60.0, lr)));
      mx = std::max(mx, rows);
      tot += rows * (4.0 * s.w_out + 4.0) + 65536.0;
    }
    (*cost)[i] = tot;
    (*max_rows)[i] = mx;
  }
  return DM_OK;
}

int plan_cost(dm_ctx *c, const std::vector<StepSpec> &steps, bool use_model, double *cost, double *max_rows,
              std::vector<float> *growth_out = nullptr) {
  const int n = (int)steps.size();
  std::vector<float> x((size_t)std::max(1, n) * NFEAT), growth(std::max(1, n));
  for (int j = 0; j < n; j++) {
    model_input(steps[j].feat, &x[(size_t)j * NFEAT]);
    growth[j] = x[(size_t)j * NFEAT + 22];
  }
  if (use_model && n > 0) {
    std::vector<float> xn;
    normalise(c, x.data(), n, xn);
    RET(model_run(c, xn.data(), nullptr, n, growth.data(), nullptr, nullptr));
  }
  double lr = 0, total = 0, mx = 0;
  for (int j = 0; j < n; j++) {
    lr += growth[j];
    double rows = exp(std::min(60.0, std::max(-60.0, lr)));
    mx = std::max(mx, rows);
    total += rows * (4.0 * steps[j].w_out + 4.0) + 65536.0;
  }
  *cost = total;
  *max_rows = mx;
  if (growth_out) growth_out->assign(growth.begin(), growth.begin() + n);
  return DM_OK;
}

// The candidate decompositions DM_ORDER_LEARNED chooses from: the paper's rule and the greedy
// heuristic order, each over the plan's motif set and over sets with a motif typical of the
// topology (M8, M12-O or the claw M4-1 at degree <= 3, M6-2O or M6 at degree 4), and, for patterns of
// 16+ vertices, over a set with two paths of about half the pattern: a long cycle then becomes
// one path joined with a second path on both of its end vertices (a two-key join) instead of
// a path grown to nearly the pattern's length and closed by a back-edge. Half-length paths are
// offered only when their tables are estimated (edges x branching^(k - 2)) at 4M rows or less.
struct CandidatePlan {
  std::vector<int32_t> motifs;
  int order = DM_ORDER_PAPER;
  std::vector<StepSpec> steps;
  int32_t col_vertex[MAXW] = {};
};

// The candidate motif sets of a pattern; builds their motif tables (device work, calling
// thread) and adds them to the graph statistics.
int candidate_sets(dm_ctx *c, DevGraph *g, const Plan &p, bool user_motifs, GraphStats &gs,
                   std::vector<std::vector<int32_t>> *out) {
  std::vector<std::vector<int32_t>> &sets = *out;
  sets.assign(1, p.motifs);
  std::vector<int32_t> extra;
  if (!user_motifs) {
    if (g->max_deg <= 3) extra = {8, DM_MOTIF_CYCLE(12), DM_MOTIF_M4_1};
    else if (g->max_deg == 4) extra = {DM_MOTIF_M6_2O, 6};
    else extra = {4};
  }
  for (int id : extra) {
    RET(ensure_motif(c, g, id));
    gs.motifs.push_back({id, g->motifs.at(id).n});
    std::vector<int32_t> set{id};
    set.insert(set.end(), p.motifs.begin(), p.motifs.end());
    sets.push_back(set);
  }
  if (!user_motifs && p.n_p >= 16) {
    const int a = p.n_p / 2 + 1, b = (p.n_p + 1) / 2 + 1;
    const double branch = std::max(1.0, g->avg_deg - 1.0);
    const double est = (double)g->nnz * pow(branch, (double)(b - 2));
    if (b <= MAXM && est <= 4.0e6) {
      std::vector<int32_t> set{b};
      if (a != b) set.push_back(a);
      for (int id : set) {
        RET(ensure_motif(c, g, id));
        gs.motifs.push_back({id, g->motifs.at(id).n});
      }
      set.insert(set.end(), p.motifs.begin(), p.motifs.end());
      sets.push_back(set);
    }
  }
  return DM_OK;
}

// Every (motif set, order) decomposition of a pattern; host work only.
void decompose_candidates(const Plan &p, const std::vector<std::vector<int32_t>> &sets, const GraphStats &gs,
                          std::vector<CandidatePlan> *out) {
  out->clear();
  for (auto &set : sets)
    for (int ord : {DM_ORDER_PAPER, DM_ORDER_HEURISTIC}) {
      CandidatePlan cp;
      cp.motifs = set;
      cp.order = ord;
      if (decompose(p, set, ord, gs, &cp.steps, cp.col_vertex) != DM_OK) continue;
      out->push_back(std::move(cp));
    }
}

int candidate_plans(dm_ctx *c, DevGraph *g, const Plan &p, bool user_motifs, GraphStats &gs,
                    std::vector<CandidatePlan> *out) {
  std::vector<std::vector<int32_t>> sets;
  RET(candidate_sets(c, g, p, user_motifs, gs, &sets));
  decompose_candidates(p, sets, gs, out);
  return DM_OK;
}

void reset_stats(dm_ctx *c) {
  memset(&c->stats, 0, sizeof(c->stats));
  c->stats.kernel_launches = -dmk::launch_count();
}
void finish_stats(dm_ctx *c, std::chrono::steady_clock::time_point t0) {
  c->stats.kernel_launches += dmk::launch_count();
  c->stats.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

// Change the load factor of two-key hash indices: the existing ones are dropped (after the
// stream drains) and rebuilt at the new factor when a plan next needs them.
void set_hash_load_factor(dm_ctx *c, double lf) {
  if (lf == c->hash_lf) return;
  cudaStreamSynchronize(c->stream);
  c->hash_lf = lf;
  for (DevGraph *g : c->graphs) {
    if (!g) continue;
    for (auto it = g->indices.begin(); it != g->indices.end();) {
      if (it->second.v.nkeys == 2 && !it->second.keys) {
        dfree(c, it->second.rows);
        if (it->second.score) dfree(c, it->second.score);
        dfree(c, it->second.slots);
        it = g->indices.erase(it);
      } else {
        ++it;
      }
    }
  }
}

// Everything a data graph holds on the device: CSR, weights, bitmap, motif tables, indices.
void free_graph(dm_ctx *c, DevGraph *g) {
  if (!g) return;
  for (auto &kv : g->motifs) {
    dfree(c, kv.second.rows);
    if (kv.second.score) dfree(c, kv.second.score);
  }
  for (auto &kv : g->indices) {
    dfree(c, kv.second.rows);
    if (kv.second.score) dfree(c, kv.second.score);
    if (kv.second.offsets) dfree(c, kv.second.offsets);
    if (kv.second.slots) dfree(c, kv.second.slots);
    if (kv.second.keys) dfree(c, kv.second.keys);
  }
  cudaFree(g->row_ptr);
  cudaFree(g->col_idx);
  cudaFree(g->eerr);
  cudaFree(g->qerr);
  cudaFree(g->edir);
  cudaFree(g->adj);
  delete g;
}

// =================================================================== C ABI ==============
extern "C" {

const char *dm_strerror(int code) {
  switch (code) {
    case DM_OK: return "ok";
    case DM_E_INVAL: return "invalid argument or malformed graph";
    case DM_E_DISCONNECTED: return "graph not connected";
    case DM_E_NOMEM: return "out of memory";
    case DM_E_CAPACITY: return "capacity exceeded";
    case DM_E_TIMEOUT: return "device wait timed out";
    case DM_E_CUDA: return "CUDA error";
    case DM_E_CANCELLED: return "cancelled by callback";
    case DM_E_NOTFOUND: return "unknown graph or motif";
    default: return "unknown error";
  }
}

const char *dm_last_error(dm_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int dm_create(dm_ctx **out, int device, uint64_t mem_budget_bytes) {
  if (!out) return DM_E_INVAL;
  dm_ctx *c = new dm_ctx();
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    return DM_E_CUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return DM_E_CUDA;
  }
  c->stream = c->own;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (cudaMalloc(&c->d_ctr, sizeof(unsigned long long) * CTR_N) != cudaSuccess ||
      cudaMallocHost(&c->h_ctr, sizeof(unsigned long long) * CTR_N) != cudaSuccess) {
    dm_destroy(c);
    return DM_E_NOMEM;
  }
  if (cudaMalloc(&c->d_ctr_steps, sizeof(unsigned long long) * CTR_N * DM_MAX_STEPS) != cudaSuccess ||
      cudaMallocHost(&c->h_ctr_steps, sizeof(unsigned long long) * CTR_N * DM_MAX_STEPS) != cudaSuccess) {
    dm_destroy(c);
    return DM_E_NOMEM;
  }
  c->h_stage_bytes = 64ull << 20;
  if (cudaMallocHost(&c->h_stage, c->h_stage_bytes) != cudaSuccess) {
    dm_destroy(c);
    return DM_E_NOMEM;
  }
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  if (dm_set_budget(c, mem_budget_bytes) != DM_OK) {
    dm_destroy(c);
    return DM_E_CUDA;
  }
  *out = c;
  return DM_OK;
}

int dm_set_budget(dm_ctx *c, uint64_t bytes) {
  if (!c) return DM_E_INVAL;
  cudaSetDevice(c->device);
  if (bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return DM_E_CUDA;
    bytes = fr / 2;
  }
  c->budget = bytes;
  return DM_OK;
}

int dm_set_stream(dm_ctx *c, void *stream) {
  if (!c) return DM_E_INVAL;
  c->stream = stream ? (cudaStream_t)stream : c->own;
  return DM_OK;
}

int dm_destroy(dm_ctx *c) {
  if (!c) return DM_E_INVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  batch_release(c, c->batch);
  c->batch = nullptr;
  for (DevGraph *g : c->graphs) free_graph(c, g);
  cudaStreamSynchronize(c->stream);
  if (c->d_ctr) cudaFree(c->d_ctr);
  if (c->d_ctr_steps) cudaFree(c->d_ctr_steps);
  if (c->h_ctr_steps) cudaFreeHost(c->h_ctr_steps);
  if (c->arena) cudaFree(c->arena);
  cudaFree(c->m_params);
  cudaFree(c->m_grads);
  cudaFree(c->m_m);
  cudaFree(c->m_v);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
  return DM_OK;
}

int dm_load_data_graph(dm_ctx *c, int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *edge_err,
                       const float *qubit_err, dm_graph *out) {
  return dm_load_data_graph_ex(c, n, row_ptr, col_idx, edge_err, qubit_err, DM_SCORE_ERROR_SUM, out);
}

int dm_load_data_graph_ex(dm_ctx *c, int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *edge_err,
                          const float *qubit_err, int32_t score_form, dm_graph *out) {
  if (!c || !out || n < 1) return DM_E_INVAL;
  if (score_form != DM_SCORE_ERROR_SUM && score_form != DM_SCORE_LOG_FIDELITY) return DM_E_INVAL;
  cudaSetDevice(c->device);
  HostCSR h;
  RET(validate_csr(n, row_ptr, col_idx, edge_err, &h));
  bool nonneg = true;  // weights must be finite; negative ones are kept but switch off pruning
  for (float e : h.ee) {
    if (!std::isfinite(e)) return DM_E_INVAL;
    nonneg &= e >= 0.f;
  }
  if (qubit_err)
    for (int32_t v = 0; v < n; v++) {
      if (!std::isfinite(qubit_err[v])) return DM_E_INVAL;
      nonneg &= qubit_err[v] >= 0.f;
    }
  if (score_form == DM_SCORE_LOG_FIDELITY) {  // error rates must leave a positive fidelity
    for (float e : h.ee)
      if (!(e >= 0.f && e < 1.f)) return DM_E_INVAL;
    if (qubit_err)
      for (int32_t v = 0; v < n; v++)
        if (!(qubit_err[v] >= 0.f && qubit_err[v] < 1.f)) return DM_E_INVAL;
  }
  if (!connected(h, n)) return DM_E_DISCONNECTED;
  DevGraph *g = new DevGraph();
  g->V = n;
  g->nnz = (int64_t)h.ci.size();
  int32_t md = 0;
  for (int32_t u = 0; u < n; u++) md = std::max(md, h.rp[u + 1] - h.rp[u]);
  g->max_deg = md;
  g->avg_deg = (double)g->nnz / n;
  g->nonneg_weights = nonneg;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) return DM_E_NOMEM;
    if (bytes && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return DM_E_CUDA;
    return DM_OK;
  };
  int r = up((void **)&g->row_ptr, h.rp.data(), sizeof(int32_t) * (n + 1));
  if (r == DM_OK) r = up((void **)&g->col_idx, h.ci.data(), sizeof(int32_t) * h.ci.size());
  if (r == DM_OK && edge_err) r = up((void **)&g->eerr, h.ee.data(), sizeof(float) * h.ee.size());
  if (r == DM_OK && qubit_err) r = up((void **)&g->qerr, qubit_err, sizeof(float) * n);
  if (r == DM_OK && score_form == DM_SCORE_LOG_FIDELITY) {  // weights -log(1 - e): scores add up
    if (g->eerr && dmk::launch_neg_log1m(g->eerr, (int64_t)h.ee.size(), c->stream) != cudaSuccess) r = DM_E_CUDA;
    if (g->qerr && dmk::launch_neg_log1m(g->qerr, n, c->stream) != cudaSuccess) r = DM_E_CUDA;
  }
  if (r == DM_OK && n <= 65536) {
    g->adj_words = (n + 63) / 64;
    size_t bytes = (size_t)n * g->adj_words * 8;
    if (cudaMalloc(&g->adj, bytes) != cudaSuccess) r = DM_E_NOMEM;
    else if (cudaMemsetAsync(g->adj, 0, bytes, c->stream) != cudaSuccess) r = DM_E_CUDA;
    else if (dmk::launch_bitmap(g->row_ptr, g->col_idx, n, g->nnz, g->adj_words, g->adj, c->stream) != cudaSuccess)
      r = DM_E_CUDA;
  }
  if (r == DM_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) r = DM_E_CUDA;
  if (r == DM_OK) r = ensure_motif(c, g, 2);
  if (r != DM_OK) {  // a graph that failed to load is neither registered nor kept
    cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    free_graph(c, g);
    return r;
  }
  c->graphs.push_back(g);
  *out = (dm_graph)(c->graphs.size() - 1);
  return DM_OK;
}

int dm_motif_table(dm_ctx *c, dm_graph gh, int32_t motif_id, int32_t *out_rows, int64_t cap, int64_t *out_n,
                   int32_t *out_k) {
  DevGraph *g = get_graph(c, gh);
  if (!g) return DM_E_NOTFOUND;
  cudaSetDevice(c->device);
  RET(ensure_motif(c, g, motif_id));
  DevTable &T = g->motifs.at(motif_id);
  if (out_n) *out_n = T.n;
  if (out_k) *out_k = T.w;
  if (out_rows && cap > 0 && T.n > 0) {
    DevTable s;
    s.n = T.n;
    s.w = T.w;
    RET(dalloc_t(c, &s.rows, (size_t)T.n * T.w));
    CK(cudaMemcpyAsync(s.rows, T.rows, sizeof(int32_t) * T.n * T.w, cudaMemcpyDeviceToDevice, c->stream));
    RET(sort_canonical(c, s, graph_bits(g)));
    int64_t m = std::min(cap, s.n);
    CK(cudaMemcpyAsync(out_rows, s.rows, sizeof(int32_t) * m * s.w, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    free_table(c, s);
  }
  return DM_OK;
}

}  // extern "C"

namespace {

// Validate the pattern, fill the plan's fields and motif set (preset by the data graph's degree
// unless given), and make sure the motif tables exist.
int plan_setup(dm_ctx *c, dm_graph gh, int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx,
               const dm_plan_opts *opts, Plan &p, DevGraph **gout, GraphStats &gs) {
  if (!c) return DM_E_INVAL;
  DevGraph *g = get_graph(c, gh);
  if (!g) return DM_E_NOTFOUND;
  if (n_p < 1 || n_p > MAXW) return DM_E_INVAL;
  if (opts && (opts->induced < 0 || opts->induced > 1)) return DM_E_INVAL;
  cudaSetDevice(c->device);
  HostCSR h;
  RET(validate_csr(n_p, p_row_ptr, p_col_idx, nullptr, &h));
  if (!connected(h, n_p)) return DM_E_DISCONNECTED;
  p.n_p = n_p;
  p.rp = h.rp;
  p.ci = h.ci;
  p.graph = gh;
  p.order = opts ? opts->order : DM_ORDER_PAPER;
  p.join_algo = opts ? opts->join_algo : DM_JOIN_AUTO;
  p.induced = opts ? opts->induced : 0;
  p.chunk_rows = opts ? opts->chunk_rows : 0;
  p.max_rows = opts ? opts->max_rows : 0;
  if (opts && opts->motifs && opts->n_motifs > 0) {
    p.motifs.assign(opts->motifs, opts->motifs + opts->n_motifs);
  } else if (g->max_deg <= 3) {
    p.motifs = {4, 2};  // heavy-hex preset of Sec. 5.1: {M2, M4}
  } else if (g->max_deg == 4) {
    p.motifs = {DM_MOTIF_CYCLE(4), DM_MOTIF_CYCLE(6), 2};  // square-grid preset: {M2, M4-O, M6-O}
  } else {
    p.motifs = {3, 2};
  }
  gs.V = g->V;
  gs.nnz = g->nnz;
  gs.avg_deg = g->avg_deg;
  gs.max_deg = g->max_deg;
  for (int id : p.motifs) {
    MotifDef md;
    if (!motif_def(id, &md) || md.k < 2 || md.k > MAXM) return DM_E_NOTFOUND;
    RET(ensure_motif(c, g, id));
    gs.motifs.push_back({id, g->motifs.at(id).n});
  }
  if (n_p == 1) RET(ensure_motif(c, g, MOTIF_VERTEX));
  *gout = g;
  return DM_OK;
}

// A decomposed plan is runnable once its step count fits and every step's index exists.
int plan_finish(dm_ctx *c, DevGraph *g, const Plan &p) {
  if (p.steps.empty()) return DM_E_INVAL;
  if ((int)p.steps.size() > DM_MAX_STEPS) return DM_E_CAPACITY;
  for (size_t j = 1; j < p.steps.size(); j++) {
    Index *ix;
    const StepSpec &s = p.steps[j];
    RET(ensure_index(c, g, s.motif, s.key_mpos[0], s.n_keys >= 2 ? s.key_mpos[1] : -1,
                     p.join_algo == DM_JOIN_SORTMERGE, &ix));
  }
  return DM_OK;
}

}  // namespace

extern "C" {

int dm_plan(dm_ctx *c, dm_graph gh, int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx,
            const dm_plan_opts *opts, dm_plan_t **out) {
  if (!c || !out) return DM_E_INVAL;
  std::unique_ptr<dm_plan_t> pl(new dm_plan_t());
  Plan &p = pl->p;
  DevGraph *g = nullptr;
  GraphStats gs;
  RET(plan_setup(c, gh, n_p, p_row_ptr, p_col_idx, opts, p, &g, gs));
  const bool learned = p.order == DM_ORDER_LEARNED && c->m_trained;
  if (!learned) {
    RET(decompose(p, p.motifs, p.order == DM_ORDER_LEARNED ? DM_ORDER_HEURISTIC : p.order, gs, &p.steps,
                  p.col_vertex));
    RET(plan_cost(c, p.steps, false, &p.pred_cost, &p.pred_max_rows, &p.pred_growth));
  } else {
    // The trained model picks the plan among the candidate decompositions, costed with the
    // model's per-step cardinalities.
    std::vector<CandidatePlan> cands;
    RET(candidate_plans(c, g, p, opts && opts->motifs && opts->n_motifs > 0, gs, &cands));
    std::vector<const std::vector<StepSpec> *> steps;
    for (auto &cp : cands) steps.push_back(&cp.steps);
    std::vector<double> cost, maxr;
    std::vector<std::vector<float>> growths;
    RET(plan_costs(c, steps, &cost, &maxr, &growths));  // one model evaluation for every candidate
    double best = 1e308;
    for (size_t i = 0; i < cands.size(); i++) {
      if (cost[i] < best) {
        best = cost[i];
        p.steps = cands[i].steps;
        memcpy(p.col_vertex, cands[i].col_vertex, sizeof(cands[i].col_vertex));
        p.pred_cost = cost[i];
        p.pred_max_rows = maxr[i];
        p.pred_growth = growths[i];
        p.motifs = cands[i].motifs;
      }
    }
  }
  RET(plan_finish(c, g, p));
  *out = pl.release();
  return DM_OK;
}

int dm_plan_batch(dm_ctx *c, dm_graph gh, int32_t n_patterns, const int32_t *n_p, const int32_t *const *p_row_ptr,
                  const int32_t *const *p_col_idx, const dm_plan_opts *opts, dm_plan_t **out) {
  if (!c || !out || n_patterns < 0 || (n_patterns > 0 && (!n_p || !p_row_ptr || !p_col_idx))) return DM_E_INVAL;
  for (int32_t i = 0; i < n_patterns; i++) out[i] = nullptr;
  const int order = opts ? opts->order : DM_ORDER_PAPER;
  const bool learned = order == DM_ORDER_LEARNED && c->m_trained;
  const bool user_motifs = opts && opts->motifs && opts->n_motifs > 0;
  std::vector<std::unique_ptr<dm_plan_t>> pl(n_patterns);
  std::vector<GraphStats> gs(n_patterns);
  std::vector<std::vector<std::vector<int32_t>>> sets(n_patterns);
  DevGraph *g = nullptr;
  // the calling thread: checks, motif tables (device work)
  for (int32_t i = 0; i < n_patterns; i++) {
    pl[i].reset(new dm_plan_t());
    RET(plan_setup(c, gh, n_p[i], p_row_ptr[i], p_col_idx[i], opts, pl[i]->p, &g, gs[i]));
    if (learned) RET(candidate_sets(c, g, pl[i]->p, user_motifs, gs[i], &sets[i]));
  }
  // host threads: the decompositions
  std::vector<std::vector<CandidatePlan>> cands(n_patterns);
  std::vector<int> rc(n_patterns, DM_OK);
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    for (int32_t i; (i = next.fetch_add(1)) < n_patterns;) {
      Plan &p = pl[i]->p;
      if (learned) {
        decompose_candidates(p, sets[i], gs[i], &cands[i]);
        if (cands[i].empty()) rc[i] = DM_E_INVAL;
      } else {
        rc[i] = decompose(p, p.motifs, p.order == DM_ORDER_LEARNED ? DM_ORDER_HEURISTIC : p.order, gs[i], &p.steps,
                          p.col_vertex);
      }
    }
  };
  const int nt = (int)std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
  std::vector<std::thread> th;
  for (int t = 1; t < nt && t < n_patterns; t++) th.emplace_back(work);
  work();
  for (auto &t : th) t.join();
  for (int32_t i = 0; i < n_patterns; i++) RET(rc[i]);
  // costs: one model evaluation for every candidate of every pattern, or the heuristic chain
  if (learned) {
    std::vector<const std::vector<StepSpec> *> steps;
    for (auto &cv : cands)
      for (auto &cp : cv) steps.push_back(&cp.steps);
    std::vector<double> cost, maxr;
    std::vector<std::vector<float>> growths;
    RET(plan_costs(c, steps, &cost, &maxr, &growths));
    size_t k = 0;
    for (int32_t i = 0; i < n_patterns; i++) {
      Plan &p = pl[i]->p;
      double best = 1e308;
      for (auto &cp : cands[i]) {
        if (cost[k] < best) {
          best = cost[k];
          p.steps = cp.steps;
          memcpy(p.col_vertex, cp.col_vertex, sizeof(cp.col_vertex));
          p.pred_cost = cost[k];
          p.pred_max_rows = maxr[k];
          p.pred_growth = growths[k];
          p.motifs = cp.motifs;
        }
        k++;
      }
    }
  } else {
    for (int32_t i = 0; i < n_patterns; i++) {
      Plan &p = pl[i]->p;
      RET(plan_cost(c, p.steps, false, &p.pred_cost, &p.pred_max_rows, &p.pred_growth));
    }
  }
  for (int32_t i = 0; i < n_patterns; i++) RET(plan_finish(c, g, pl[i]->p));
  for (int32_t i = 0; i < n_patterns; i++) out[i] = pl[i].release();
  return DM_OK;
}

int32_t dm_plan_candidates(dm_ctx *c, dm_graph gh, int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx,
                           const dm_plan_opts *opts, dm_plan_t **out, int32_t max_out) {
  if (!c || max_out < 0 || (max_out > 0 && !out)) return DM_E_INVAL;
  Plan base;
  DevGraph *g = nullptr;
  GraphStats gs;
  RET(plan_setup(c, gh, n_p, p_row_ptr, p_col_idx, opts, base, &g, gs));
  std::vector<CandidatePlan> cands;
  RET(candidate_plans(c, g, base, opts && opts->motifs && opts->n_motifs > 0, gs, &cands));
  const int32_t n = (int32_t)cands.size();
  for (int32_t i = 0; i < n && i < max_out; i++) {
    std::unique_ptr<dm_plan_t> pl(new dm_plan_t());
    Plan &p = pl->p;
    p = base;
    p.order = cands[i].order;
    p.motifs = cands[i].motifs;
    p.steps = cands[i].steps;
    memcpy(p.col_vertex, cands[i].col_vertex, sizeof(p.col_vertex));
    int r = plan_cost(c, p.steps, false, &p.pred_cost, &p.pred_max_rows, &p.pred_growth);
    if (r == DM_OK) r = plan_finish(c, g, p);
    if (r != DM_OK) {
      for (int32_t j = 0; j < i; j++) {
        delete out[j];
        out[j] = nullptr;
      }
      return r;
    }
    out[i] = pl.release();
  }
  return n;
}

void dm_plan_free(dm_plan_t *p) { delete p; }

static int32_t describe_steps(const std::vector<StepSpec> &steps, int32_t *buf, int32_t buf_len) {
  std::vector<int32_t> v;
  v.push_back((int32_t)steps.size());
  for (auto &s : steps) {
    v.push_back(s.motif);
    v.push_back(s.k);
    for (int i = 0; i < s.k; i++) v.push_back(s.slice[i]);
    v.push_back(s.n_keys);
    v.push_back(s.n_be);
    for (int i = 0; i < s.n_be; i++) {
      v.push_back(s.be_vtx[i][0]);
      v.push_back(s.be_vtx[i][1]);
    }
  }
  if (buf)
    for (int32_t i = 0; i < buf_len && i < (int32_t)v.size(); i++) buf[i] = v[i];
  return (int32_t)v.size();
}

int32_t dm_plan_describe(const dm_plan_t *pl, int32_t *buf, int32_t buf_len) {
  if (!pl) return DM_E_INVAL;
  return describe_steps(pl->p.steps, buf, buf_len);
}

int32_t dm_decompose(int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx, const int32_t *motifs,
                     int32_t n_motifs, int32_t order, int32_t *buf, int32_t buf_len) {
  if (n_p < 1 || n_p > MAXW || (n_motifs > 0 && !motifs) || n_motifs < 0) return DM_E_INVAL;
  HostCSR h;
  RET(validate_csr(n_p, p_row_ptr, p_col_idx, nullptr, &h));
  if (!connected(h, n_p)) return DM_E_DISCONNECTED;
  Plan p;
  p.n_p = n_p;
  p.rp = h.rp;
  p.ci = h.ci;
  std::vector<int32_t> set(motifs, motifs + n_motifs);
  GraphStats gs;
  gs.V = 1;
  gs.avg_deg = 1;
  gs.max_deg = 1;
  for (int id : set) gs.motifs.push_back({id, 1});
  RET(decompose(p, set, order, gs, &p.steps, p.col_vertex));
  return describe_steps(p.steps, buf, buf_len);
}

int dm_match(dm_ctx *c, const dm_plan_t *pl, int mode, dm_chunk_cb cb, void *user, uint64_t *out_count,
             uint64_t *out_checksum) {
  if (!c || !pl) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  int base_mode = mode & 0xF;
  if (base_mode != DM_ALL && base_mode != DM_COUNT) return DM_E_INVAL;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &pl->p;
  ex.mode = base_mode;
  ex.use_qerr = true;
  ex.chunk_rows = pl->p.chunk_rows;
  ex.max_rows = pl->p.max_rows;
  c->inflight = 0;
  AllSink sink;
  sink.flags = mode;
  sink.cb = cb;
  sink.user = user;
  sink.bits = graph_bits(g);
  ex.sink = &sink;
  int r = ex.run();
  uint64_t cnt = ex.count, cs = ex.checksum;
  if (r == DM_OK && base_mode == DM_ALL) {
    r = sink.finish(c, pl->p.n_p, g->eerr != nullptr);
    cnt = sink.count;
    cs = sink.checksum;
  }
  for (auto &h : sink.held) free_table(c, h);
  cudaStreamSynchronize(c->stream);
  finish_stats(c, t0);
  if (r != DM_OK) return r;
  log_plan_steps(c, pl->p);
  if (out_count) *out_count = cnt;
  if (out_checksum) *out_checksum = cs;
  return DM_OK;
}

int dm_match_shard(dm_ctx *c, const dm_plan_t *pl, int32_t shard, int32_t n_shards, uint64_t *out_count,
                   uint64_t *out_checksum) {
  if (!c || !pl || n_shards < 1 || shard < 0 || shard >= n_shards) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &pl->p;
  ex.mode = DM_COUNT;
  ex.use_qerr = false;
  ex.shard = shard;
  ex.n_shards = n_shards;
  ex.chunk_rows = pl->p.chunk_rows;
  ex.max_rows = pl->p.max_rows;
  c->inflight = 0;
  const int r = ex.run();
  cudaStreamSynchronize(c->stream);
  finish_stats(c, t0);
  if (r != DM_OK) return r;
  if (out_count) *out_count = ex.count;
  if (out_checksum) *out_checksum = ex.checksum;
  return DM_OK;
}

int dm_match_batch(dm_ctx *c, const dm_plan_t *const *plans, int32_t n_plans, int mode, uint64_t *out_counts,
                   uint64_t *out_checksums) {
  if (!c || (!plans && n_plans > 0) || n_plans < 0 || (mode & 0xF) != DM_COUNT) return DM_E_INVAL;
  if (n_plans == 0) return DM_OK;
  DevGraph *g = get_graph(c, plans[0] ? plans[0]->p.graph : -1);
  if (!g) return DM_E_NOTFOUND;
  for (int32_t i = 0; i < n_plans; i++)
    if (!plans[i] || plans[i]->p.graph != plans[0]->p.graph) return DM_E_INVAL;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  BatchState *b = c->batch;
  bool same = b && b->hash_lf == c->hash_lf && (int32_t)b->key.size() == n_plans &&
              std::equal(b->key.begin(), b->key.end(), plans);
  if (!same) {
    batch_release(c, b);
    c->batch = nullptr;
    int TR = 64;
    int64_t chunk = 16;
    double heavy = c->heavy_rows;
    int threads = c->batch_threads, ctas = c->batch_ctas;
    if (c->autotune) {  // time the candidate configurations on this batch, keep the fastest
      auto trial = [&](int tr, int64_t ch, double hv, int th, int cps, double *ms) {
        BatchState *t = nullptr;
        int r = batch_build(c, g, plans, n_plans, tr, ch, hv, th, cps, &t);
        if (r == DM_OK) {
          auto s0 = std::chrono::steady_clock::now();
          r = batch_run(c, g, t);
          *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s0).count();
        }
        batch_release(c, t);
        return r;
      };
      // coordinate search: tile rows x root chunk, then the split between the persistent
      // launch and step-by-step execution, then the block shape (and the root chunk again when
      // the shape changed), then the hash load factor
      double best = 1e300, ms = 0;
      for (int tr : {32, 64, 128})
        for (int64_t ch : {4, 16, 64})
          if (trial(tr, ch, heavy, threads, ctas, &ms) == DM_OK && ms < best) {
            best = ms;
            TR = tr;
            chunk = ch;
          }
      for (double hv : {1e300, 1048576.0, 262144.0, 65536.0, 16384.0})
        if (trial(TR, chunk, hv, threads, ctas, &ms) == DM_OK && ms < best) {
          best = ms;
          heavy = hv;
        }
      const int shapes[5][2] = {{256, 1}, {128, 0}, {128, 2}, {256, 0}, {32, 0}};  // 32: warp walks
      int TR_shape = TR;
      const int threads0 = threads, ctas0 = ctas;
      for (auto &sh : shapes)
        if (trial(TR, chunk, heavy, sh[0], sh[1], &ms) == DM_OK && ms < best) {
          best = ms;
          threads = sh[0];
          ctas = sh[1];
          TR_shape = sh[0] == 32 ? 32 : TR;  // warp walks always take 32-row tiles
        }
      TR = TR_shape;
      if (threads != threads0 || ctas != ctas0)  // the root chunk again, for the shape chosen
        for (int64_t ch : {4, 16, 64})
          if (ch != chunk && trial(TR, ch, heavy, threads, ctas, &ms) == DM_OK && ms < best) {
            best = ms;
            chunk = ch;
          }
      const double lf0 = c->hash_lf;
      double lf_best = lf0;
      for (double lf : {0.25, 0.5, 0.75}) {
        if (lf == lf0) continue;
        set_hash_load_factor(c, lf);
        if (trial(TR, chunk, heavy, threads, ctas, &ms) == DM_OK && ms < best) {
          best = ms;
          lf_best = lf;
        }
      }
      set_hash_load_factor(c, lf_best);
    }
    RET(batch_build(c, g, plans, n_plans, TR, chunk, heavy, threads, ctas, &b));
    b->tuned = c->autotune != 0;
    c->batch = b;
  }
  RET(batch_run(c, g, b));
  for (int32_t i = 0; i < n_plans; i++) {
    if (out_counts) out_counts[i] = b->h_out[2 + 2 * i];
    if (out_checksums) out_checksums[i] = b->h_out[3 + 2 * i];
  }
  finish_stats(c, t0);
  return DM_OK;
}

int dm_batch_config(dm_ctx *c, int32_t *tile_rows, int64_t *root_chunk, int32_t *grid, int32_t *n_stepwise,
                    double *heavy_rows, int32_t *threads_per_cta, int32_t *ctas_per_sm, double *hash_load_factor) {
  if (!c || !c->batch) return DM_E_INVAL;
  if (threads_per_cta) *threads_per_cta = c->batch->threads;
  if (ctas_per_sm) *ctas_per_sm = c->batch->grid / std::max(1, c->num_sms);
  if (hash_load_factor) *hash_load_factor = c->batch->hash_lf;
  if (tile_rows) *tile_rows = c->batch->TR;
  if (root_chunk) *root_chunk = c->batch->root_chunk;
  if (grid) *grid = c->batch->grid;
  if (n_stepwise) *n_stepwise = (int32_t)c->batch->heavy.size();
  if (heavy_rows) *heavy_rows = c->batch->heavy_rows;
  return DM_OK;
}

int dm_batch_latency(dm_ctx *c, double *out_ms, int32_t n) {
  if (!c || !out_ms || n != (int32_t)c->batch_latency.size()) return DM_E_INVAL;
  for (int32_t i = 0; i < n; i++) out_ms[i] = c->batch_latency[i];
  return DM_OK;
}

int dm_set_batch_shape(dm_ctx *c, int32_t threads_per_cta, int32_t ctas_per_sm) {
  if (!c || (threads_per_cta != 32 && threads_per_cta != 128 && threads_per_cta != 256) || ctas_per_sm < 0)
    return DM_E_INVAL;
  if (c->batch_threads == threads_per_cta && c->batch_ctas == ctas_per_sm) return DM_OK;
  c->batch_threads = threads_per_cta;
  c->batch_ctas = ctas_per_sm;
  if (c->batch) {
    batch_release(c, c->batch);
    c->batch = nullptr;
  }
  return DM_OK;
}

int dm_set_fusion(dm_ctx *c, int on) {
  if (!c) return DM_E_INVAL;
  c->fuse_last = on != 0;
  return DM_OK;
}

int dm_set_tuning(dm_ctx *c, int autotune, double hash_load_factor, double heavy_rows) {
  if (!c || hash_load_factor <= 0.0 || hash_load_factor > 0.95) return DM_E_INVAL;
  c->autotune = autotune;
  c->heavy_rows = heavy_rows > 0 ? heavy_rows : 1e300;
  if (c->batch) {  // the next batch is rebuilt under the new settings
    batch_release(c, c->batch);
    c->batch = nullptr;
  }
  set_hash_load_factor(c, hash_load_factor);
  return DM_OK;
}

int dm_score_topk(dm_ctx *c, const dm_plan_t *pl, int32_t k, int32_t *out_rows, float *out_scores, int32_t *out_n) {
  if (!c || !pl || k < 1 || !out_rows || !out_n) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  if (!g->eerr) return DM_E_INVAL;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &pl->p;
  ex.mode = DM_ALL;
  ex.use_qerr = true;
  ex.chunk_rows = pl->p.chunk_rows;
  ex.max_rows = pl->p.max_rows;
  c->inflight = 0;
  TopkSink sink;
  sink.g = g;
  sink.k = k;
  // bound pruning is exact only when no weight is negative (a partial score is then a lower
  // bound of every completion's score)
  sink.prune_ptr = g->nonneg_weights ? &ex.prune : nullptr;
  ex.sink = &sink;
  int r = ex.run();
  if (r == DM_OK) {
    int64_t m = sink.have ? sink.best.n : 0;
    if (m > 0) {
      CK(cudaMemcpyAsync(out_rows, sink.best.rows, sizeof(int32_t) * m * sink.best.w, cudaMemcpyDeviceToHost, c->stream));
      if (out_scores)
        CK(cudaMemcpyAsync(out_scores, sink.best.score, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    *out_n = (int32_t)m;
  }
  if (sink.have) free_table(c, sink.best);
  cudaStreamSynchronize(c->stream);
  finish_stats(c, t0);
  return r;
}

int dm_load_directed_errors(dm_ctx *c, dm_graph gh, const float *e_dir) {
  DevGraph *g = get_graph(c, gh);
  if (!g || !e_dir) return g ? DM_E_INVAL : DM_E_NOTFOUND;
  for (int64_t i = 0; i < g->nnz; i++)
    if (!std::isfinite(e_dir[i])) return DM_E_INVAL;
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream));  // no queued work still reads the previous array
  float *d = nullptr;
  if (cudaMalloc(&d, sizeof(float) * std::max<int64_t>(1, g->nnz)) != cudaSuccess) {
    cudaGetLastError();
    return DM_E_NOMEM;
  }
  if (cudaMemcpy(d, e_dir, sizeof(float) * g->nnz, cudaMemcpyHostToDevice) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    cudaFree(d);
    return cuda_fail(c, e, "directed errors upload");
  }
  cudaFree(g->edir);
  g->edir = d;
  return DM_OK;
}

int dm_score_topk_directed(dm_ctx *c, const dm_plan_t *pl, const float *w_dir, int32_t k, int32_t *out_rows,
                           float *out_scores, int32_t *out_n) {
  if (!c || !pl || !w_dir || k < 1 || !out_rows || !out_n) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  if (!g->edir) return DM_E_INVAL;
  const Plan &P = pl->p;
  std::vector<int32_t> hp, hq;  // the pattern's weighted slots p -> q
  std::vector<float> hw;
  for (int32_t u = 0; u < P.n_p; u++)
    for (int32_t e = P.rp[u]; e < P.rp[u + 1]; e++) {
      if (!std::isfinite(w_dir[e])) return DM_E_INVAL;
      if (w_dir[e] != 0.f) {
        hp.push_back(u);
        hq.push_back(P.ci[e]);
        hw.push_back(w_dir[e]);
      }
    }
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  const size_t ns = hw.size();
  int32_t *dp = nullptr, *dq = nullptr;
  float *dw = nullptr;
  int r = dalloc_t(c, &dp, std::max<size_t>(1, ns));
  if (r == DM_OK) r = dalloc_t(c, &dq, std::max<size_t>(1, ns));
  if (r == DM_OK) r = dalloc_t(c, &dw, std::max<size_t>(1, ns));
  if (r == DM_OK && ns) {
    if (cudaMemcpyAsync(dp, hp.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(dq, hq.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(dw, hw.data(), sizeof(float) * ns, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      r = cuda_fail(c, cudaGetLastError(), "directed slots upload");
  }
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &P;
  ex.mode = DM_ALL;
  ex.use_qerr = false;
  ex.chunk_rows = P.chunk_rows;
  ex.max_rows = P.max_rows;
  c->inflight = 0;
  TopkSink tk;  // no bound pruning: partial undirected scores bound nothing here
  tk.g = g;
  tk.k = k;
  DirectedSink ds;
  ds.g = g;
  ds.tk = &tk;
  ds.np = P.n_p;
  ds.nslots = (int32_t)ns;
  ds.sp = dp;
  ds.sq = dq;
  ds.sw = dw;
  ex.sink = &ds;
  if (r == DM_OK) r = ex.run();
  if (r == DM_OK) {
    const int64_t m = tk.have ? tk.best.n : 0;
    if (m > 0) {
      CK(cudaMemcpyAsync(out_rows, tk.best.rows, sizeof(int32_t) * m * tk.best.w, cudaMemcpyDeviceToHost, c->stream));
      if (out_scores)
        CK(cudaMemcpyAsync(out_scores, tk.best.score, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    *out_n = (int32_t)m;
  }
  if (tk.have) free_table(c, tk.best);
  dfree(c, dp);
  dfree(c, dq);
  dfree(c, dw);
  cudaStreamSynchronize(c->stream);
  finish_stats(c, t0);
  return r;
}

int dm_match_topk(dm_ctx *c, const dm_plan_t *pl, int mode, dm_chunk_cb cb, void *user, int32_t k, int32_t *out_rows,
                  float *out_scores, int32_t *out_n, uint64_t *out_count, uint64_t *out_checksum) {
  if (!c || !pl || k < 1 || !out_rows || !out_n || (mode & 0xF) != DM_ALL) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  if (!g->eerr) return DM_E_INVAL;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &pl->p;
  ex.mode = DM_ALL;
  ex.use_qerr = true;
  ex.chunk_rows = pl->p.chunk_rows;
  ex.max_rows = pl->p.max_rows;
  c->inflight = 0;
  TopkSink tk;
  tk.g = g;
  tk.k = k;
  tk.input_sorted = true;
  AllSink sink;
  sink.flags = mode;
  sink.cb = cb;
  sink.user = user;
  sink.bits = graph_bits(g);
  sink.tap = &tk;
  sink.final_rows = out_rows;
  sink.final_scores = out_scores;
  ex.sink = &sink;
  int r = ex.run();
  if (r == DM_OK) r = sink.finish(c, pl->p.n_p, true);
  for (auto &h : sink.held) free_table(c, h);
  if (r == DM_OK && sink.final_done) {  // copied out with the last flush
    *out_n = (int32_t)sink.final_n;
    if (out_count) *out_count = sink.count;
    if (out_checksum) *out_checksum = sink.checksum;
  } else if (r == DM_OK) {
    int64_t m = tk.have ? tk.best.n : 0;
    if (m > 0) {
      CK(cudaMemcpyAsync(out_rows, tk.best.rows, sizeof(int32_t) * m * tk.best.w, cudaMemcpyDeviceToHost, c->stream));
      if (out_scores) CK(cudaMemcpyAsync(out_scores, tk.best.score, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    *out_n = (int32_t)m;
    if (out_count) *out_count = sink.count;
    if (out_checksum) *out_checksum = sink.checksum;
  }
  if (tk.have) free_table(c, tk.best);
  cudaStreamSynchronize(c->stream);
  finish_stats(c, t0);
  return r;
}

int dm_model_init(dm_ctx *c, uint64_t seed) {
  if (!c) return DM_E_INVAL;
  cudaSetDevice(c->device);
  RET(model_alloc(c));
  const int64_t P = dmk::mlp_param_count();
  std::vector<float> w(P, 0.f);
  uint64_t st = seed;
  auto next = [&]() {  // SplitMix64
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto unif = [&]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; };
  const int H = 128, IN = NFEAT;
  double a1 = sqrt(6.0 / IN), a2 = sqrt(6.0 / H), a3 = sqrt(3.0 / H);  // He-uniform
  size_t o = 0;
  for (int i = 0; i < H * IN; i++) w[o++] = (float)(a1 * unif());
  o += H;
  for (int i = 0; i < H * H; i++) w[o++] = (float)(a2 * unif());
  o += H;
  for (int i = 0; i < H; i++) w[o++] = (float)(a3 * unif());
  CK(cudaMemcpy(c->m_params, w.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
  CK(cudaMemset(c->m_m, 0, sizeof(float) * P));
  CK(cudaMemset(c->m_v, 0, sizeof(float) * P));
  c->m_step = 0;
  c->m_trained = false;
  for (int k = 0; k < NFEAT; k++) {
    c->m_mean[k] = 0.f;
    c->m_std[k] = 1.f;
  }
  return DM_OK;
}

int dm_model_weights(dm_ctx *c, float *out, int64_t *n_floats) {
  if (!c) return DM_E_INVAL;
  const int64_t P = dmk::mlp_param_count();
  if (n_floats) *n_floats = P + 2 * NFEAT;
  if (!out) return DM_OK;
  if (!c->m_params) return DM_E_INVAL;
  CK(cudaMemcpy(out, c->m_params, sizeof(float) * P, cudaMemcpyDeviceToHost));
  memcpy(out + P, c->m_mean, sizeof(float) * NFEAT);
  memcpy(out + P + NFEAT, c->m_std, sizeof(float) * NFEAT);
  return DM_OK;
}

int dm_model_set_weights(dm_ctx *c, const float *w, int64_t n) {
  const int64_t P = dmk::mlp_param_count();
  if (!c || !w || n != P + 2 * NFEAT) return DM_E_INVAL;
  cudaSetDevice(c->device);
  RET(model_alloc(c));
  CK(cudaMemcpy(c->m_params, w, sizeof(float) * P, cudaMemcpyHostToDevice));
  for (int k = 0; k < NFEAT; k++) {
    c->m_mean[k] = w[P + k];
    c->m_std[k] = w[P + NFEAT + k] > 0.f ? w[P + NFEAT + k] : 1.f;
  }
  c->m_trained = true;
  return DM_OK;
}

int dm_model_grad(dm_ctx *c, const float *feats, const float *targets, int32_t n, float *out_pred,
                  float *out_grads, float *out_loss) {
  if (!c || !feats || n < 1 || !c->m_params) return DM_E_INVAL;
  cudaSetDevice(c->device);
  const int64_t P = dmk::mlp_param_count();
  if (targets) CK(cudaMemset(c->m_grads, 0, sizeof(float) * P));
  RET(model_run(c, feats, targets, n, out_pred, targets ? c->m_grads : nullptr, out_loss));
  if (targets && out_grads) CK(cudaMemcpy(out_grads, c->m_grads, sizeof(float) * P, cudaMemcpyDeviceToHost));
  return DM_OK;
}

int dm_model_train(dm_ctx *c, const float *feats, const float *targets, int32_t n, int32_t epochs, int32_t batch,
                   float lr, uint64_t seed, float *out_loss) {
  if (!c || !feats || !targets || n < 1 || epochs < 1 || batch < 16) return DM_E_INVAL;
  cudaSetDevice(c->device);
  if (!c->m_params) RET(dm_model_init(c, seed));
  if (!c->m_trained) {  // standardise each input feature over the training set
    for (int k = 0; k < NFEAT; k++) {
      double s = 0, s2 = 0;
      for (int32_t i = 0; i < n; i++) {
        double v = feats[(size_t)i * NFEAT + k];
        s += v;
        s2 += v * v;
      }
      double mu = s / n, var = s2 / n - mu * mu;
      c->m_mean[k] = (float)mu;
      c->m_std[k] = var > 1e-12 ? (float)sqrt(var) : 1.f;
    }
  }
  std::vector<float> xn;
  normalise(c, feats, n, xn);
  const int64_t P = dmk::mlp_param_count();
  std::vector<int32_t> idx(n);
  for (int32_t i = 0; i < n; i++) idx[i] = i;
  uint64_t st = seed ^ 0xA5A5A5A5ull;
  std::vector<float> bx, bt;
  for (int32_t ep = 0; ep < epochs; ep++) {
    for (int32_t i = n - 1; i > 0; i--) {  // Fisher-Yates with SplitMix64
      st += 0x9E3779B97F4A7C15ull;
      uint64_t z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      std::swap(idx[i], idx[(int32_t)(z % (uint64_t)(i + 1))]);
    }
    double ep_loss = 0;
    for (int32_t b0 = 0; b0 < n; b0 += batch) {
      int32_t m = std::min(batch, n - b0);
      bx.resize((size_t)m * NFEAT);
      bt.resize(m);
      for (int32_t i = 0; i < m; i++) {
        memcpy(&bx[(size_t)i * NFEAT], &xn[(size_t)idx[b0 + i] * NFEAT], sizeof(float) * NFEAT);
        bt[i] = targets[idx[b0 + i]];
      }
      float loss = 0;
      CK(cudaMemsetAsync(c->m_grads, 0, sizeof(float) * P, c->stream));
      RET(model_run(c, bx.data(), bt.data(), m, nullptr, c->m_grads, &loss));
      c->m_step++;
      CK(dmk::mlp_adam(c->m_params, c->m_grads, c->m_m, c->m_v, P, lr, c->m_step, c->stream));
      ep_loss += (double)loss * m;
    }
    if (out_loss) out_loss[ep] = (float)(ep_loss / n);
  }
  CK(cudaStreamSynchronize(c->stream));
  c->m_trained = true;
  return DM_OK;
}

int dm_model_predict(dm_ctx *c, const float *feats, int32_t n, float *out) {
  if (!c || !feats || !out || n < 1 || !c->m_params) return DM_E_INVAL;
  cudaSetDevice(c->device);
  std::vector<float> xn;
  normalise(c, feats, n, xn);
  return model_run(c, xn.data(), nullptr, n, out, nullptr, nullptr);
}

int dm_step_log(dm_ctx *c, float *feats, float *targets, int64_t cap, int64_t *out_n, int clear) {
  if (!c) return DM_E_INVAL;
  int64_t n = (int64_t)c->log_target.size();
  if (out_n) *out_n = n;
  int64_t m = std::min(n, cap);
  if (feats && m > 0) memcpy(feats, c->log_feat.data(), sizeof(float) * m * NFEAT);
  if (targets && m > 0) memcpy(targets, c->log_target.data(), sizeof(float) * m);
  if (clear) {
    c->log_feat.clear();
    c->log_target.clear();
  }
  return DM_OK;
}

int dm_plan_cost(const dm_plan_t *pl, double *cost, double *max_rows) {
  if (!pl) return DM_E_INVAL;
  if (cost) *cost = pl->p.pred_cost;
  if (max_rows) *max_rows = pl->p.pred_max_rows;
  return DM_OK;
}

int32_t dm_plan_predicted_rows(const dm_plan_t *pl, double *rows, int32_t cap) {
  if (!pl || cap < 0 || (cap > 0 && !rows)) return DM_E_INVAL;
  const int32_t n = (int32_t)pl->p.pred_growth.size();
  double lr = 0;
  for (int32_t j = 0; j < n && j < cap; j++) {
    lr += pl->p.pred_growth[j];
    rows[j] = exp(std::min(60.0, std::max(-60.0, lr)));
  }
  return n;
}

int dm_plan_estimates(const dm_plan_t *pl, float *feats, float *heur_growth, int32_t cap) {
  if (!pl) return DM_E_INVAL;
  int32_t n = (int32_t)pl->p.steps.size();
  for (int32_t j = 0; j < n && j < cap; j++) {
    float x[NFEAT];
    model_input(pl->p.steps[j].feat, x);
    if (feats) memcpy(feats + (size_t)j * NFEAT, x, sizeof(x));
    if (heur_growth) heur_growth[j] = x[22];
  }
  return n;
}

int dm_images(dm_ctx *c, const dm_plan_t *pl, int32_t *out_sets, int64_t cap, int64_t *out_n) {
  if (!c || !pl) return DM_E_INVAL;
  DevGraph *g = get_graph(c, pl->p.graph);
  if (!g) return DM_E_NOTFOUND;
  cudaSetDevice(c->device);
  auto t0 = std::chrono::steady_clock::now();
  reset_stats(c);
  Exec ex;
  ex.c = c;
  ex.g = g;
  ex.p = &pl->p;
  ex.mode = DM_ALL;
  ex.use_qerr = false;
  ex.chunk_rows = pl->p.chunk_rows;
  ex.max_rows = pl->p.max_rows;
  c->inflight = 0;
  CollectSink sink;
  ex.sink = &sink;
  RET(ex.run());
  DevTable t;
  RET(sink.concat(c, pl->p.n_p, false, &t));
  const int64_t n = t.n;
  const int32_t w = t.w;
  int64_t m = 0;
  if (n > 0) {
    CK(dmk::images_prepare(t.rows, n, w, c->stream));
    RET(sort_canonical(c, t, graph_bits(g)));
    int32_t *flag = nullptr, *uniq = nullptr;
    int64_t *pos = nullptr, *tmp = nullptr;
    RET(dalloc_t(c, &flag, n));
    RET(dalloc_t(c, &pos, n + 1));
    RET(dalloc_t(c, &tmp, dmk::scan_tmp_elems(n)));
    RET(dalloc_t(c, &uniq, (size_t)n * w));
    CK(dmk::unique_rows(t.rows, n, w, flag, pos, tmp, uniq, c->stream));
    CK(cudaMemcpyAsync(&m, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (out_sets && cap > 0 && m > 0)
      CK(cudaMemcpyAsync(out_sets, uniq, sizeof(int32_t) * std::min(cap, m) * w, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, flag);
    dfree(c, pos);
    dfree(c, tmp);
    dfree(c, uniq);
  }
  free_table(c, t);
  if (out_n) *out_n = m;
  finish_stats(c, t0);
  return DM_OK;
}

int dm_get_stats(dm_ctx *c, dm_stats *out) {
  if (!c || !out) return DM_E_INVAL;
  *out = c->stats;
  return DM_OK;
}

int dm_enable_timing(dm_ctx *c, int on) {
  if (!c) return DM_E_INVAL;
  c->timing = on != 0;
  return DM_OK;
}

}  // extern "C"
