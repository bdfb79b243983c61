// Internal types of the Delta-Motif GB300 library: plan steps (host) and the POD argument
// blocks the kernels receive by value. Nothing here is part of the C ABI.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace dmi {

constexpr int MAXW = 128;  // pattern vertices = maximum row width of an intermediate table
constexpr int MAXM = 24;   // motif vertices
constexpr int MAXBE = 64;  // back-edge checks in one step
constexpr int MAXSTEPS = 128;

// Shared-memory row stride (in int32 words) of an R tile of width w: a multiple of 4 so that a
// row can be read as int4 vectors, with an odd number of int4s so that the rows read by the 8
// lanes of one 128-bit shared-memory phase fall on distinct banks. Padding words hold -1,
// which matches no vertex id.
#ifdef __CUDACC__
__host__ __device__
#endif
inline int join_row_stride(int w) {
  int s = (w + 3) / 4 * 4;
  if (s == 0) s = 4;
  if (((s / 4) & 1) == 0) s += 4;
  return s;
}

constexpr int MOTIF_VERTEX = 1;  // the one-vertex "motif" (degenerate single-vertex pattern)

// ------------------------------------------------------------------- motifs (host) -----
struct MotifDef {
  int id = 0;
  int k = 0;
  std::vector<std::pair<int, int>> edges;
  uint32_t adj[MAXM] = {};  // adjacency bitmask per motif position
  int parent[MAXM] = {};    // an earlier neighbour of each position (-1 for position 0)
  std::string name;
};

bool motif_def(int id, MotifDef *out);

// ------------------------------------------------------------------- plans (host) ------
// One join step of Alg. 1: R <- FilterOverlappingNodes(InnerJoin(R, Res(M), C)).
struct StepSpec {
  int32_t motif = 0;
  int32_t k = 0;
  int32_t slice[MAXM] = {};    // motif position -> pattern vertex (the slice S_i)
  int32_t n_keys = 0;          // motif positions whose pattern vertex is already mapped
  int32_t key_mpos[MAXM] = {}; // ... ascending
  int32_t key_col[MAXM] = {};  // ... and the working column holding that vertex
  int32_t n_new = 0;           // new positions (ascending); they become columns w_in + i
  int32_t new_mpos[MAXM] = {};
  int32_t w_in = 0, w_out = 0;
  int32_t n_be = 0;            // uncovered pattern edges closed by this step (back-edges)
  int32_t be_col[MAXBE][2] = {};
  int32_t be_vtx[MAXBE][2] = {};
  // induced matching: per new vertex i, the working columns (< w_in + i) whose pattern vertex
  // is not adjacent to it in the pattern (bit c of word c / 64); their images must not be
  // adjacent in the data graph
  uint64_t nonadj[MAXM][2] = {};
  double est_rows = 0.0;       // planner's estimate of the rows after the step
  float feat[32] = {};         // features seen by the cardinality model
};

struct MotifStats {
  int32_t id;
  int64_t rows;      // |Res(M)|
};

struct GraphStats {
  int32_t V = 0;
  int64_t nnz = 0;
  double avg_deg = 0, max_deg = 0;
  std::vector<MotifStats> motifs;
  int64_t rows_of(int id) const {
    for (auto &m : motifs)
      if (m.id == id) return m.rows;
    return -1;
  }
};

// Features per candidate step seen by the cardinality model (DM_ORDER_LEARNED).
constexpr int NFEAT = 32;

struct Plan {
  int32_t n_p = 0;
  std::vector<int32_t> rp, ci;          // pattern CSR
  std::vector<int32_t> motifs;          // motif set used
  std::vector<StepSpec> steps;
  int32_t col_vertex[MAXW] = {};        // working column -> pattern vertex
  int32_t graph = -1;
  int32_t order = 0, join_algo = 0;
  int32_t induced = 0;                  // 1: non-adjacent pattern pairs must map to non-adjacent vertices
  int64_t chunk_rows = 0, max_rows = 0;
  double pred_cost = 0;      // predicted bytes moved by the joins plus a per-step overhead
  double pred_max_rows = 0;  // predicted largest intermediate table
  std::vector<float> pred_growth;  // predicted log growth of each step (model or heuristic)
};

// Decompose a pattern (Sec. 3.2). Returns 0 or a DM_E_* code.
int decompose(const Plan &pat, const std::vector<int32_t> &motif_set, int order,
              const GraphStats &gs, std::vector<StepSpec> *out, int32_t *col_vertex);

// Features of a candidate step (for the heuristic and the learned model).
void step_features(const StepSpec &s, int n_edges, double log_rows_prev, int n_p, int mapped_before,
                   int uncovered_before, const GraphStats &gs, float *feat);
double heuristic_log_rows(const float *feat);

// ------------------------------------------------------------------- device args -------
struct HashSlot {
  unsigned long long key;
  int32_t start;
  int32_t len;
};
constexpr unsigned long long HASH_EMPTY = ~0ull;

struct IndexView {
  int32_t nkeys;          // 0 = every row matches, 1 = direct offsets, 2 = hashed packed key
  int32_t kpos[2];        // motif positions forming the key
  const int32_t *rows;    // motif rows sorted by key, [n x mw]
  const float *score;     // edge-error sum of each motif row (nullable)
  int64_t n;
  int32_t mw;
  const int32_t *offsets; // nkeys == 1: [V + 1]
  const HashSlot *slots;  // nkeys == 2: 2^log2cap slots
  uint32_t log2cap;
  const unsigned long long *keys;  // sort-merge join: packed key of every row, ascending (then
                                   // offsets and slots are unused)
};

enum { CTR_ROWS = 0, CTR_NEXT = 1, CTR_SUM = 2, CTR_OVF = 3, CTR_CAND = 4, CTR_N = 8 };

struct JoinArgs {
  // input table R (row-major, width w); R == nullptr with w == 0 seeds from the motif table
  const int32_t *R;
  const float *Rs;
  int64_t N;
  const unsigned long long *n_dev;  // when set, the row count of R is read from here on the device,
  int64_t in_cap;                   // clamped to in_cap (rows R can hold; a producer may have overflowed)
  int32_t w;
  // the motif side
  IndexView ix;
  int32_t key_col[2];
  int32_t n_chk;
  int8_t chk_mpos[MAXM];
  int8_t chk_col[MAXM];
  int32_t n_new;
  int8_t new_mpos[MAXM];
  int32_t n_be;
  int8_t be_a[MAXBE];
  int8_t be_b[MAXBE];
  int32_t induced;                   // 1: also require non-adjacency for the columns in nonadj
  unsigned long long nonadj[MAXM][2];  // per new vertex: working columns it must not be adjacent to
  int32_t wo;                // output width = w + n_new
  int8_t src_col[MAXW];      // position q of a written row holds working column src_col[q]
  // data graph
  const unsigned long long *adj;
  int32_t adj_words;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const float *eerr;
  const float *qerr;
  int32_t scored;
  float prune;               // drop rows whose score exceeds this (no pruning: +inf)
  // output
  int32_t mode;              // 0 = write rows, 1 = count + checksum
  int32_t *out;
  float *outs;
  int32_t *out_next;         // candidate count of each written row for the next step (nullable)
  int64_t out_cap;
  unsigned long long *ctr;   // CTR_* counters
  IndexView nx;              // next step's index (nkeys < 0: none)
  int32_t nx_key_col[2];
  // seed mode (R == nullptr): motif rows [seed_lo, seed_hi) are the candidates
  int64_t seed_lo, seed_hi;
  // seed mode with n_shards > 1: keep only motif rows whose position-0 vertex is congruent to
  // shard modulo n_shards (one shard of the first table R_0)
  int32_t shard, n_shards;
  // padded layouts of the intermediate tables a device-driven chain passes from launch to
  // launch: rows of rs_in (R) / rs_out (out) words, a multiple of 4, so every row starts on a
  // 16-byte boundary; the words past w (past wo) are -1. 0: rows are packed (stride w / wo).
  // A padded output needs the working-column order (the row's w words, then the n_new <= 4 new
  // vertices).
  int32_t rs_in, rs_out;
};

}  // namespace dmi
