// Pattern decomposition into motif slices (Sec. 3.2) and join ordering.
//
// Decomposition loop (Sec. 3.2): the motif set is scanned largest first; a small
// backtracking matcher (the role VF2 plays in the paper) finds one slice S_i of the reduced
// pattern graph; the slice's pattern vertices that were mapped before become join keys
// (the overlap constraints, e.g. S_0[0] = S_1[3] in the 6-cycle example); the slice's edges
// are removed from the reduced graph, and vertices left without uncovered edges drop out.
//
// Readings where the paper leaves a choice open:
//  * which match is taken: the lexicographically smallest tuple of pattern ids (motif
//    positions in order) among matches that share at least one vertex with the mapped set
//    (any match for S_0); the result set does not depend on this choice;
//  * a slice matches the reduced graph on uncovered edges only, so no pattern edge is
//    covered twice, and a pattern edge whose two endpoints are mapped but which no slice
//    covered is checked against the data graph in the step that maps its second endpoint
//    (a back-edge; the paper would join Res(M2) on both endpoints instead);
//  * M2 always matches an uncovered edge that touches the mapped set (the pattern is
//    connected), so the loop always ends.
// DM_ORDER_HEURISTIC instead picks, among candidate slices of every motif, the one with the
// smallest estimated growth of the intermediate table per newly mapped vertex (independence
// estimate). DM_ORDER_LEARNED chooses among whole candidate plans (api.cu) by the trained
// model's predicted cost.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "../../include/dm.h"
#include "dm_internal.h"

namespace dmi {

static void add_edge(MotifDef *m, int a, int b) {
  m->edges.push_back({a, b});
  m->adj[a] |= 1u << b;
  m->adj[b] |= 1u << a;
}

bool motif_def(int id, MotifDef *out) {
  MotifDef m;
  m.id = id;
  if (id == MOTIF_VERTEX) {
    m.k = 1;
    m.name = "M1";
  } else if (id >= 2 && id <= MAXM) {  // M_k: path on k vertices
    m.k = id;
    for (int i = 0; i + 1 < id; i++) add_edge(&m, i, i + 1);
    m.name = "M" + std::to_string(id);
  } else if (id >= 103 && id <= 100 + MAXM) {  // M_{k-O}: k-cycle
    m.k = id - 100;
    for (int i = 0; i < m.k; i++) add_edge(&m, i, (i + 1) % m.k);
    m.name = "M" + std::to_string(m.k) + "-O";
  } else if (id == DM_MOTIF_M4_1) {  // claw: centre 0, leaves 1..3
    m.k = 4;
    for (int i = 1; i < 4; i++) add_edge(&m, 0, i);
    m.name = "M4-1";
  } else if (id == DM_MOTIF_M6_2O) {  // 2 x 3 grid: 0-1-2 / 3-4-5, rungs 0-3, 1-4, 2-5
    m.k = 6;
    add_edge(&m, 0, 1);
    add_edge(&m, 1, 2);
    add_edge(&m, 3, 4);
    add_edge(&m, 4, 5);
    add_edge(&m, 0, 3);
    add_edge(&m, 1, 4);
    add_edge(&m, 2, 5);
    m.name = "M6-2O";
  } else if (id == DM_MOTIF_M18_O_6) {  // 12-cycle, pendant 12 + i/2 on each even i
    m.k = 18;
    for (int i = 0; i < 12; i++) add_edge(&m, i, (i + 1) % 12);
    for (int i = 0; i < 12; i += 2) add_edge(&m, i, 12 + i / 2);
    m.name = "M18-O-6";
  } else {
    return false;
  }
  for (int p = 0; p < m.k; p++) {
    m.parent[p] = -1;
    for (int q = 0; q < p; q++)
      if (m.adj[p] >> q & 1u) {
        m.parent[p] = q;
        break;
      }
    if (p > 0 && m.parent[p] < 0) return false;  // positions must grow a connected prefix
  }
  *out = m;
  return true;
}

// ---------------------------------------------------------------- reduced pattern -----
static inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

// A set of pattern vertices (ids < MAXW = 128).
struct VSet {
  uint64_t w[2] = {0, 0};
  bool test(int v) const { return (w[v >> 6] >> (v & 63)) & 1ull; }
  void set(int v) { w[v >> 6] |= 1ull << (v & 63); }
  void clear(int v) { w[v >> 6] &= ~(1ull << (v & 63)); }
  bool any() const { return (w[0] | w[1]) != 0; }
  int count() const { return popc64(w[0]) + popc64(w[1]); }
  VSet operator&(const VSet &o) const {
    VSet r;
    r.w[0] = w[0] & o.w[0];
    r.w[1] = w[1] & o.w[1];
    return r;
  }
  VSet without(const VSet &o) const {
    VSet r;
    r.w[0] = w[0] & ~o.w[0];
    r.w[1] = w[1] & ~o.w[1];
    return r;
  }
  VSet with(int v) const {
    VSet r = *this;
    r.set(v);
    return r;
  }
  int pop_lowest() {  // smallest member, removed; the set must not be empty
    const int h = w[0] ? 0 : 1;
    const int b = __builtin_ctzll(w[h]);
    w[h] &= w[h] - 1;
    return 64 * h + b;
  }
};
static_assert(MAXW <= 128, "VSet holds 128 vertices");

struct PState {
  int n = 0;
  VSet adj0[MAXW];  // pattern adjacency
  VSet unc[MAXW];   // uncovered pattern edges
  VSet mapped;
  int ncols = 0;
  int col_of[MAXW];
  int col_vertex[MAXW];
  int uncovered_edges = 0;
};

// Visit matches of motif `m` in the uncovered graph in lexicographic order of the tuple
// (image of position 0, 1, ...). `f(img)` returns false to stop. `budget` bounds the
// number of search nodes.
template <class F>
static bool match_rec(const MotifDef &m, const PState &st, bool need_overlap, int p, int *img,
                      const VSet &used, long long &budget, F &f) {
  if (--budget < 0) return false;
  if (p == m.k) {
    if (need_overlap && !(used & st.mapped).any()) return true;
    return f(img);
  }
  VSet cand;
  int deg_p = __builtin_popcount(m.adj[p]);
  if (p == 0) {
    for (int v = 0; v < st.n; v++)
      if (st.unc[v].any()) cand.set(v);
  } else {
    cand = st.unc[img[m.parent[p]]];
  }
  cand = cand.without(used);
  while (cand.any()) {
    int v = cand.pop_lowest();
    if (st.unc[v].count() < deg_p) continue;
    bool ok = true;
    for (int q = 0; q < p && ok; q++)
      if (m.adj[p] >> q & 1u) ok = st.unc[v].test(img[q]);
    if (!ok) continue;
    img[p] = v;
    if (!match_rec(m, st, need_overlap, p + 1, img, used.with(v), budget, f)) return false;
  }
  return true;
}

static void make_step(const MotifDef &m, const int *img, const PState &st, StepSpec *s) {
  memset(s, 0, sizeof(*s));
  s->motif = m.id;
  s->k = m.k;
  s->w_in = st.ncols;
  for (int p = 0; p < m.k; p++) {
    s->slice[p] = img[p];
    if (st.mapped.test(img[p])) {
      s->key_mpos[s->n_keys] = p;
      s->key_col[s->n_keys] = st.col_of[img[p]];
      s->n_keys++;
    } else {
      s->new_mpos[s->n_new++] = p;
    }
  }
  s->w_out = s->w_in + s->n_new;
  for (int i = 0; i < s->n_new; i++) {  // non-edges to check under induced matching
    const int p = img[s->new_mpos[i]];
    for (int c = 0; c < s->w_in + i; c++) {
      const int q = c < s->w_in ? st.col_vertex[c] : img[s->new_mpos[c - s->w_in]];
      if (!st.adj0[p].test(q)) s->nonadj[i][c >> 6] |= 1ull << (c & 63);
    }
  }
  // back-edges: uncovered pattern edges with both ends mapped after this step, that the
  // slice itself does not cover
  VSet after = st.mapped;
  for (int p = 0; p < m.k; p++) after.set(img[p]);
  VSet cov[MAXW];
  for (auto &e : m.edges) {
    cov[img[e.first]].set(img[e.second]);
    cov[img[e.second]].set(img[e.first]);
  }
  int colmap[MAXW];
  for (int v = 0; v < st.n; v++) colmap[v] = st.mapped.test(v) ? st.col_of[v] : -1;
  for (int i = 0; i < s->n_new; i++) colmap[img[s->new_mpos[i]]] = s->w_in + i;
  for (int a = 0; a < st.n; a++) {
    if (!after.test(a)) continue;
    VSet rest = st.unc[a].without(cov[a]) & after;
    while (rest.any()) {
      int b = rest.pop_lowest();
      if (b <= a) continue;
      // only edges that become checkable now: at least one endpoint is new in this step
      bool a_new = !st.mapped.test(a), b_new = !st.mapped.test(b);
      if (!a_new && !b_new) continue;
      if (s->n_be < MAXBE) {
        s->be_vtx[s->n_be][0] = a;
        s->be_vtx[s->n_be][1] = b;
        s->be_col[s->n_be][0] = colmap[a];
        s->be_col[s->n_be][1] = colmap[b];
      }
      s->n_be++;
    }
  }
}

static void apply_step(const MotifDef &m, const StepSpec &s, PState *st) {
  for (auto &e : m.edges) {
    int a = s.slice[e.first], b = s.slice[e.second];
    if (st->unc[a].test(b)) st->uncovered_edges--;
    st->unc[a].clear(b);
    st->unc[b].clear(a);
  }
  for (int i = 0; i < s.n_new; i++) {
    int v = s.slice[s.new_mpos[i]];
    st->col_of[v] = st->ncols;
    st->col_vertex[st->ncols] = v;
    st->ncols++;
    st->mapped.set(v);
  }
  for (int i = 0; i < s.n_be && i < MAXBE; i++) {
    int a = s.be_vtx[i][0], b = s.be_vtx[i][1];
    if (st->unc[a].test(b)) st->uncovered_edges--;
    st->unc[a].clear(b);
    st->unc[b].clear(a);
  }
}

void step_features(const StepSpec &s, int n_edges, double log_rows_prev, int n_p, int mapped_before,
                   int uncovered_before, const GraphStats &gs, float *f) {
  memset(f, 0, sizeof(float) * NFEAT);
  double T = 1.0;
  for (auto &ms : gs.motifs)
    if (ms.id == s.motif) T = (double)std::max<int64_t>(1, ms.rows);
  double V = std::max(1, gs.V);
  bool cyc = s.motif >= 103 && s.motif <= 100 + MAXM;
  bool pth = s.motif >= 2 && s.motif <= MAXM;
  f[0] = (float)log_rows_prev;
  f[1] = (float)log(T);
  f[2] = (float)log(V);
  f[3] = (float)gs.avg_deg;
  f[4] = (float)gs.max_deg;
  f[5] = (float)s.k;
  f[6] = (float)s.n_keys;
  f[7] = (float)s.n_new;
  f[8] = (float)s.n_be;
  f[9] = cyc ? 1.f : 0.f;
  f[10] = pth ? 1.f : 0.f;
  f[11] = (!cyc && !pth) ? 1.f : 0.f;
  f[12] = (float)std::min(2, s.n_keys);
  f[13] = (float)std::max(0, s.n_keys - 2);
  f[14] = (float)s.w_in / (float)std::max(1, n_p);
  f[15] = (float)mapped_before / (float)std::max(1, n_p);
  f[16] = (float)uncovered_before;
  f[17] = (float)n_edges;
  f[18] = (float)(log(T) - log(V));
  f[19] = (float)s.w_in;
  f[20] = (float)n_p;
  f[21] = mapped_before == 0 ? 1.f : 0.f;
  // independence estimate (the plain heuristic), also given to the model as a feature
  double lr;
  double lsel = log(std::max(1e-9, gs.avg_deg / V));
  if (mapped_before == 0) lr = log(T) + s.n_be * lsel;
  else lr = log_rows_prev + log(T) - s.n_keys * log(V) + s.n_be * lsel;
  f[22] = (float)lr;
}

double heuristic_log_rows(const float *f) { return (double)f[22]; }

static int build_pstate(const Plan &pat, PState *st) {
  st->n = pat.n_p;
  for (int u = 0; u < pat.n_p; u++)
    for (int k = pat.rp[u]; k < pat.rp[u + 1]; k++) {
      int v = pat.ci[k];
      st->unc[u].set(v);
      st->adj0[u].set(v);
      if (u < v) st->uncovered_edges++;
    }
  for (int i = 0; i < MAXW; i++) st->col_of[i] = -1;
  return 0;
}

int decompose(const Plan &pat, const std::vector<int32_t> &motif_set, int order,
              const GraphStats &gs, std::vector<StepSpec> *out, int32_t *col_vertex) {
  out->clear();
  PState st;
  build_pstate(pat, &st);
  if (pat.n_p == 1) {  // single vertex: every data vertex is an embedding
    StepSpec s;
    memset(&s, 0, sizeof(s));
    s.motif = MOTIF_VERTEX;
    s.k = 1;
    s.slice[0] = 0;
    s.n_new = 1;
    s.new_mpos[0] = 0;
    s.w_out = 1;
    s.est_rows = gs.V;
    out->push_back(s);
    col_vertex[0] = 0;
    return DM_OK;
  }
  // motif set, largest first (ties: the given order); M2 always present
  std::vector<MotifDef> defs;
  bool has_m2 = false;
  for (int id : motif_set) {
    MotifDef d;
    if (!motif_def(id, &d) || d.k < 2) return DM_E_NOTFOUND;
    if (id == 2) has_m2 = true;
    bool dup = false;
    for (auto &e : defs) dup |= e.id == id;
    if (!dup) defs.push_back(d);
  }
  if (!has_m2) {
    MotifDef d;
    motif_def(2, &d);
    defs.push_back(d);
  }
  std::stable_sort(defs.begin(), defs.end(), [](const MotifDef &a, const MotifDef &b) { return a.k > b.k; });

  double log_rows = 0.0;
  int guard = 0;
  while (st.uncovered_edges > 0) {
    if (++guard > MAXSTEPS) return DM_E_INVAL;
    bool first = !st.mapped.any();
    StepSpec best;
    bool found = false;
    if (order == DM_ORDER_PAPER) {
      for (auto &m : defs) {
        int img[MAXM];
        long long budget = 2000000;
        StepSpec s;
        auto f = [&](const int *im) {
          make_step(m, im, st, &s);
          return false;  // first match is enough
        };
        match_rec(m, st, !first, 0, img, VSet(), budget, f);
        if (budget >= 0 && s.k == m.k && s.motif == m.id) {
          best = s;
          found = true;
          break;
        }
      }
      if (found) {
        MotifDef bd;
        motif_def(best.motif, &bd);
        step_features(best, (int)bd.edges.size(), log_rows, pat.n_p, st.mapped.count(), st.uncovered_edges, gs,
                      best.feat);
        best.est_rows = exp(heuristic_log_rows(best.feat));
      }
    } else {
      // greedy: the match with the smallest estimated growth per new vertex (independence
      // estimate); ties: the larger motif, then enumeration order
      double bscore = 1e300;
      const int mapped_before = st.mapped.count();
      StepSpec s;
      float f[NFEAT];
      for (auto &m : defs) {
        int img[MAXM];
        long long budget = 400000;
        int taken = 0;
        const int n_edges = (int)m.edges.size();
        auto visit = [&](const int *im) {
          make_step(m, im, st, &s);
          if (s.n_be > MAXBE) return true;
          step_features(s, n_edges, log_rows, pat.n_p, mapped_before, st.uncovered_edges, gs, f);
          const double growth = ((double)heuristic_log_rows(f) - log_rows) / std::max(1, s.n_new);
          if (!found || growth < bscore - 1e-9 || (fabs(growth - bscore) <= 1e-9 && s.k > best.k)) {
            bscore = growth;
            best = s;
            memcpy(best.feat, f, sizeof(f));
            found = true;
          }
          return ++taken < 256;
        };
        match_rec(m, st, !first, 0, img, VSet(), budget, visit);
      }
      if (!found) return DM_E_INVAL;
      best.est_rows = exp(heuristic_log_rows(best.feat));
    }
    if (!found) return DM_E_INVAL;
    if (best.n_be > MAXBE) return DM_E_INVAL;
    MotifDef md;
    motif_def(best.motif, &md);
    apply_step(md, best, &st);
    log_rows = log(std::max(1.0, best.est_rows));
    out->push_back(best);
  }
  if (st.ncols != pat.n_p) return DM_E_DISCONNECTED;
  for (int c = 0; c < st.ncols; c++) col_vertex[c] = st.col_vertex[c];
  return DM_OK;
}

}  // namespace dmi
