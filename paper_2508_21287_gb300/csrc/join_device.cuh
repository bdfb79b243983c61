// Device side of one join step of Alg. 1 (InnerJoin + FilterOverlappingNodes + back-edge test
// + score + compaction) on one tile of the intermediate table R, as a whole block: the tile
// routine of the persistent batch kernel (batch.cu). The per-step kernel (join_warp.cu) uses
// the helpers here with one warp per tile instead.
//
// A block stages up to TR rows of R in shared memory (row stride join_row_stride(w): int4
// reads, padding words -1), looks up each row's key group in the motif index, and scans the
// group sizes into a candidate range. The candidates are then processed in rounds of BLK *
// CPT: each thread first issues the motif-row loads of its CPT candidates, then checks them
// (extra key equalities, injectivity of the new vertices against the whole row with int4
// compares, back-edges in the adjacency bitmap, FP32 score); survivors are compacted with a
// block scan, their output range is reserved once per round, and the block writes the rows
// element by element so that consecutive threads store consecutive words.
//
// Checksum of a row (count mode): H = mix64(n + sum_q mix64(((q + 1) << 32) | f(q))) over the
// output positions q, sums mod 2^64. The terms of the columns that come from the R row are
// summed once per tile row; each surviving candidate adds the terms of its new vertices.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dm_internal.h"

namespace dmk {

using namespace dmi;

#define FULL_MASK 0xffffffffu

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ unsigned long long dmix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// GPU global timer (ns).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Programmatic dependent launch: wait until the previous grid in the stream has completed and
// its writes are visible (a no-op when the kernel was launched without the attribute), and
// allow the next grid to be scheduled.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Order-preserving key of an FP32 score: unsigned comparison of the keys orders the scores by
// value for either sign (negative scores have their bits inverted, non-negative ones get the
// sign bit set); -0 and +0 share one key. Scores are finite (weights are checked on load).
__device__ __forceinline__ uint32_t score_key(float f) {
  uint32_t b = __float_as_uint(f);
  if (b == 0x80000000u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------------ index lookup -------
__device__ __forceinline__ void ix_lookup(const IndexView &ix, int32_t ka, int32_t kb, int32_t &start,
                                          int32_t &len) {
  if (ix.keys && ix.nkeys > 0) {  // sort-merge: the key's run in the sorted key column
    const unsigned long long key =
        ix.nkeys == 2 ? (((unsigned long long)(uint32_t)ka << 32) | (uint32_t)kb) : (unsigned long long)(uint32_t)ka;
    int64_t lo = 0, hi = ix.n;
    while (lo < hi) {  // first position with keys >= key
      const int64_t mid = (lo + hi) >> 1;
      if (__ldg(ix.keys + mid) < key) lo = mid + 1;
      else hi = mid;
    }
    int64_t e = lo, h2 = ix.n;
    while (e < h2) {  // first position with keys > key
      const int64_t mid = (e + h2) >> 1;
      if (__ldg(ix.keys + mid) <= key) e = mid + 1;
      else h2 = mid;
    }
    start = (int32_t)lo;
    len = (int32_t)(e - lo);
  } else if (ix.nkeys == 1) {
    start = __ldg(ix.offsets + ka);
    len = __ldg(ix.offsets + ka + 1) - start;
  } else if (ix.nkeys == 2) {
    unsigned long long key = ((unsigned long long)(uint32_t)ka << 32) | (uint32_t)kb;
    unsigned long long mask = (1ull << ix.log2cap) - 1;
    unsigned long long h = (key * 0x9E3779B97F4A7C15ull) >> (64 - ix.log2cap);
    start = 0;
    len = 0;
    for (unsigned long long probe = 0; probe <= mask; probe++) {
      const HashSlot *sl = ix.slots + h;
      unsigned long long k = sl->key;
      if (k == key) {
        start = sl->start;
        len = sl->len;
        break;
      }
      if (k == HASH_EMPTY) break;
      h = (h + 1) & mask;
    }
  } else {
    start = 0;
    len = (int32_t)ix.n;
  }
}

__device__ __forceinline__ bool adjacent(const JoinArgs &a, int32_t u, int32_t v) {
  if (a.adj) {
    unsigned long long word = __ldg(a.adj + (int64_t)u * a.adj_words + (v >> 6));
    return (word >> (v & 63)) & 1ull;
  }
  int32_t lo = __ldg(a.row_ptr + u), hi = __ldg(a.row_ptr + u + 1);
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    int32_t x = __ldg(a.col_idx + mid);
    if (x == v) return true;
    if (x < v) lo = mid + 1;
    else hi = mid;
  }
  return false;
}

__device__ __forceinline__ float edge_weight(const JoinArgs &a, int32_t u, int32_t v) {
  int32_t lo = __ldg(a.row_ptr + u), hi = __ldg(a.row_ptr + u + 1);
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    int32_t x = __ldg(a.col_idx + mid);
    if (x == v) return __ldg(a.eerr + mid);
    if (x < v) lo = mid + 1;
    else hi = mid;
  }
  return 0.f;
}

// ------------------------------------------------------------------ block helpers ------
template <int BLK>
__device__ __forceinline__ int block_excl_scan(int x, int &total, int *s_warp) {
  constexpr int NW = BLK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int wv = lane < NW ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(FULL_MASK, wv, o);
      if (lane >= o) wv += t;
    }
    if (lane < NW) s_warp[lane] = wv;
  }
  __syncthreads();
  int woff = warp ? s_warp[warp - 1] : 0;
  total = s_warp[NW - 1];
  __syncthreads();
  return woff + v - x;
}

template <int BLK>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long *s_red) {
  constexpr int NW = BLK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL_MASK, x, o);
  if (lane == 0) s_red[warp] = x;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NW; i++) t += s_red[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// Checksum term of value v at output position p - 1 (p = 1 + position < 2^30): SplitMix64's
// finaliser of (p << 32) | v, whose first xorshift leaves the high word p unchanged.
__device__ __forceinline__ unsigned long long pos_term(uint32_t p, int32_t v) {
  const uint32_t lo = (uint32_t)v ^ ((uint32_t)v >> 30) ^ (p << 2);
  unsigned long long z = (((unsigned long long)p << 32) | lo) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Checksum term of vertex v at output position q.
__device__ __forceinline__ unsigned long long col_term(int q, int32_t v) {
  return pos_term((uint32_t)(q + 1), v);
}

// true when v equals one of the first w words of a shared-memory row (stride join_row_stride,
// padding -1, so whole int4s can be compared)
__device__ __forceinline__ bool row_has(const int32_t *row, int w, int32_t v) {
  const int4 *r4 = (const int4 *)row;
  bool hit = false;
#pragma unroll 2
  for (int c4 = 0; c4 < (w + 3) >> 2; c4++) {
    const int4 x = r4[c4];
    hit |= (x.x == v) | (x.y == v) | (x.z == v) | (x.w == v);
  }
  return hit;
}

// Sum of the checksum terms of the first w words of a shared-memory row; ipos[c] is the output
// position of column c (-1: not output), defined for c < 4 * ceil(w / 4) <= MAXW.
__device__ __forceinline__ unsigned long long row_terms(const int32_t *row, int w, const int8_t *ipos) {
  const int4 *r4 = (const int4 *)row;
  unsigned long long p = 0;
  for (int c4 = 0; c4 < (w + 3) >> 2; c4++) {
    const int4 x = r4[c4];
    const int c = 4 * c4;
    if (ipos[c] >= 0) p += col_term(ipos[c], x.x);
    if (ipos[c + 1] >= 0) p += col_term(ipos[c + 1], x.y);
    if (ipos[c + 2] >= 0) p += col_term(ipos[c + 2], x.z);
    if (ipos[c + 3] >= 0) p += col_term(ipos[c + 3], x.w);
  }
  return p;
}

struct JoinSmem {
  int32_t *tile_buf[2];  // R tiles
  float *ts_buf[2];
  unsigned long long *part;  // per row: checksum terms of its columns (count mode)
  int32_t *gstart, *goff;
  int32_t *surv_r, *surv_m;
  int32_t *cand_row;
  int16_t *code;  // per output position: working column (< 0x100: from the R row) or 0x100 | motif position
  int8_t *ipos;   // per R column: its output position (-1: none)
  int8_t *npos;   // per new vertex: its output position
  unsigned long long *bm;  // optional: per tile row, a bitmap of its vertex ids (bmw words a row)
  int bmw;
};

__host__ __device__ __forceinline__ size_t join_smem_layout(int TR, int ws, int BLKCPT, int nbuf, size_t *offs) {
  size_t off = 0;
  for (int b = 0; b < 2; b++) {
    offs[b] = off;
    if (b < nbuf) off += ((size_t)TR * ws * 4 + 15) / 16 * 16;
  }
  for (int b = 0; b < 2; b++) {
    offs[2 + b] = off;
    if (b < nbuf) off += ((size_t)TR * 4 + 15) / 16 * 16;
  }
  offs[4] = off;  // partial checksums
  off += (size_t)TR * 8;
  offs[5] = off;  // group starts, offsets
  off += (size_t)TR * 4 + (size_t)(TR + 1) * 4;
  off = (off + 15) / 16 * 16;
  offs[6] = off;  // survivors, candidate rows, codes
  off += (size_t)BLKCPT * 4 * 3 + (size_t)MAXW * 3 + MAXM;
  return (off + 15) / 16 * 16;
}

__device__ __forceinline__ JoinSmem join_smem(unsigned char *smem, int TR, int ws, int BLKCPT, int nbuf) {
  size_t o[7];
  join_smem_layout(TR, ws, BLKCPT, nbuf, o);
  JoinSmem m;
  m.tile_buf[0] = (int32_t *)(smem + o[0]);
  m.tile_buf[1] = (int32_t *)(smem + (nbuf > 1 ? o[1] : o[0]));
  m.ts_buf[0] = (float *)(smem + o[2]);
  m.ts_buf[1] = (float *)(smem + (nbuf > 1 ? o[3] : o[2]));
  m.part = (unsigned long long *)(smem + o[4]);
  m.gstart = (int32_t *)(smem + o[5]);
  m.goff = m.gstart + TR;
  m.surv_r = (int32_t *)(smem + o[6]);
  m.surv_m = m.surv_r + BLKCPT;
  m.cand_row = m.surv_m + BLKCPT;
  m.code = (int16_t *)(m.cand_row + BLKCPT);
  m.ipos = (int8_t *)(m.code + MAXW);
  m.npos = m.ipos + MAXW;
  m.bm = nullptr;
  m.bmw = 0;
  return m;
}

// Copy nr rows (width w) from src into a shared tile of row stride join_row_stride(w), with
// -1 in the padding words, and their scores.
template <int BLK>
__device__ __forceinline__ void load_tile(int32_t *tile, float *ts, const int32_t *src, const float *srcs, int nr,
                                          int w) {
  const int ws = join_row_stride(w);
  const int ne = nr * w;
  const int dr = BLK / w, dc = BLK % w;
  int r = threadIdx.x / w, c = threadIdx.x % w;  // element e = r * w + c, advanced with carry
  for (int e = threadIdx.x; e < ne; e += BLK) {
    tile[r * ws + c] = __ldg(src + e);
    r += dr;
    c += dc;
    if (c >= w) {
      c -= w;
      r++;
    }
  }
  const int np = ws - w;
  for (int e = threadIdx.x; e < nr * np; e += BLK) tile[(e / np) * ws + w + e % np] = -1;
  if (srcs)
    for (int i = threadIdx.x; i < nr; i += BLK) ts[i] = __ldg(srcs + i);
}

// Induced matching: every new vertex must not be adjacent to the images of the columns its
// pattern vertex is not adjacent to (the columns in a.nonadj[i]).
template <int MAXNEW>
__device__ __forceinline__ int32_t nv_pick(const int32_t (&nv)[MAXNEW], int k) {
  int32_t v = 0;
#pragma unroll
  for (int i = 0; i < MAXNEW; i++)
    if (i == k) v = nv[i];
  return v;
}

template <int MAXNEW>
__device__ __forceinline__ bool induced_ok(const JoinArgs &a, const int32_t *rrow, const int32_t (&nv)[MAXNEW]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < MAXNEW; i++) {
    if (i < a.n_new && ok) {
      for (int h = 0; h < 2 && ok; h++) {
        unsigned long long mk = a.nonadj[i][h];
        while (mk && ok) {
          const int c = 64 * h + __ffsll((long long)mk) - 1;
          mk &= mk - 1;
          const int32_t v = c < a.w ? rrow[c] : nv_pick<MAXNEW>(nv, c - a.w);
          ok = !adjacent(a, nv[i], v);
        }
      }
    }
  }
  return ok;
}

// Value of working column `col` of the joined row (R row `rrow`, motif row `trow`).
__device__ __forceinline__ int32_t join_value(const JoinArgs &a, const int32_t *rrow, const int32_t *trow, int col) {
  return col < a.w ? rrow[col] : __ldg(trow + a.new_mpos[col - a.w]);
}

// New vertex i of a candidate: preloaded in registers for steps with few new vertices; read
// from the motif row when needed (and only while the candidate survives) for the wide variant,
// whose candidates mostly fail after a few of their many new vertices.
template <int MAXNEW>
__device__ __forceinline__ int32_t new_vertex(const JoinArgs &a, const int32_t *trow, const int32_t (&nv)[MAXNEW],
                                              int i) {
  return MAXNEW > 4 ? __ldg(trow + a.new_mpos[i]) : nv[i];
}

template <int MAXNEW>
__device__ __forceinline__ bool induced_ok_lazy(const JoinArgs &a, const int32_t *rrow, const int32_t *trow) {
  bool ok = true;
  for (int i = 0; i < a.n_new && ok; i++) {
    const int32_t vi = __ldg(trow + a.new_mpos[i]);
    for (int h = 0; h < 2 && ok; h++) {
      unsigned long long mk = a.nonadj[i][h];
      while (mk && ok) {
        const int c = 64 * h + __ffsll((long long)mk) - 1;
        mk &= mk - 1;
        const int32_t v = c < a.w ? rrow[c] : __ldg(trow + a.new_mpos[c - a.w]);
        ok = !adjacent(a, vi, v);
      }
    }
  }
  return ok;
}

// Join, filter and score one candidate (R row r of the tile, motif row m); for MAXNEW <= 4 its
// new vertices nv were loaded beforehand.
template <int MAXNEW>
__device__ __forceinline__ bool join_check(const JoinArgs &a, const JoinSmem &S, const int32_t *tile, const float *ts,
                                           int ws, bool seed, int r, int m, const int32_t (&nv)[MAXNEW], float &sc) {
  const int32_t *rrow = tile + r * ws;
  const int32_t *trow = a.ix.rows + (int64_t)m * a.ix.mw;
  bool ok = true;
  for (int i = 0; i < a.n_chk; i++) ok &= __ldg(trow + a.chk_mpos[i]) == rrow[a.chk_col[i]];
  if (ok && !seed) {  // FilterOverlappingNodes: new vertices must not repeat a mapped one
    if (MAXNEW > 4 && S.bm) {  // many new vertices: one bit test each in the row's id bitmap
      const unsigned long long *b = S.bm + (size_t)r * S.bmw;
      for (int i = 0; i < a.n_new && ok; i++) {
        const int32_t v = new_vertex<MAXNEW>(a, trow, nv, i);
        ok = !((b[v >> 6] >> (v & 63)) & 1ull);
      }
    } else if (MAXNEW > 4) {
      for (int i = 0; i < a.n_new && ok; i++) ok = !row_has(rrow, a.w, new_vertex<MAXNEW>(a, trow, nv, i));
    } else {
#pragma unroll
      for (int i = 0; i < MAXNEW; i++)
        if (i < a.n_new && ok) ok = !row_has(rrow, a.w, nv[i]);
    }
  }
  sc = 0.f;
  if (a.scored && ok) {
    sc = (!seed && a.Rs) ? ts[r] : 0.f;
    if (a.ix.score) sc += __ldg(a.ix.score + m);
    if (a.qerr) {
      if (MAXNEW > 4) {
        for (int i = 0; i < a.n_new; i++) sc += __ldg(a.qerr + new_vertex<MAXNEW>(a, trow, nv, i));
      } else {
#pragma unroll
        for (int i = 0; i < MAXNEW; i++)
          if (i < a.n_new) sc += __ldg(a.qerr + nv[i]);
      }
    }
  }
  for (int e = 0; e < a.n_be && ok; e++) {
    int32_t va = join_value(a, rrow, trow, a.be_a[e]);
    int32_t vb = join_value(a, rrow, trow, a.be_b[e]);
    ok = adjacent(a, va, vb);
    if (ok && a.scored && a.eerr) sc += edge_weight(a, va, vb);
  }
  if (ok && a.induced) ok = MAXNEW > 4 ? induced_ok_lazy<MAXNEW>(a, rrow, trow) : induced_ok<MAXNEW>(a, rrow, nv);
  if (sc > a.prune) ok = false;
  return ok;
}

// Where the rows of a tile go: a global table with an atomic row counter (k_join) or a
// block-private buffer with a shared-memory counter (batch kernel).
struct TileOut {
  int32_t *out;
  float *outs;
  int32_t *out_next;
  int64_t cap;
  unsigned long long *gctr;  // global row counter, or nullptr
  long long *lctr;           // shared-memory row counter when gctr == nullptr
  unsigned long long *ovf;   // set to 1 when a round did not fit
  unsigned long long *next_ctr;  // total next-step candidates of the written rows (nullable)
};

// Process one tile: rows src[0 .. nr) of R (width a.w) -- already in shared buffer `buf` when
// `loaded` --, or, in seed mode (src == nullptr), motif rows [seed_m0, seed_m0 + seed_C) as
// candidates. MODE 0 writes survivors through `o`; MODE 1 adds their count and checksum hashes
// to acc_rows / acc_sum (per thread).
template <int BLK, int MAXNEW, int CPT, int MODE>
__device__ __forceinline__ void join_tile(const JoinArgs &a, const JoinSmem &S, int TR, int buf, bool loaded,
                                          const int32_t *src, const float *srcs, int nr, int64_t seed_m0, int seed_C,
                                          const TileOut &o, int *s_warp, unsigned long long *s_red, long long *s_base,
                                          unsigned long long &acc_rows, unsigned long long &acc_sum,
                                          unsigned long long &acc_cand) {
  const bool seed = src == nullptr;
  const int w = a.w, wo = a.wo;
  const int ws = join_row_stride(w);
  const int tid = threadIdx.x;
  int32_t *tile = S.tile_buf[buf];
  float *ts = S.ts_buf[buf];
  // output position -> source, in shared memory: lanes look it up with different indices,
  // which the constant bank would serialise
  if (MODE == 1)
    for (int q = tid; q < MAXW; q += BLK) S.ipos[q] = -1;
  for (int q = tid; q < wo; q += BLK) {
    const int col = a.src_col[q];
    S.code[q] = (int16_t)(col < w ? col : (0x100 | a.new_mpos[col - w]));
    if (MODE == 1 && col >= w) S.npos[col - w] = (int8_t)q;
  }
  if (MODE == 1) {
    __syncthreads();
    for (int q = tid; q < wo; q += BLK) {
      const int col = a.src_col[q];
      if (col < w) S.ipos[col] = (int8_t)q;
    }
  }
  int C;
  if (seed) __syncthreads();
  if (!seed) {
    if (!loaded) load_tile<BLK>(tile, ts, src, srcs, nr, w);
    __syncthreads();
    int len = 0, start = 0;
    if (tid < nr) {
      const int32_t *row = tile + tid * ws;
      if (MODE == 1) {  // checksum terms of the row's own columns
        S.part[tid] = row_terms(row, w, S.ipos);
      }
      if (MAXNEW > 4 && S.bm) {  // the row's id bitmap (ids < 64 * bmw)
        unsigned long long *b = S.bm + (size_t)tid * S.bmw;
        for (int q = 0; q < S.bmw; q++) b[q] = 0ull;
        for (int c = 0; c < w; c++) b[row[c] >> 6] |= 1ull << (row[c] & 63);
      }
      ix_lookup(a.ix, row[a.key_col[0]], a.ix.nkeys == 2 ? row[a.key_col[1]] : 0, start, len);
    }
    int total;
    int off = block_excl_scan<BLK>(tid < TR ? len : 0, total, s_warp);
    if (tid < TR) {
      S.gstart[tid] = start;
      S.goff[tid] = off;
    }
    if (tid == 0) S.goff[TR] = total;
    __syncthreads();
    C = total;
  } else {
    C = seed_C;
  }
  acc_cand += tid == 0 ? (unsigned long long)C : 0ull;
  const int st_s0 = tid / wo, st_q0 = tid % wo, st_ds = BLK / wo, st_dq = BLK % wo;
  const int32_t *mrows = a.ix.rows;
  const int mw = a.ix.mw;

  for (int rb = 0; rb < C; rb += BLK * CPT) {
    if (!seed) {  // tile row of every candidate of this round
      if (MODE == 1 && rb > 0) __syncthreads();  // the previous round's readers are done
      const int re = rb + BLK * CPT;
      for (int r = tid; r < TR; r += BLK) {
        int lo = max(S.goff[r], rb), hi = min(S.goff[r + 1], re);
        for (int c = lo; c < hi; c++) S.cand_row[c - rb] = r;
      }
      __syncthreads();
    }
    int myr[CPT];
    int mym[CPT];  // motif tables hold fewer than 2^31 rows
    float mys[CPT];
    int32_t nv[CPT][MAXNEW];
    // all motif-row loads of the thread's candidates first, then the dependent checks
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      const int c = rb + k * BLK + tid;
      int r = 0, m = 0;
      if (c < C) {
        if (seed) {
          m = (int)(seed_m0 + c);
        } else {
          r = S.cand_row[c - rb];
          m = S.gstart[r] + (c - S.goff[r]);
        }
      }
      myr[k] = r;
      mym[k] = m;
      const int32_t *trow = mrows + (int64_t)m * mw;  // row 0 for idle lanes: a valid address
      if (MAXNEW <= 4) {  // the wide variant reads its new vertices lazily (join_check)
#pragma unroll
        for (int i = 0; i < MAXNEW; i++)
          if (i < a.n_new) nv[k][i] = __ldg(trow + a.new_mpos[i]);
      }
    }
    unsigned pass = 0;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      const int c = rb + k * BLK + tid;
      mys[k] = 0.f;
      if (c < C) {
        float sc;
        if (join_check<MAXNEW>(a, S, tile, ts, ws, seed, myr[k], mym[k], nv[k], sc)) {
          pass |= 1u << k;
          mys[k] = sc;
          if (MODE == 1) {
            unsigned long long p = seed ? 0ull : S.part[myr[k]];
            const int32_t *trow = mrows + (int64_t)mym[k] * mw;
            if (MAXNEW > 4) {
              for (int i = 0; i < a.n_new; i++) p += col_term(S.npos[i], __ldg(trow + a.new_mpos[i]));
            } else {
#pragma unroll
              for (int i = 0; i < MAXNEW; i++)
                if (i < a.n_new) p += col_term(S.npos[i], nv[k][i]);
            }
            acc_sum += dmix64(p + (unsigned long long)(uint32_t)wo);
            acc_rows++;
          }
        }
      }
    }
    if (MODE == 1) continue;
    // compaction: block scan of per-thread survivor counts, one reservation per round
    int K;
    const int pos0 = block_excl_scan<BLK>(__popc(pass), K, s_warp);
    if (K == 0) continue;
    if (tid == 0) {
      if (o.gctr) *s_base = (long long)atomicAdd(o.gctr, (unsigned long long)K);
      else {
        *s_base = *o.lctr;
        *o.lctr += K;
      }
    }
    __syncthreads();
    const long long base = *s_base;
    int Kc = K;
    if (base + K > o.cap) {
      Kc = (int)imax64(0, o.cap - base);
      if (tid == 0) atomicOr(o.ovf, 1ull);
    }
    unsigned long long nsum = 0;
    int pos = pos0;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      if (pass >> k & 1u) {
        S.surv_r[pos] = myr[k];
        S.surv_m[pos] = mym[k];
        if (pos < Kc) {
          if (o.outs) o.outs[base + pos] = mys[k];
          if (o.out_next) {
            const int32_t *rrow = tile + myr[k] * ws;
            const int32_t *trow = mrows + (int64_t)mym[k] * mw;
            int32_t st, ln;
            ix_lookup(a.nx, join_value(a, rrow, trow, a.nx_key_col[0]),
                      a.nx.nkeys == 2 ? join_value(a, rrow, trow, a.nx_key_col[1]) : 0, st, ln);
            o.out_next[base + pos] = ln;
            nsum += (unsigned long long)ln;
          }
        }
        pos++;
      }
    }
    __syncthreads();
    int32_t *dst = o.out + base * wo;
    const int ne = Kc * wo;
    {  // element e = sidx * wo + q; (sidx, q) advance by (BLK / wo, BLK % wo) with carry
      int sidx = st_s0, q = st_q0;
      for (int e = tid; e < ne; e += BLK) {
        const int cd = S.code[q];
        dst[e] = cd < 0x100 ? tile[S.surv_r[sidx] * ws + cd]
                            : __ldg(mrows + (int64_t)S.surv_m[sidx] * mw + (cd & 0xff));
        sidx += st_ds;
        q += st_dq;
        if (q >= wo) {
          q -= wo;
          sidx++;
        }
      }
    }
    if (o.out_next) {
      unsigned long long tot = block_sum_u64<BLK>(nsum, s_red);
      if (tid == 0 && tot && o.next_ctr) atomicAdd(o.next_ctr, tot);
    }
    __syncthreads();
  }
  __syncthreads();  // the next tile overwrites the shared-memory tile
}

}  // namespace dmk
