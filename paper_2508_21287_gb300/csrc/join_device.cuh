// Device side of one join step of Alg. 1 (InnerJoin + FilterOverlappingNodes + back-edge test
// + score + compaction) on one tile of the intermediate table R. Shared by the per-step kernel
// (k_join, kernels.cu) and the persistent batch kernel (batch.cu).
//
// A block stages up to TR rows of R in shared memory (odd row stride: conflict-free column
// reads across rows; the per-step kernel prefetches the next tile with cp.async while it
// works on the current one), computes a 256-bit two-hash signature of each row's vertex ids,
// looks up each row's key group in the motif index, and scans the group sizes into a
// candidate range. The candidates are then processed in rounds of BLK * CPT: each thread
// first issues the motif-row loads of its CPT candidates, then checks them (extra key
// equalities, injectivity against the row -- a full scan only when both signature bits of a
// new vertex are set --, back-edges in the adjacency bitmap, FP32 score); survivors are
// compacted with a block scan, their output range is reserved once per round, and the block
// writes the rows element by element so that consecutive threads store consecutive words.
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

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------------ index lookup -------
__device__ __forceinline__ void ix_lookup(const IndexView &ix, int32_t ka, int32_t kb, int32_t &start,
                                          int32_t &len) {
  if (ix.nkeys == 1) {
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

// Two positions of a vertex id in the 256-bit row signature (independent multiplicative hashes).
__device__ __forceinline__ unsigned sig_h1(int32_t v) { return ((uint32_t)v * 0x9E3779B1u) >> 24; }
__device__ __forceinline__ unsigned sig_h2(int32_t v) { return ((uint32_t)v * 0x85EBCA77u) >> 24; }

struct JoinSmem {
  int32_t *tile_buf[2];  // R tiles (two for the prefetching per-step kernel)
  float *ts_buf[2];
  unsigned long long *sig;  // 4 words per row
  int32_t *gstart, *goff;
  int32_t *surv_r, *surv_m;
  int32_t *cand_row;
  int16_t *code;  // per output position: working column (< 0x100: from the R row) or 0x100 | motif position
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
  offs[4] = off;  // signatures
  off += (size_t)TR * 32;
  offs[5] = off;  // group starts, offsets
  off += (size_t)TR * 4 + (size_t)(TR + 1) * 4;
  off = (off + 15) / 16 * 16;
  offs[6] = off;  // survivors, candidate rows, codes
  off += (size_t)BLKCPT * 4 * 3 + (size_t)MAXW * 2;
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
  m.sig = (unsigned long long *)(smem + o[4]);
  m.gstart = (int32_t *)(smem + o[5]);
  m.goff = m.gstart + TR;
  m.surv_r = (int32_t *)(smem + o[6]);
  m.surv_m = m.surv_r + BLKCPT;
  m.cand_row = m.surv_m + BLKCPT;
  m.code = (int16_t *)(m.cand_row + BLKCPT);
  return m;
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }

// Copy nr rows (width w) from src into a shared tile of row stride ws, and their scores.
// ASYNC: with cp.async (the caller commits and waits); else with plain loads and stores.
template <int BLK, bool ASYNC>
__device__ __forceinline__ void load_tile(int32_t *tile, float *ts, const int32_t *src, const float *srcs, int nr,
                                          int w) {
  const int ws = w | 1;
  const int ne = nr * w;
  const int dr = BLK / w, dc = BLK % w;
  int r = threadIdx.x / w, c = threadIdx.x % w;  // element e = r * w + c, advanced with carry
  for (int e = threadIdx.x; e < ne; e += BLK) {
    if (ASYNC) cp_async4(tile + r * ws + c, src + e);
    else tile[r * ws + c] = __ldg(src + e);
    r += dr;
    c += dc;
    if (c >= w) {
      c -= w;
      r++;
    }
  }
  if (srcs)
    for (int i = threadIdx.x; i < nr; i += BLK) {
      if (ASYNC) cp_async4(ts + i, srcs + i);
      else ts[i] = __ldg(srcs + i);
    }
}

// Value of working column `col` of the joined row (R row `rrow`, motif row `trow`).
__device__ __forceinline__ int32_t join_value(const JoinArgs &a, const int32_t *rrow, const int32_t *trow, int col) {
  return col < a.w ? rrow[col] : __ldg(trow + a.new_mpos[col - a.w]);
}

// Join, filter and score one candidate (R row r of the tile, motif row m) whose new vertices
// nv were loaded beforehand.
template <int MAXNEW>
__device__ __forceinline__ bool join_check(const JoinArgs &a, const JoinSmem &S, const int32_t *tile, const float *ts,
                                           int ws, bool seed, int r, int m, const int32_t (&nv)[MAXNEW], float &sc) {
  const int32_t *rrow = tile + r * ws;
  const int32_t *trow = a.ix.rows + (int64_t)m * a.ix.mw;
  bool ok = true;
  for (int i = 0; i < a.n_chk; i++) ok &= __ldg(trow + a.chk_mpos[i]) == rrow[a.chk_col[i]];
  if (ok && !seed) {  // FilterOverlappingNodes: new vertices must not repeat a mapped one
    const unsigned long long *sg = S.sig + 4 * r;
#pragma unroll
    for (int i = 0; i < MAXNEW; i++) {
      if (i < a.n_new && ok) {
        const unsigned h1 = sig_h1(nv[i]), h2 = sig_h2(nv[i]);
        if (((sg[h1 >> 6] >> (h1 & 63)) & (sg[h2 >> 6] >> (h2 & 63)) & 1ull))
          for (int c = a.w - 1; c >= 0; c--)  // likely collisions are recent columns
            if (rrow[c] == nv[i]) {
              ok = false;
              break;
            }
      }
    }
  }
  sc = 0.f;
  if (a.scored) {
    sc = (!seed && a.Rs) ? ts[r] : 0.f;
    if (a.ix.score) sc += __ldg(a.ix.score + m);
    if (a.qerr) {
#pragma unroll
      for (int i = 0; i < MAXNEW; i++)
        if (i < a.n_new) sc += __ldg(a.qerr + nv[i]);
    }
  }
  for (int e = 0; e < a.n_be && ok; e++) {
    int32_t va = join_value(a, rrow, trow, a.be_a[e]);
    int32_t vb = join_value(a, rrow, trow, a.be_b[e]);
    ok = adjacent(a, va, vb);
    if (ok && a.scored && a.eerr) sc += edge_weight(a, va, vb);
  }
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
  const int ws = w > 0 ? (w | 1) : 1;
  const int tid = threadIdx.x;
  int32_t *tile = S.tile_buf[buf];
  float *ts = S.ts_buf[buf];
  // output position -> source, in shared memory: lanes look it up with different indices,
  // which the constant bank would serialise
  for (int q = tid; q < wo; q += BLK) {
    const int col = a.src_col[q];
    S.code[q] = (int16_t)(col < w ? col : (0x100 | a.new_mpos[col - w]));
  }
  int C;
  if (seed) __syncthreads();
  if (!seed) {
    if (!loaded) {
      load_tile<BLK, false>(tile, ts, src, srcs, nr, w);
      __syncthreads();
    }
    int len = 0, start = 0;
    if (tid < nr) {
      const int32_t *row = tile + tid * ws;
      unsigned long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int c = 0; c < w; c++) {
        const unsigned h1 = sig_h1(row[c]), h2 = sig_h2(row[c]);
        const unsigned long long b1 = 1ull << (h1 & 63), b2 = 1ull << (h2 & 63);
        s0 |= (h1 >> 6) == 0 ? b1 : 0ull;
        s1 |= (h1 >> 6) == 1 ? b1 : 0ull;
        s2 |= (h1 >> 6) == 2 ? b1 : 0ull;
        s3 |= (h1 >> 6) == 3 ? b1 : 0ull;
        s0 |= (h2 >> 6) == 0 ? b2 : 0ull;
        s1 |= (h2 >> 6) == 1 ? b2 : 0ull;
        s2 |= (h2 >> 6) == 2 ? b2 : 0ull;
        s3 |= (h2 >> 6) == 3 ? b2 : 0ull;
      }
      unsigned long long *sg = S.sig + 4 * tid;
      sg[0] = s0;
      sg[1] = s1;
      sg[2] = s2;
      sg[3] = s3;
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
#pragma unroll
      for (int i = 0; i < MAXNEW; i++)
        if (i < a.n_new) nv[k][i] = __ldg(trow + a.new_mpos[i]);
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
            const int32_t *rrow = tile + myr[k] * ws;
            const int32_t *trow = mrows + (int64_t)mym[k] * mw;
            unsigned long long h = dmix64((unsigned long long)(uint32_t)wo);
            for (int q = 0; q < wo; q++) {
              const int cd = S.code[q];
              const int32_t v = cd < 0x100 ? rrow[cd] : __ldg(trow + (cd & 0xff));
              h = dmix64(h ^ (unsigned long long)(uint32_t)v);
            }
            acc_sum += h;
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
