// Device side of one join step of Alg. 1 (InnerJoin + FilterOverlappingNodes + back-edge test
// + score + compaction) on one tile of the intermediate table R. Shared by the per-step kernel
// (k_join, kernels.cu) and the persistent batch kernel (batch.cu).
//
// A block stages up to TR rows of R in shared memory (odd row stride: conflict-free column
// reads across rows), computes a 128-bit signature of each row's vertex ids, looks up each
// row's key group in the motif index, and scans the group sizes into a candidate range. The
// candidates are then processed in rounds of BLK * CPT: each thread evaluates CPT candidates
// (extra key equalities, injectivity against the row via the signature, back-edges in the
// adjacency bitmap, FP32 score); survivors are compacted with a block scan, their output range
// is reserved once per round, and the block writes the rows element by element so that
// consecutive threads store consecutive words.
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

// 7-bit position of a vertex id in the 128-bit row signature.
__device__ __forceinline__ unsigned sig_bit(int32_t v) { return ((uint32_t)v * 0x9E3779B1u) >> 25; }

struct JoinSmem {
  int32_t *tile;
  unsigned long long *sig;
  float *tile_s;
  int32_t *gstart, *goff;
  int32_t *surv_r, *surv_m;
  int32_t *cand_row;
};

__device__ __forceinline__ JoinSmem join_smem(unsigned char *smem, int TR, int ws, int BLKCPT) {
  JoinSmem m;
  size_t off = 0;
  m.tile = (int32_t *)(smem + off);
  off += (size_t)TR * ws * 4;
  off = (off + 15) / 16 * 16;
  m.sig = (unsigned long long *)(smem + off);
  off += (size_t)TR * 16;
  m.tile_s = (float *)(smem + off);
  off += (size_t)TR * 4;
  m.gstart = (int32_t *)(smem + off);
  off += (size_t)TR * 4;
  m.goff = (int32_t *)(smem + off);
  off += (size_t)(TR + 1) * 4;
  off = (off + 15) / 16 * 16;
  m.surv_r = (int32_t *)(smem + off);
  m.surv_m = m.surv_r + BLKCPT;
  m.cand_row = m.surv_m + BLKCPT;
  return m;
}

// Value of working column `col` of the joined row (R row `rrow`, motif row `trow`).
__device__ __forceinline__ int32_t join_value(const JoinArgs &a, const int32_t *rrow, const int32_t *trow, int col) {
  return col < a.w ? rrow[col] : __ldg(trow + a.new_mpos[col - a.w]);
}

// Join, filter and score one candidate (R row r of the tile, motif row m).
template <int MAXNEW>
__device__ __forceinline__ bool join_eval(const JoinArgs &a, const JoinSmem &S, int ws, bool seed, int r, int64_t m,
                                          float &sc) {
  const int32_t *rrow = S.tile + r * ws;
  const int32_t *trow = a.ix.rows + m * a.ix.mw;
  bool ok = true;
  for (int i = 0; i < a.n_chk; i++) ok &= __ldg(trow + a.chk_mpos[i]) == rrow[a.chk_col[i]];
  int32_t nv[MAXNEW];
#pragma unroll
  for (int i = 0; i < MAXNEW; i++)
    if (i < a.n_new) nv[i] = __ldg(trow + a.new_mpos[i]);
  if (ok && !seed) {  // FilterOverlappingNodes: new vertices must not repeat a mapped one
    const unsigned long long s0 = S.sig[2 * r], s1 = S.sig[2 * r + 1];
#pragma unroll
    for (int i = 0; i < MAXNEW; i++) {
      if (i < a.n_new) {
        unsigned b = sig_bit(nv[i]);
        unsigned long long word = b < 64 ? s0 : s1;
        if ((word >> (b & 63)) & 1ull)  // likely collisions are recent columns: scan backwards
          for (int c = a.w - 1; c >= 0; c--)
            if (rrow[c] == nv[i]) {
              ok = false;
              break;
            }
      }
    }
  }
  sc = 0.f;
  if (a.scored) {
    sc = (!seed && a.Rs) ? S.tile_s[r] : 0.f;
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

// Process one tile: rows src[0 .. nr) of R (width a.w), or, in seed mode (src == nullptr),
// motif rows [seed_m0, seed_m0 + seed_C) as candidates. MODE 0 writes survivors through `o`;
// MODE 1 adds their count and checksum hashes to acc_rows / acc_sum (per thread).
template <int BLK, int MAXNEW, int CPT, int MODE>
__device__ __forceinline__ void join_tile(const JoinArgs &a, const JoinSmem &S, int TR, const int32_t *src,
                                          const float *srcs, int nr, int64_t seed_m0, int seed_C, const TileOut &o,
                                          int *s_warp, unsigned long long *s_red, long long *s_base,
                                          unsigned long long &acc_rows, unsigned long long &acc_sum,
                                          unsigned long long &acc_cand) {
  const bool seed = src == nullptr;
  const int w = a.w, wo = a.wo;
  const int ws = w > 0 ? (w | 1) : 1;
  const int tid = threadIdx.x;
  int C;
  if (!seed) {
    const int ne = nr * w;
    {  // element e = r * w + c of the tile; (r, c) advance by (BLK / w, BLK % w) with carry
      const int dr = BLK / w, dc = BLK % w;
      int r = tid / w, c = tid % w;
      for (int e = tid; e < ne; e += BLK) {
        S.tile[r * ws + c] = __ldg(src + e);
        r += dr;
        c += dc;
        if (c >= w) {
          c -= w;
          r++;
        }
      }
    }
    if (srcs)
      for (int r = tid; r < nr; r += BLK) S.tile_s[r] = __ldg(srcs + r);
    __syncthreads();
    int len = 0, start = 0;
    if (tid < nr) {
      const int32_t *row = S.tile + tid * ws;
      unsigned long long s0 = 0, s1 = 0;
      for (int c = 0; c < w; c++) {
        unsigned b = sig_bit(row[c]);
        if (b < 64) s0 |= 1ull << b;
        else s1 |= 1ull << (b - 64);
      }
      S.sig[2 * tid] = s0;
      S.sig[2 * tid + 1] = s1;
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
    int64_t mym[CPT];
    float mys[CPT];
    unsigned pass = 0;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      const int c = rb + k * BLK + tid;
      myr[k] = 0;
      mym[k] = 0;
      mys[k] = 0.f;
      if (c < C) {
        int r = 0;
        int64_t m;
        if (seed) {
          m = seed_m0 + c;
        } else {
          r = S.cand_row[c - rb];
          m = (int64_t)S.gstart[r] + (c - S.goff[r]);
        }
        float sc;
        if (join_eval<MAXNEW>(a, S, ws, seed, r, m, sc)) {
          pass |= 1u << k;
          myr[k] = r;
          mym[k] = m;
          mys[k] = sc;
          if (MODE == 1) {
            const int32_t *rrow = S.tile + r * ws;
            const int32_t *trow = a.ix.rows + m * a.ix.mw;
            unsigned long long h = dmix64((unsigned long long)(uint32_t)wo);
            for (int q = 0; q < wo; q++)
              h = dmix64(h ^ (unsigned long long)(uint32_t)join_value(a, rrow, trow, a.src_col[q]));
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
        S.surv_m[pos] = (int32_t)mym[k];
        if (pos < Kc) {
          if (o.outs) o.outs[base + pos] = mys[k];
          if (o.out_next) {
            const int32_t *rrow = S.tile + myr[k] * ws;
            const int32_t *trow = a.ix.rows + mym[k] * a.ix.mw;
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
        const int col = a.src_col[q];
        const int32_t *rrow = S.tile + S.surv_r[sidx] * ws;
        dst[e] = col < w ? rrow[col] : __ldg(a.ix.rows + (int64_t)S.surv_m[sidx] * a.ix.mw + a.new_mpos[col - w]);
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
