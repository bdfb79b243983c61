// sm_103a kernels of the Delta-Motif library.
//
// The hot kernel is k_join: one launch performs one iteration of Alg. 1 over a tile-
// partitioned intermediate table R (row-major, width w):
//   InnerJoin(R, Res(M), C)   - every R row looks up its key (the R columns that the slice
//                               shares with earlier slices, Sec. 3.2) in an index of the
//                               motif table: direct offsets for one key column, an
//                               open-addressing hash on the packed 64-bit key for two;
//   FilterOverlappingNodes    - a joined row survives only if the motif's new vertices are
//                               distinct from every vertex already in the row (Sec. 3.2:
//                               duplicates beyond the join constraints are invalid);
//   back-edge filter          - pattern edges between mapped vertices that no slice covers
//                               are tested in the data graph's adjacency bitmap;
//   score                     - FP32 layout score += motif-row edge errors + vertex errors
//                               of the new vertices + back-edge errors (Sec. 5.4);
//   compaction                - warp ballots + a block scan place survivors contiguously in
//                               shared memory; one atomic per block chunk reserves the output
//                               range, then the block writes it with coalesced stores.
// The R tile is staged in shared memory once; every candidate row of the tile reads it
// there. The same kernel also emits the candidate count of every written row for the next
// step, which sizes the next output and drives chunked streaming.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "kernels.h"

using namespace dmi;

namespace dmk {

std::atomic<int64_t> g_launches{0};
int64_t launch_count() { return g_launches.load(); }

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

// ------------------------------------------------------------------ join kernel --------
int join_tile_rows(int w) {
  if (w <= 0) return JOIN_BLK;
  int ws = w | 1;
  int tr = 32768 / (ws * 4);
  tr = tr / 32 * 32;
  if (tr < 32) tr = 32;
  if (tr > JOIN_BLK) tr = JOIN_BLK;
  return tr;
}

static int join_cpt(int n_new) { return n_new <= 4 ? 4 : 1; }

size_t join_smem_bytes(int w, int wo, int tile_rows) {
  (void)wo;
  int ws = w > 0 ? (w | 1) : 1;
  size_t b = (size_t)tile_rows * ws * 4;  // tile
  b = (b + 15) / 16 * 16;
  b += (size_t)tile_rows * 16;            // 128-bit vertex signature per row
  b += (size_t)tile_rows * 4;             // tile scores
  b += (size_t)tile_rows * 4;             // group starts
  b += (size_t)(tile_rows + 1) * 4;       // group offsets
  b = (b + 15) / 16 * 16;
  b += (size_t)JOIN_BLK * 4 * 8;          // survivor (row, motif row) pairs of one round
  b += (size_t)JOIN_BLK * 4 * 4;          // tile row of each candidate of one round
  return b;
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

template <int BLK, int MAXNEW, int CPT, int MODE>
__global__ void __launch_bounds__(BLK, 4) k_join(const __grid_constant__ JoinArgs a, int TR) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_warp[BLK / 32];
  __shared__ unsigned long long s_red[BLK / 32];
  __shared__ long long s_base;

  const bool seed = a.R == nullptr;
  const int w = a.w, wo = a.wo;
  const int ws = w > 0 ? (w | 1) : 1;
  const int tid = threadIdx.x;
  const JoinSmem S = join_smem(smem, TR, ws, BLK * CPT);
  const int64_t N = seed ? 0 : (a.n_dev ? imin64((int64_t)*a.n_dev, a.in_cap) : a.N);
  const int64_t nt = seed ? (a.seed_hi - a.seed_lo + (int64_t)BLK * CPT - 1) / ((int64_t)BLK * CPT)
                          : (N + TR - 1) / TR;
  const int ld_r0 = w > 0 ? tid / w : 0, ld_c0 = w > 0 ? tid % w : 0;
  const int ld_dr = w > 0 ? BLK / w : 0, ld_dc = w > 0 ? BLK % w : 0;
  const int st_s0 = tid / wo, st_q0 = tid % wo, st_ds = BLK / wo, st_dq = BLK % wo;

  unsigned long long acc_rows = 0, acc_sum = 0, acc_cand = 0;

  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    int C;
    if (!seed) {
      const int64_t r0 = t * TR;
      const int nr = (int)imin64(TR, N - r0);
      const int32_t *src = a.R + r0 * w;
      const int ne = nr * w;
      {  // element e = r * w + c of the tile; (r, c) advance by (BLK / w, BLK % w) with carry
        int r = ld_r0, c = ld_c0;
        for (int e = tid; e < ne; e += BLK) {
          S.tile[r * ws + c] = __ldg(src + e);
          r += ld_dr;
          c += ld_dc;
          if (c >= w) {
            c -= w;
            r++;
          }
        }
      }
      if (a.Rs)
        for (int r = tid; r < nr; r += BLK) S.tile_s[r] = __ldg(a.Rs + r0 + r);
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
      C = (int)imin64((int64_t)BLK * CPT, a.seed_hi - (a.seed_lo + t * BLK * CPT));
    }
    acc_cand += tid == 0 ? (unsigned long long)C : 0ull;

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
            m = a.seed_lo + t * BLK * CPT + c;
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
      // compaction: block scan of per-thread survivor counts, one atomic per round
      int K;
      const int pos0 = block_excl_scan<BLK>(__popc(pass), K, s_warp);
      if (K == 0) continue;
      if (tid == 0) s_base = (long long)atomicAdd(a.ctr + CTR_ROWS, (unsigned long long)K);
      __syncthreads();
      const long long base = s_base;
      int Kc = K;
      if (base + K > a.out_cap) {
        Kc = (int)imax64(0, a.out_cap - base);
        if (tid == 0) atomicOr(a.ctr + CTR_OVF, 1ull);
      }
      unsigned long long nsum = 0;
      int pos = pos0;
#pragma unroll
      for (int k = 0; k < CPT; k++) {
        if (pass >> k & 1u) {
          S.surv_r[pos] = myr[k];
          S.surv_m[pos] = (int32_t)mym[k];
          if (pos < Kc) {
            if (a.outs) a.outs[base + pos] = mys[k];
            if (a.out_next) {
              const int32_t *rrow = S.tile + myr[k] * ws;
              const int32_t *trow = a.ix.rows + mym[k] * a.ix.mw;
              int32_t st, ln;
              ix_lookup(a.nx, join_value(a, rrow, trow, a.nx_key_col[0]),
                        a.nx.nkeys == 2 ? join_value(a, rrow, trow, a.nx_key_col[1]) : 0, st, ln);
              a.out_next[base + pos] = ln;
              nsum += (unsigned long long)ln;
            }
          }
          pos++;
        }
      }
      __syncthreads();
      // coalesced materialisation: element e of the block's output range is row e / wo,
      // position e % wo (the float quotient is exact for e < 2^20)
      int32_t *dst = a.out + base * wo;
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
      if (a.out_next) {
        unsigned long long tot = block_sum_u64<BLK>(nsum, s_red);
        if (tid == 0 && tot) atomicAdd(a.ctr + CTR_NEXT, tot);
      }
      __syncthreads();
    }
    __syncthreads();  // the next tile overwrites the shared-memory tile
  }
  unsigned long long tc = block_sum_u64<BLK>(acc_cand, s_red);
  if (tid == 0 && tc) atomicAdd(a.ctr + CTR_CAND, tc);
  if (MODE == 1) {
    unsigned long long tr = block_sum_u64<BLK>(acc_rows, s_red);
    unsigned long long ts = block_sum_u64<BLK>(acc_sum, s_red);
    if (tid == 0) {
      if (tr) atomicAdd(a.ctr + CTR_ROWS, tr);
      atomicAdd(a.ctr + CTR_SUM, ts);
    }
  }
}

typedef void (*JoinKernel)(JoinArgs, int);

static JoinKernel pick_join(const JoinArgs &a, int *cpt) {
  *cpt = join_cpt(a.n_new);
  if (a.mode == 1) {
    if (a.n_new <= 1) return k_join<JOIN_BLK, 1, 4, 1>;
    if (a.n_new <= 4) return k_join<JOIN_BLK, 4, 4, 1>;
    return k_join<JOIN_BLK, MAXM, 1, 1>;
  }
  if (a.n_new <= 1) return k_join<JOIN_BLK, 1, 4, 0>;
  if (a.n_new <= 4) return k_join<JOIN_BLK, 4, 4, 0>;
  return k_join<JOIN_BLK, MAXM, 1, 0>;
}

static void set_join_attrs() {
  static bool done = false;
  if (done) return;
  JoinKernel ks[] = {k_join<JOIN_BLK, 1, 4, 1>, k_join<JOIN_BLK, 4, 4, 1>, k_join<JOIN_BLK, MAXM, 1, 1>,
                     k_join<JOIN_BLK, 1, 4, 0>, k_join<JOIN_BLK, 4, 4, 0>, k_join<JOIN_BLK, MAXM, 1, 0>};
  for (auto k : ks) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  done = true;
}

cudaError_t launch_join(const JoinArgs &a, int grid, int tile_rows, cudaStream_t s) {
  set_join_attrs();
  int cpt;
  JoinKernel k = pick_join(a, &cpt);
  size_t smem = join_smem_bytes(a.w, a.wo, tile_rows);
  if (grid < 1) grid = 1;
  g_launches++;
  k<<<grid, JOIN_BLK, smem, s>>>(a, tile_rows);
  return cudaGetLastError();
}

int join_grid(const JoinArgs &a, int tile_rows, int num_sms) {
  set_join_attrs();
  int cpt;
  JoinKernel k = pick_join(a, &cpt);
  int64_t nt;
  if (a.R == nullptr) nt = (a.seed_hi - a.seed_lo + (int64_t)JOIN_BLK * cpt - 1) / ((int64_t)JOIN_BLK * cpt);
  else if (a.n_dev) nt = INT64_MAX;  // row count known only on the device: fill the GPU
  else nt = (a.N + tile_rows - 1) / tile_rows;
  size_t smem = join_smem_bytes(a.w, a.wo, tile_rows);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, JOIN_BLK, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t g = (int64_t)num_sms * per_sm;
  if (nt < g) g = nt;
  return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------------ graph prep ---------
__device__ __forceinline__ int32_t slot_source(const int32_t *row_ptr, int32_t V, int64_t e) {
  int32_t lo = 0, hi = V;  // largest u with row_ptr[u] <= e
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_csr_to_m2(const int32_t *row_ptr, const int32_t *col_idx, const float *eerr, int32_t V,
                            int64_t nnz, int32_t *rows, float *score) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    rows[2 * e] = slot_source(row_ptr, V, e);
    rows[2 * e + 1] = __ldg(col_idx + e);
    if (score) score[e] = eerr ? __ldg(eerr + e) : 0.f;
  }
}

cudaError_t launch_csr_to_m2(const int32_t *row_ptr, const int32_t *col_idx, const float *eerr, int32_t V,
                             int64_t nnz, int32_t *rows, float *score, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  int grid = (int)imin64((nnz + 255) / 256, 4096);
  g_launches++;
  k_csr_to_m2<<<grid, 256, 0, s>>>(row_ptr, col_idx, eerr, V, nnz, rows, score);
  return cudaGetLastError();
}

__global__ void k_vertex_table(int32_t V, int32_t *rows, float *score) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    rows[v] = v;
    if (score) score[v] = 0.f;
  }
}

cudaError_t launch_vertex_table(int32_t V, int32_t *rows, float *score, cudaStream_t s) {
  if (V == 0) return cudaSuccess;
  g_launches++;
  k_vertex_table<<<(V + 255) / 256, 256, 0, s>>>(V, rows, score);
  return cudaGetLastError();
}

__global__ void k_bitmap(const int32_t *row_ptr, const int32_t *col_idx, int32_t V, int64_t nnz, int32_t words,
                         unsigned long long *adj) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = slot_source(row_ptr, V, e), v = __ldg(col_idx + e);
    atomicOr(adj + (int64_t)u * words + (v >> 6), 1ull << (v & 63));
  }
}

cudaError_t launch_bitmap(const int32_t *row_ptr, const int32_t *col_idx, int32_t V, int64_t nnz, int32_t words,
                          unsigned long long *adj, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  int grid = (int)imin64((nnz + 255) / 256, 4096);
  g_launches++;
  k_bitmap<<<grid, 256, 0, s>>>(row_ptr, col_idx, V, nnz, words, adj);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ scan ---------------
constexpr int SCAN_BLK = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_BLK * SCAN_ITEMS;

template <class T>
__global__ void __launch_bounds__(SCAN_BLK) k_scan_tile(const T *in, int64_t *out, int64_t n, int64_t *sums) {
  __shared__ long long s_w[SCAN_BLK / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)tid * SCAN_ITEMS;
  long long v[SCAN_ITEMS];
  long long tsum = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    int64_t i = base + j;
    v[j] = i < n ? (long long)in[i] : 0;
    tsum += v[j];
  }
  long long x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(FULL_MASK, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long wv = lane < SCAN_BLK / 32 ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(FULL_MASK, wv, o);
      if (lane >= o) wv += t;
    }
    if (lane < SCAN_BLK / 32) s_w[lane] = wv;
  }
  __syncthreads();
  long long run = (warp ? s_w[warp - 1] : 0) + x - tsum;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    int64_t i = base + j;
    if (i < n) out[i] = run;
    run += v[j];
  }
  if (tid == SCAN_BLK - 1) {
    long long total = s_w[SCAN_BLK / 32 - 1];
    if (sums) sums[blockIdx.x] = total;
    else out[n] = total;
  }
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *sums_scan, int64_t nb) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const long long add = sums_scan[blockIdx.x];
  for (int j = threadIdx.x; j < SCAN_TILE; j += blockDim.x) {
    int64_t i = base + j;
    if (i < n) out[i] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums_scan[nb];
}

int64_t scan_tmp_elems(int64_t n) {
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= 1) return 1;
  return 2 * nb + 1 + scan_tmp_elems(nb);
}

template <class T>
static cudaError_t scan_impl(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    g_launches++;
    k_scan_tile<T><<<1, SCAN_BLK, 0, s>>>(in, out, n, nullptr);
    return cudaGetLastError();
  }
  int64_t *sums = tmp, *sums_scan = tmp + nb, *rest = tmp + 2 * nb + 1;
  g_launches++;
  k_scan_tile<T><<<(unsigned)nb, SCAN_BLK, 0, s>>>(in, out, n, sums);
  cudaError_t e = scan_impl<int64_t>(sums, sums_scan, nb, rest, s);
  if (e != cudaSuccess) return e;
  g_launches++;
  k_scan_add<<<(unsigned)nb, SCAN_BLK, 0, s>>>(out, n, sums_scan, nb);
  return cudaGetLastError();
}

cudaError_t scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, tmp, s);
}
cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, tmp, s);
}

// ------------------------------------------------------------------ radix sort ---------
constexpr int RS_BLK = 256, RS_ITEMS = 8, RS_TILE = RS_BLK * RS_ITEMS;

int64_t radix_hist_elems(int64_t n) { return 256 * ((n + RS_TILE - 1) / RS_TILE); }

__global__ void __launch_bounds__(RS_BLK) k_radix_hist(const uint32_t *keys, int64_t stride, const int32_t *perm,
                                                       int64_t n, int shift, int64_t *hist, int nb) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; j++) {
    int64_t i = base + j * RS_BLK + threadIdx.x;
    if (i < n) {
      int64_t src = perm ? (int64_t)perm[i] : i;
      uint32_t k = __ldg(keys + src * stride);
      atomicAdd(&h[(k >> shift) & 255u], 1);
    }
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_BLK) k_radix_scatter(const uint32_t *keys, int64_t stride,
                                                          const int32_t *perm_in, int64_t n, int shift,
                                                          const int64_t *off, int nb, int32_t *perm_out) {
  __shared__ int wcnt[RS_BLK / 32][256];
  __shared__ int run[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = 0;
  for (int w = 0; w < RS_BLK / 32; w++) wcnt[w][tid] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int j = 0; j < RS_ITEMS; j++) {
    int64_t i = base + j * RS_BLK + tid;
    bool valid = i < n;
    int32_t p = 0;
    unsigned d = 256;
    if (valid) {
      p = perm_in ? perm_in[i] : (int32_t)i;
      d = (__ldg(keys + (int64_t)p * stride) >> shift) & 255u;
    }
    unsigned peers = __match_any_sync(FULL_MASK, d);
    int rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pre = run[d];
      for (int w = 0; w < warp; w++) pre += wcnt[w][d];
      perm_out[off[(int64_t)d * nb + blockIdx.x] + pre + rank] = p;
    }
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < RS_BLK / 32; w++) {
      tot += wcnt[w][tid];
      wcnt[w][tid] = 0;
    }
    run[tid] += tot;
    __syncthreads();
  }
}

cudaError_t radix_pass(const uint32_t *keys, int64_t stride, const int32_t *perm_in, int32_t *perm_out,
                       int64_t n, int shift, int64_t *hist, int64_t *hist_scan, int64_t *tmp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  g_launches++;
  k_radix_hist<<<nb, RS_BLK, 0, s>>>(keys, stride, perm_in, n, shift, hist, nb);
  cudaError_t e = scan_i64(hist, hist_scan, (int64_t)256 * nb, tmp, s);
  if (e != cudaSuccess) return e;
  g_launches++;
  k_radix_scatter<<<nb, RS_BLK, 0, s>>>(keys, stride, perm_in, n, shift, hist_scan, nb, perm_out);
  return cudaGetLastError();
}

__global__ void k_iota(int32_t *p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

cudaError_t launch_iota(int32_t *p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_iota<<<(int)imin64((n + 255) / 256, 8192), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

__global__ void k_gather_rows(const int32_t *in, const float *ins, const int32_t *perm, int64_t n, int32_t w,
                              int32_t *out, float *outs) {
  const int64_t ne = n * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / w;
    int32_t c = (int32_t)(e - i * w);
    int64_t src = perm[i];
    out[e] = __ldg(in + src * w + c);
    if (c == 0 && outs) outs[i] = __ldg(ins + src);
  }
}

cudaError_t launch_gather_rows(const int32_t *in, const float *ins, const int32_t *perm, int64_t n, int32_t w,
                               int32_t *out, float *outs, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t ne = n * w;
  g_launches++;
  k_gather_rows<<<(int)imin64((ne + 255) / 256, 16384), 256, 0, s>>>(in, ins, perm, n, w, out, outs);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ indices ------------
__global__ void k_offsets_direct(const int32_t *rows, int32_t mw, int32_t kpos, int64_t n, int32_t V,
                                 int32_t *offsets) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= V; v += gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = n;  // first i with key >= v
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (__ldg(rows + mid * mw + kpos) < v) lo = mid + 1;
      else hi = mid;
    }
    offsets[v] = (int32_t)lo;
  }
}

cudaError_t launch_offsets_direct(const int32_t *rows, int32_t mw, int32_t kpos, int64_t n, int32_t V,
                                  int32_t *offsets, cudaStream_t s) {
  g_launches++;
  k_offsets_direct<<<(V + 256) / 256, 256, 0, s>>>(rows, mw, kpos, n, V, offsets);
  return cudaGetLastError();
}

__global__ void k_hash_build(const int32_t *rows, int32_t mw, int32_t kp0, int32_t kp1, int64_t n,
                             HashSlot *slots, uint32_t log2cap, unsigned long long *ctr) {
  const unsigned long long mask = (1ull << log2cap) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    auto key_at = [&](int64_t j) {
      return ((unsigned long long)(uint32_t)__ldg(rows + j * mw + kp0) << 32) | (uint32_t)__ldg(rows + j * mw + kp1);
    };
    unsigned long long key = key_at(i);
    if (i > 0 && key_at(i - 1) == key) continue;
    int64_t len = 1;
    while (i + len < n && key_at(i + len) == key) len++;
    unsigned long long h = (key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap);
    for (unsigned long long probe = 0; probe <= mask; probe++) {
      unsigned long long prev = atomicCAS(&slots[h].key, HASH_EMPTY, key);
      if (prev == HASH_EMPTY) {
        slots[h].start = (int32_t)i;
        slots[h].len = (int32_t)len;
        break;
      }
      h = (h + 1) & mask;
    }
    atomicAdd(ctr + 0, 1ull);
    atomicMax(ctr + 1, (unsigned long long)len);
  }
}

cudaError_t launch_hash_build(const int32_t *rows, int32_t mw, int32_t kp0, int32_t kp1, int64_t n,
                              HashSlot *slots, uint32_t log2cap, unsigned long long *ctr, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_hash_build<<<(int)imin64((n + 255) / 256, 8192), 256, 0, s>>>(rows, mw, kp0, kp1, n, slots, log2cap, ctr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ top-k select -------
__global__ void k_score_hist(const float *sc, int64_t n, uint32_t prefix, uint32_t pmask, int shift,
                             unsigned long long *hist) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = __float_as_uint(__ldg(sc + i));
    if ((b & pmask) == prefix) atomicAdd(&h[(b >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

cudaError_t launch_score_hist(const float *sc, int64_t n, uint32_t prefix, uint32_t pmask, int shift,
                              unsigned long long *hist, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_score_hist<<<(int)imin64((n + 255) / 256, 2048), 256, 0, s>>>(sc, n, prefix, pmask, shift, hist);
  return cudaGetLastError();
}

__global__ void k_select_le(const float *sc, int64_t n, uint32_t T, int32_t *out_idx, unsigned long long *ctr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = __float_as_uint(__ldg(sc + i));
    if (b <= T) out_idx[atomicAdd(ctr, 1ull)] = (int32_t)i;
  }
}

cudaError_t launch_select_le(const float *sc, int64_t n, uint32_t T, int32_t *out_idx, unsigned long long *ctr,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_select_le<<<(int)imin64((n + 255) / 256, 4096), 256, 0, s>>>(sc, n, T, out_idx, ctr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ checksum -----------
__global__ void k_hash_rows(const int32_t *rows, int64_t n, int32_t w, unsigned long long *ctr) {
  __shared__ unsigned long long s_red[8];
  unsigned long long hs = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *row = rows + i * w;
    unsigned long long h = dmix64((unsigned long long)(uint32_t)w);
    for (int c = 0; c < w; c++) h = dmix64(h ^ (unsigned long long)(uint32_t)__ldg(row + c));
    hs += h;
  }
  unsigned long long t = block_sum_u64<256>(hs, s_red);
  if (threadIdx.x == 0 && t) atomicAdd(ctr + CTR_SUM, t);
}

cudaError_t launch_hash_rows(const int32_t *rows, int64_t n, int32_t w, unsigned long long *ctr, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_hash_rows<<<(int)imin64((n + 255) / 256, 2048), 256, 0, s>>>(rows, n, w, ctr);
  return cudaGetLastError();
}

}  // namespace dmk
