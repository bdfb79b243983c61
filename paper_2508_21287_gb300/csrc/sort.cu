// Canonical (lexicographic) order of embedding rows, and top-k by (score, row).
//
// Rows are sorted by comparison on packed keys: every row's ids are packed, bits(V) bits each
// and most significant first, into up to MS_KW 64-bit words (floor(64 / bits) ids per word).
// When the whole row fits (w * bits <= MS_KW * 64 in practice) the key is exact and every
// comparison stays in registers and shared memory; otherwise ties on the packed prefix fall
// back to the remaining columns of the rows themselves. Tiles of 1024 rows are sorted by a
// bitonic network in shared memory; runs are then merged pairwise, each element finding its
// output position by a binary search in the other run (stable: ties keep run order). A sort
// of N rows takes 2 + ceil(log2(N / 1024)) launches; tables of up to 16 tiles instead place
// every row at its final position in one rank-scatter launch (msort_rows_into). The
// key-packing kernel can also add the rows' checksum hashes (the same H as the join's count
// mode) into a counter, so that delivering a table needs no separate hashing pass.
//
// Top-k runs on a canonically sorted table: the key of row i is (score_key(score), i), where
// score_key maps an FP32 score to an unsigned key that orders like its value (either sign),
// and i orders like the row.
// Each block sorts a tile of keys and keeps its k smallest; the candidates shrink by that
// factor per pass until one tile holds them all.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "join_device.cuh"
#include "kernels.h"

namespace dmk {

constexpr int MS_TILE = 1024;
constexpr int MS_BLK = 512;
constexpr int MS_KW = 4;
constexpr unsigned long long KEY_INF = ~0ull;

struct SortKeys {
  const int32_t *rows;
  int32_t w;
  int packed;  // columns held in the key words; ties beyond them read the rows
};

// a < b for rows with packed keys ka / kb and indices ia / ib; an index < 0 is a padding
// element greater than every row.
template <int KW>
__device__ __forceinline__ bool row_less(const SortKeys &S, const unsigned long long (&ka)[KW], int32_t ia,
                                         const unsigned long long (&kb)[KW], int32_t ib) {
#pragma unroll
  for (int j = 0; j < KW; j++)
    if (ka[j] != kb[j]) return ka[j] < kb[j];
  if (ia < 0 || ib < 0) return ib < 0 && ia >= 0;
  if (S.packed < S.w) {
    const int32_t *ra = S.rows + (int64_t)ia * S.w, *rb = S.rows + (int64_t)ib * S.w;
    for (int c = S.packed; c < S.w; c++) {
      int32_t x = __ldg(ra + c), y = __ldg(rb + c);
      if (x != y) return x < y;
    }
  }
  return ia < ib;
}

// key[j * n + i]: word j of row i's packed key (structure of arrays: coalesced per word).
template <int KW>
__global__ void k_pack_keys(const int32_t *rows, int64_t n, int32_t w, int bits, int cpw,
                            unsigned long long *key, int32_t *idx, unsigned long long *sum) {
  __shared__ unsigned long long s_red[8];
  griddep_wait();
  griddep_launch_dependents();
  unsigned long long hs = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *r = rows + i * w;
    unsigned long long p = 0;
#pragma unroll
    for (int j = 0; j < KW; j++) {
      unsigned long long k = 0;
      for (int c = 0; c < cpw; c++) {
        const int col = j * cpw + c;
        unsigned long long v = 0;
        if (col < w) {
          const int32_t x = __ldg(r + col);
          v = (uint32_t)x;
          if (sum) p += col_term(col, x);
        }
        k |= v << (64 - bits * (c + 1));
      }
      key[(int64_t)j * n + i] = k;
    }
    if (sum) {
      for (int col = KW * cpw; col < w; col++) p += col_term(col, __ldg(r + col));
      hs += dmix64(p + (unsigned long long)(uint32_t)w);
    }
    idx[i] = (int32_t)i;
  }
  if (sum) {
    unsigned long long t = block_sum_u64<256>(hs, s_red);
    if (threadIdx.x == 0 && t) atomicAdd(sum, t);
  }
}

template <int KW>
__global__ void __launch_bounds__(MS_BLK) k_sort_tiles(const SortKeys S, int64_t n, unsigned long long *key,
                                                       int32_t *idx) {
  __shared__ unsigned long long sk[KW][MS_TILE];
  __shared__ int32_t si[MS_TILE];
  griddep_wait();
  griddep_launch_dependents();
  const int64_t base = (int64_t)blockIdx.x * MS_TILE;
  for (int i = threadIdx.x; i < MS_TILE; i += MS_BLK) {
    int64_t g = base + i;
#pragma unroll
    for (int j = 0; j < KW; j++) sk[j][i] = g < n ? key[(int64_t)j * n + g] : KEY_INF;
    si[i] = g < n ? idx[g] : -1;
  }
  __syncthreads();
  for (int k = 2; k <= MS_TILE; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < MS_TILE / 2; t += MS_BLK) {
        int i = 2 * t - (t & (j - 1));
        int p = i + j;
        bool up = (i & k) == 0;
        unsigned long long ki[KW], kp[KW];
#pragma unroll
        for (int q = 0; q < KW; q++) {
          ki[q] = sk[q][i];
          kp[q] = sk[q][p];
        }
        const int32_t ii = si[i], ip = si[p];
        if (row_less<KW>(S, kp, ip, ki, ii) == up) {
#pragma unroll
          for (int q = 0; q < KW; q++) {
            sk[q][i] = kp[q];
            sk[q][p] = ki[q];
          }
          si[i] = ip;
          si[p] = ii;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < MS_TILE; i += MS_BLK) {
    int64_t g = base + i;
    if (g < n) {
#pragma unroll
      for (int j = 0; j < KW; j++) key[(int64_t)j * n + g] = sk[j][i];
      idx[g] = si[i];
    }
  }
}

// Merge the sorted runs [b, b+L) and [b+L, b+2L) of (key, idx) into (okey, oidx).
template <int KW>
__global__ void k_merge_pass(const SortKeys S, int64_t n, int64_t L, const unsigned long long *key,
                             const int32_t *idx, unsigned long long *okey, int32_t *oidx) {
  griddep_wait();
  griddep_launch_dependents();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pair = i / (2 * L);
    const int64_t b = pair * 2 * L;
    const bool inA = i < b + L;
    const int64_t ob = inA ? b + L : b;                 // the other run
    const int64_t oe = inA ? (b + 2 * L < n ? b + 2 * L : n) : b + L;
    unsigned long long kx[KW];
#pragma unroll
    for (int j = 0; j < KW; j++) kx[j] = key[(int64_t)j * n + i];
    const int32_t ix = idx[i];
    int64_t lo = ob, hi = oe > ob ? oe : ob;
    // A elements go before equal B elements: count B < x for A, A <= x for B
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      unsigned long long km[KW];
#pragma unroll
      for (int j = 0; j < KW; j++) km[j] = key[(int64_t)j * n + mid];
      const int32_t im = idx[mid];
      bool before = inA ? row_less<KW>(S, km, im, kx, ix) : !row_less<KW>(S, kx, ix, km, im);
      if (before) lo = mid + 1;
      else hi = mid;
    }
    const int64_t pos = b + (i - (inA ? b : b + L)) + (lo - ob);
#pragma unroll
    for (int j = 0; j < KW; j++) okey[(int64_t)j * n + pos] = kx[j];
    oidx[pos] = ix;
  }
}

// Up to RS_LANES tiles: instead of merge passes and a gather, one launch gives every element
// of the tile-sorted (key, idx) arrays its final position, its rank in its own tile plus, for
// each other tile, the number of that tile's elements before it (a lower bound by binary
// search, one lane of a 16-lane group per tile), and copies its row (and score) there. The
// order is the same strict order as the tile sort's (key, remaining columns, index), so the
// positions are a permutation.
constexpr int RS_LANES = 16;

template <int KW>
__device__ __forceinline__ void rank_scatter_one(const SortKeys &S, int64_t n, const unsigned long long *key,
                                                 const int32_t *idx, const float *ins, int32_t *out, float *outs,
                                                 int64_t e) {
  const int l = threadIdx.x % RS_LANES;
  const unsigned seg = 0xFFFFu << (threadIdx.x & 16);
  const int t = (int)(e / MS_TILE);
  const int ntiles = (int)((n + MS_TILE - 1) / MS_TILE);
  unsigned long long kx[KW];
#pragma unroll
  for (int j = 0; j < KW; j++) kx[j] = key[(int64_t)j * n + e];
  const int32_t ix = idx[e];
  int64_t cnt = 0;
  if (l < ntiles && l != t) {
    const int64_t b = (int64_t)l * MS_TILE;
    int64_t lo = b, hi = b + MS_TILE < n ? b + MS_TILE : n;
    while (lo < hi) {  // first element of tile l not before x
      const int64_t mid = (lo + hi) >> 1;
      unsigned long long km[KW];
#pragma unroll
      for (int j = 0; j < KW; j++) km[j] = key[(int64_t)j * n + mid];
      if (row_less<KW>(S, km, idx[mid], kx, ix)) lo = mid + 1;
      else hi = mid;
    }
    cnt = lo - b;
  }
#pragma unroll
  for (int o = RS_LANES / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(seg, cnt, o, RS_LANES);
  const int64_t pos = (e - (int64_t)t * MS_TILE) + cnt;
  if (pos >= n) return;  // cannot happen for sorted tiles; no write outside the table regardless
  const int32_t *src = S.rows + (int64_t)ix * S.w;
  for (int c = l; c < S.w; c += RS_LANES) out[pos * S.w + c] = __ldg(src + c);
  if (l == 0 && outs) outs[pos] = __ldg(ins + ix);
}

template <int KW>
__global__ void k_rank_scatter(const SortKeys S, int64_t n, const unsigned long long *key, const int32_t *idx,
                               const float *ins, int32_t *out, float *outs) {
  griddep_wait();
  griddep_launch_dependents();
  const int64_t groups = (int64_t)gridDim.x * blockDim.x / RS_LANES;
  for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / RS_LANES; e < n; e += groups)
    rank_scatter_one<KW>(S, n, key, idx, ins, out, outs, e);  // a 16-lane group shares e: it loops together
}


int64_t msort_tmp_bytes(int64_t n) { return n * (8 * MS_KW + 4) * 2 + 256; }
int64_t msort_into_max_rows() { return (int64_t)RS_LANES * MS_TILE; }

template <int KW>
static void msort_into_launch(const SortKeys &S, int64_t n, int bits, int cpw, unsigned long long *k0, int32_t *i0,
                              const float *ins, int32_t *out, float *outs, unsigned long long *sum, int max_blocks,
                              cudaStream_t s) {
  int grid = (int)((n + 255) / 256);
  k_pack_keys<KW><<<grid, 256, 0, s>>>(S.rows, n, S.w, bits, cpw, k0, i0, sum);
  launch_pdl(k_sort_tiles<KW>, dim3((unsigned)((n + MS_TILE - 1) / MS_TILE)), dim3(MS_BLK), 0, s, S, n, k0, i0);
  int64_t rs_grid = (n * RS_LANES + 255) / 256;
  if (rs_grid > max_blocks) rs_grid = max_blocks;
  launch_pdl(k_rank_scatter<KW>, dim3((unsigned)rs_grid), dim3(256), 0, s, S, n, (const unsigned long long *)k0,
             (const int32_t *)i0, ins, out, outs);
}

cudaError_t msort_rows_into(const int32_t *rows, const float *scores, int64_t n, int32_t w, int bits, void *tmp,
                            int32_t *out_rows, float *out_scores, unsigned long long *sum, int max_blocks,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (max_blocks < 1) max_blocks = 1;
  if (n > msort_into_max_rows()) return cudaErrorInvalidValue;
  if (bits < 1) bits = 1;
  if (bits > 32) bits = 32;
  const int cpw = 64 / bits;
  int kw = (w + cpw - 1) / cpw;
  if (kw < 1) kw = 1;
  if (kw > MS_KW) kw = MS_KW;
  SortKeys S;
  S.rows = rows;
  S.w = w;
  S.packed = kw * cpw < w ? kw * cpw : w;
  unsigned long long *k0 = (unsigned long long *)tmp;
  int32_t *i0 = (int32_t *)(k0 + (int64_t)kw * n);
  switch (kw) {
    case 1: msort_into_launch<1>(S, n, bits, cpw, k0, i0, scores, out_rows, out_scores, sum, max_blocks, s); break;
    case 2: msort_into_launch<2>(S, n, bits, cpw, k0, i0, scores, out_rows, out_scores, sum, max_blocks, s); break;
    case 3: msort_into_launch<3>(S, n, bits, cpw, k0, i0, scores, out_rows, out_scores, sum, max_blocks, s); break;
    default: msort_into_launch<4>(S, n, bits, cpw, k0, i0, scores, out_rows, out_scores, sum, max_blocks, s); break;
  }
  g_launches += 3;
  return cudaGetLastError();
}

template <int KW>
static int msort_launch(const SortKeys &S, int64_t n, int bits, int cpw, unsigned long long *k0,
                        unsigned long long *k1, int32_t *i0, int32_t *i1, unsigned long long *sum, int32_t **perm_out,
                        cudaStream_t s) {
  int grid = (int)((n + 255) / 256);
  if (grid > 16384) grid = 16384;
  k_pack_keys<KW><<<grid, 256, 0, s>>>(S.rows, n, S.w, bits, cpw, k0, i0, sum);
  // the sort chain is kernel to kernel: each waits for its predecessor in its prologue
  launch_pdl(k_sort_tiles<KW>, dim3((unsigned)((n + MS_TILE - 1) / MS_TILE)), dim3(MS_BLK), 0, s, S, n, k0, i0);
  int launches = 2;
  for (int64_t L = MS_TILE; L < n; L *= 2) {
    launch_pdl(k_merge_pass<KW>, dim3(grid), dim3(256), 0, s, S, n, L, (const unsigned long long *)k0,
               (const int32_t *)i0, k1, i1);
    launches++;
    std::swap(k0, k1);
    std::swap(i0, i1);
  }
  *perm_out = i0;
  return launches;
}

cudaError_t msort_rows(const int32_t *rows, int64_t n, int32_t w, int bits, void *tmp, int32_t **perm_out,
                       unsigned long long *sum, cudaStream_t s) {
  if (n <= 0) {
    *perm_out = (int32_t *)tmp;
    return cudaSuccess;
  }
  if (bits < 1) bits = 1;
  if (bits > 32) bits = 32;
  const int cpw = 64 / bits;
  int kw = (w + cpw - 1) / cpw;
  if (kw < 1) kw = 1;
  if (kw > MS_KW) kw = MS_KW;
  SortKeys S;
  S.rows = rows;
  S.w = w;
  S.packed = kw * cpw < w ? kw * cpw : w;
  unsigned long long *k0 = (unsigned long long *)tmp;
  unsigned long long *k1 = k0 + (int64_t)kw * n;
  int32_t *i0 = (int32_t *)(k1 + (int64_t)kw * n);
  int32_t *i1 = i0 + n;
  int launches;
  switch (kw) {
    case 1: launches = msort_launch<1>(S, n, bits, cpw, k0, k1, i0, i1, sum, perm_out, s); break;
    case 2: launches = msort_launch<2>(S, n, bits, cpw, k0, k1, i0, i1, sum, perm_out, s); break;
    case 3: launches = msort_launch<3>(S, n, bits, cpw, k0, k1, i0, i1, sum, perm_out, s); break;
    default: launches = msort_launch<4>(S, n, bits, cpw, k0, k1, i0, i1, sum, perm_out, s); break;
  }
  g_launches += launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ images (dedup) -----
// Sort the ids inside every row (the row becomes its vertex set), one thread per row.
__global__ void k_sort_within_rows(int32_t *rows, int64_t n, int32_t w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t *r = rows + i * w;
    for (int a = 1; a < w; a++) {  // insertion sort: rows are at most 128 ids
      int32_t x = r[a];
      int b = a - 1;
      while (b >= 0 && r[b] > x) {
        r[b + 1] = r[b];
        b--;
      }
      r[b + 1] = x;
    }
  }
}

// flag[i] = 1 when sorted row i differs from row i - 1 (first of its run).
__global__ void k_first_of_run(const int32_t *rows, int64_t n, int32_t w, int32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int f = i == 0;
    if (!f) {
      const int32_t *a = rows + i * w, *b = a - w;
      for (int c = 0; c < w && !f; c++) f = a[c] != b[c];
    }
    flag[i] = f;
  }
}

// Copy the flagged rows to their scanned positions (order kept).
__global__ void k_compact_rows(const int32_t *rows, int64_t n, int32_t w, const int32_t *flag, const int64_t *pos,
                               int32_t *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * w; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / w;
    if (flag[i]) out[pos[i] * w + (e - i * w)] = rows[e];
  }
}

cudaError_t images_prepare(int32_t *rows, int64_t n, int32_t w, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256 > 16384 ? 16384 : (n + 255) / 256);
  g_launches++;
  k_sort_within_rows<<<grid, 256, 0, s>>>(rows, n, w);
  return cudaGetLastError();
}

cudaError_t unique_rows(const int32_t *rows, int64_t n, int32_t w, int32_t *flag, int64_t *pos, int64_t *tmp,
                        int32_t *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256 > 16384 ? 16384 : (n + 255) / 256);
  k_first_of_run<<<grid, 256, 0, s>>>(rows, n, w, flag);
  cudaError_t e = scan_i32(flag, pos, n, tmp, s);
  if (e != cudaSuccess) return e;
  int64_t ne = n * w;
  int g2 = (int)((ne + 255) / 256 > 16384 ? 16384 : (ne + 255) / 256);
  k_compact_rows<<<g2, 256, 0, s>>>(rows, n, w, flag, pos, out);
  g_launches += 2;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ top-k --------------
constexpr int TK_BLK = 512;
constexpr int TK_TILE = 2048;

__global__ void k_topk_keys_from_scores(const float *sc, int64_t n, unsigned long long *key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    key[i] = ((unsigned long long)score_key(__ldg(sc + i)) << 32) | (uint32_t)i;
}

// Each block sorts TK_TILE keys and writes its k smallest (k <= TK_TILE).
__global__ void __launch_bounds__(TK_BLK) k_topk_tiles(const unsigned long long *in, int64_t n, int32_t k,
                                                       unsigned long long *out) {
  __shared__ unsigned long long sk[TK_TILE];
  griddep_wait();
  griddep_launch_dependents();
  const int64_t base = (int64_t)blockIdx.x * TK_TILE;
  for (int i = threadIdx.x; i < TK_TILE; i += TK_BLK) sk[i] = base + i < n ? in[base + i] : KEY_INF;
  __syncthreads();
  for (int kk = 2; kk <= TK_TILE; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < TK_TILE / 2; t += TK_BLK) {
        int i = 2 * t - (t & (j - 1));
        int p = i + j;
        bool up = (i & kk) == 0;
        if ((sk[i] > sk[p]) == up) {
          unsigned long long x = sk[i];
          sk[i] = sk[p];
          sk[p] = x;
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < k; i += TK_BLK) out[(int64_t)blockIdx.x * k + i] = sk[i];
}

__global__ void k_topk_gather(const unsigned long long *keys, int32_t m, const int32_t *rows, const float *sc,
                              int32_t w, int32_t *orows, float *osc) {
  griddep_wait();
  griddep_launch_dependents();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / w;
    int32_t c = (int32_t)(e - i * w);
    uint32_t src = (uint32_t)(keys[i] & 0xffffffffu);
    orows[e] = rows[(int64_t)src * w + c];
    if (c == 0 && osc) osc[i] = sc[src];
  }
}

// Top-k of up to TK_SMALL keys in one block: the keys sit in shared memory, an MSD radix
// select over their 64 bits (8 bits a pass, warp-scanned histogram) finds the k-th smallest,
// the k keys at or below it are collected and sorted by a bitonic network, and the rows are
// gathered. One launch instead of the tile passes.
constexpr int TK_SMALL = 16384;
constexpr int TK_SBLK = 1024;

__global__ void __launch_bounds__(TK_SBLK) k_topk_small(const float *sc, int32_t n, int32_t k, const int32_t *rows,
                                                       int32_t w, int32_t *orows, float *osc) {
  extern __shared__ unsigned long long K[];  // n keys
  __shared__ unsigned long long C[1024];
  __shared__ unsigned hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_need, s_cnt;
  griddep_wait();
  griddep_launch_dependents();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += TK_SBLK) K[i] = ((unsigned long long)score_key(__ldg(sc + i)) << 32) | (uint32_t)i;
  const int kk = k < n ? k : n;
  if (tid == 0) {
    s_prefix = 0;
    s_need = kk;
    s_cnt = 0;
  }
  __syncthreads();
  unsigned long long T = KEY_INF;  // the kk-th smallest key (all keys when kk == n)
  if (kk < n) {
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int d = tid; d < 256; d += TK_SBLK) hist[d] = 0;
      __syncthreads();
      const unsigned long long hi = shift == 56 ? 0ull : (~0ull << (shift + 8));
      const unsigned long long pre = s_prefix;
      for (int i = tid; i < n; i += TK_SBLK)
        if ((K[i] & hi) == pre) atomicAdd(&hist[(K[i] >> shift) & 255], 1u);
      __syncthreads();
      if (warp == 0) {  // lane l holds bins 8l .. 8l+7
        unsigned b[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          b[j] = hist[8 * lane + j];
          sum += b[j];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          unsigned v = __shfl_up_sync(FULL_MASK, incl, o);
          if (lane >= o) incl += v;
        }
        const unsigned need = (unsigned)s_need;
        const unsigned excl = incl - sum;
        if (excl < need && need <= incl) {  // exactly one lane: the bin holding the need-th key
          unsigned cum = excl;
          int d = 0;
#pragma unroll
          for (int j = 0; j < 8; j++) {
            if (cum + b[j] >= need) {
              d = j;
              break;
            }
            cum += b[j];
          }
          s_prefix = pre | ((unsigned long long)(8 * lane + d) << shift);
          s_need = (int)(need - cum);
        }
      }
      __syncthreads();
    }
    T = s_prefix;
  }
  for (int i = tid; i < n; i += TK_SBLK)
    if (K[i] <= T) C[atomicAdd(&s_cnt, 1)] = K[i];
  __syncthreads();
  int P = 1;
  while (P < kk) P <<= 1;
  for (int i = kk + tid; i < P; i += TK_SBLK) C[i] = KEY_INF;
  __syncthreads();
  for (int q = 2; q <= P; q <<= 1)
    for (int j = q >> 1; j > 0; j >>= 1) {
      for (int t = tid; t < P / 2; t += TK_SBLK) {
        int i = 2 * t - (t & (j - 1));
        int p = i + j;
        bool up = (i & q) == 0;
        if ((C[i] > C[p]) == up) {
          unsigned long long x = C[i];
          C[i] = C[p];
          C[p] = x;
        }
      }
      __syncthreads();
    }
  for (int64_t e = tid; e < (int64_t)kk * w; e += TK_SBLK) {
    const int64_t i = e / w;
    const int32_t c = (int32_t)(e - i * w);
    const uint32_t src = (uint32_t)(C[i] & 0xffffffffu);
    orows[e] = __ldg(rows + (int64_t)src * w + c);
    if (c == 0 && osc) osc[i] = __ldg(sc + src);
  }
}

int64_t topk_tmp_bytes(int64_t n) {
  int64_t tiles = (n + TK_TILE - 1) / TK_TILE;
  return ((n > TK_TILE ? n : TK_TILE) + tiles * TK_TILE) * 8 + 256;
}

cudaError_t topk_sorted(const int32_t *rows, const float *sc, int64_t n, int32_t w, int32_t k, void *tmp,
                        int32_t *orows, float *osc, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  if (k > TK_TILE / 2) return cudaErrorInvalidValue;
  if (n <= TK_SMALL) {
    static std::atomic<unsigned long long> attr{0};  // per device, as for the join kernels
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr.load() & (1ull << (dev & 63)))) {
      cudaFuncSetAttribute(k_topk_small, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SMALL * 8);
      attr.fetch_or(1ull << (dev & 63));
    }
    g_launches++;
    k_topk_small<<<1, TK_SBLK, (size_t)n * 8, s>>>(sc, (int32_t)n, k, rows, w, orows, osc);
    return cudaGetLastError();
  }
  unsigned long long *a = (unsigned long long *)tmp;
  unsigned long long *b = a + (n > TK_TILE ? n : TK_TILE);
  int grid = (int)((n + 255) / 256);
  if (grid > 16384) grid = 16384;
  k_topk_keys_from_scores<<<grid, 256, 0, s>>>(sc, n, a);
  int launches = 1;
  unsigned long long *cur = a, *other = b;
  int64_t m = n;
  while (true) {  // every pass keeps k of each 2048 keys, so m at least halves
    int64_t blocks = (m + TK_TILE - 1) / TK_TILE;
    int32_t keep = (int32_t)(m < k ? m : k);
    launch_pdl(k_topk_tiles, dim3((unsigned)blocks), dim3(TK_BLK), 0, s, (const unsigned long long *)cur, m, keep,
               other);
    launches++;
    m = blocks * keep;
    std::swap(cur, other);
    if (blocks == 1) break;
  }
  int32_t out_n = (int32_t)(m < k ? m : k);
  int64_t ne = (int64_t)out_n * w;
  int g2 = (int)((ne + 255) / 256);
  launch_pdl(k_topk_gather, dim3(g2 > 0 ? g2 : 1), dim3(256), 0, s, (const unsigned long long *)cur, out_n, rows, sc,
             w, orows, osc);
  launches++;
  g_launches += launches;
  return cudaGetLastError();
}

}  // namespace dmk
