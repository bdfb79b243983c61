// Canonical (lexicographic) order of embedding rows, and top-k by (score, row).
//
// Rows are sorted by comparison rather than digit by digit: a row's first two ids are packed
// into one 64-bit key (most rows of an embedding table already differ there), ties fall back
// to the remaining columns read from the row itself. Tiles of 1024 rows are sorted by a
// bitonic network in shared memory; runs are then merged pairwise, each element finding its
// output position by a binary search in the other run (stable: ties keep run order). A sort
// of N rows takes 3 + ceil(log2(N / 1024)) launches.
//
// Top-k runs on a canonically sorted table: the key of row i is (FP32 score bits, i); scores
// are non-negative, so the bit pattern orders like the value, and i orders like the row.
// Each block sorts a tile of keys and keeps its k smallest; the candidates shrink by that
// factor per pass until one tile holds them all.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "kernels.h"

namespace dmk {

constexpr int MS_TILE = 1024;
constexpr int MS_BLK = 512;
constexpr unsigned long long KEY_INF = ~0ull;


// a < b for rows (key0, idx); idx < 0 is a padding element greater than every row. The key
// packs the first kc columns (floor(64 / bits) of them), so ties compare from column kc on.
__device__ __forceinline__ bool row_less(const int32_t *rows, int32_t w, int kc, unsigned long long ka, int32_t ia,
                                         unsigned long long kb, int32_t ib) {
  if (ka != kb) return ka < kb;
  if (ia < 0 || ib < 0) return ib < 0 && ia >= 0;
  const int32_t *ra = rows + (int64_t)ia * w, *rb = rows + (int64_t)ib * w;
  for (int c = kc; c < w; c++) {
    int32_t x = __ldg(ra + c), y = __ldg(rb + c);
    if (x != y) return x < y;
  }
  return ia < ib;
}

__global__ void k_pack_keys(const int32_t *rows, int64_t n, int32_t w, int bits, int kcols,
                            unsigned long long *key, int32_t *idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *r = rows + i * w;
    unsigned long long k = 0;
    for (int c = 0; c < kcols; c++) {
      unsigned long long v = c < w ? (uint32_t)__ldg(r + c) : 0u;
      k |= v << (64 - bits * (c + 1));
    }
    key[i] = k;
    idx[i] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(MS_BLK) k_sort_tiles(const int32_t *rows, int32_t w, int kc, int64_t n,
                                                       unsigned long long *key, int32_t *idx) {
  __shared__ unsigned long long sk[MS_TILE];
  __shared__ int32_t si[MS_TILE];
  const int64_t base = (int64_t)blockIdx.x * MS_TILE;
  for (int i = threadIdx.x; i < MS_TILE; i += MS_BLK) {
    int64_t g = base + i;
    sk[i] = g < n ? key[g] : KEY_INF;
    si[i] = g < n ? idx[g] : -1;
  }
  __syncthreads();
  for (int k = 2; k <= MS_TILE; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < MS_TILE / 2; t += MS_BLK) {
        int i = 2 * t - (t & (j - 1));
        int p = i + j;
        bool up = (i & k) == 0;
        bool gt = row_less(rows, w, kc, sk[p], si[p], sk[i], si[i]);
        if (gt == up) {
          unsigned long long tk = sk[i];
          sk[i] = sk[p];
          sk[p] = tk;
          int32_t ti = si[i];
          si[i] = si[p];
          si[p] = ti;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < MS_TILE; i += MS_BLK) {
    int64_t g = base + i;
    if (g < n) {
      key[g] = sk[i];
      idx[g] = si[i];
    }
  }
}

// Merge the sorted runs [b, b+L) and [b+L, b+2L) of (key, idx) into (okey, oidx).
__global__ void k_merge_pass(const int32_t *rows, int32_t w, int kc, int64_t n, int64_t L, const unsigned long long *key,
                             const int32_t *idx, unsigned long long *okey, int32_t *oidx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pair = i / (2 * L);
    const int64_t b = pair * 2 * L;
    const bool inA = i < b + L;
    const int64_t ob = inA ? b + L : b;                 // the other run
    const int64_t oe = inA ? (b + 2 * L < n ? b + 2 * L : n) : b + L;
    const unsigned long long kx = key[i];
    const int32_t ix = idx[i];
    int64_t lo = ob, hi = oe > ob ? oe : ob;
    // A elements go before equal B elements: count B < x for A, A <= x for B
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      bool before = inA ? row_less(rows, w, kc, key[mid], idx[mid], kx, ix)
                        : !row_less(rows, w, kc, kx, ix, key[mid], idx[mid]);
      if (before) lo = mid + 1;
      else hi = mid;
    }
    const int64_t pos = b + (i - (inA ? b : b + L)) + (lo - ob);
    okey[pos] = kx;
    oidx[pos] = ix;
  }
}

int64_t msort_tmp_bytes(int64_t n) { return n * (8 + 4) * 2 + 256; }

cudaError_t msort_rows(const int32_t *rows, int64_t n, int32_t w, int bits, void *tmp, int32_t **perm_out,
                       cudaStream_t s) {
  unsigned long long *k0 = (unsigned long long *)tmp;
  unsigned long long *k1 = k0 + n;
  int32_t *i0 = (int32_t *)(k1 + n);
  int32_t *i1 = i0 + n;
  *perm_out = i0;
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 16384) grid = 16384;
  if (bits < 1) bits = 1;
  if (bits > 32) bits = 32;
  int kcols = 64 / bits;
  if (kcols > w) kcols = w;
  k_pack_keys<<<grid, 256, 0, s>>>(rows, n, w, bits, kcols, k0, i0);
  k_sort_tiles<<<(unsigned)((n + MS_TILE - 1) / MS_TILE), MS_BLK, 0, s>>>(rows, w, kcols, n, k0, i0);
  int launches = 2;
  for (int64_t L = MS_TILE; L < n; L *= 2) {
    k_merge_pass<<<grid, 256, 0, s>>>(rows, w, kcols, n, L, k0, i0, k1, i1);
    launches++;
    std::swap(k0, k1);
    std::swap(i0, i1);
  }
  g_launches += launches;
  *perm_out = i0;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ images (dedup) -----
// Sort the ids inside every row (the row becomes its vertex set), one thread per row.
__global__ void k_sort_within_rows(int32_t *rows, int64_t n, int32_t w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t *r = rows + i * w;
    for (int a = 1; a < w; a++) {  // insertion sort: rows are at most 64 ids
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
    key[i] = ((unsigned long long)__float_as_uint(__ldg(sc + i)) << 32) | (uint32_t)i;
}

// Each block sorts TK_TILE keys and writes its k smallest (k <= TK_TILE).
__global__ void __launch_bounds__(TK_BLK) k_topk_tiles(const unsigned long long *in, int64_t n, int32_t k,
                                                       unsigned long long *out) {
  __shared__ unsigned long long sk[TK_TILE];
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
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / w;
    int32_t c = (int32_t)(e - i * w);
    uint32_t src = (uint32_t)(keys[i] & 0xffffffffu);
    orows[e] = rows[(int64_t)src * w + c];
    if (c == 0 && osc) osc[i] = sc[src];
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
    k_topk_tiles<<<(unsigned)blocks, TK_BLK, 0, s>>>(cur, m, keep, other);
    launches++;
    m = blocks * keep;
    std::swap(cur, other);
    if (blocks == 1) break;
  }
  int32_t out_n = (int32_t)(m < k ? m : k);
  int64_t ne = (int64_t)out_n * w;
  int g2 = (int)((ne + 255) / 256);
  k_topk_gather<<<g2 > 0 ? g2 : 1, 256, 0, s>>>(cur, out_n, rows, sc, w, orows, osc);
  launches++;
  g_launches += launches;
  return cudaGetLastError();
}

}  // namespace dmk
