// sm_103a kernels of the Delta-Motif library besides the join: data-graph preparation (CSR
// to M2 table, adjacency bitmap), motif-table indexes (direct offsets, open-addressing hash on
// packed 64-bit keys), scans, LSD radix passes, row gathers, score histograms and selection,
// and the row checksum. The join of Alg. 1 is in join_warp.cu (per step) and batch.cu
// (persistent, all steps of many plans), on the device code of join_device.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "join_device.cuh"
#include "kernels.h"

using namespace dmi;

namespace dmk {

thread_local int64_t g_launches = 0;
int64_t launch_count() { return g_launches; }

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
static_assert(SCAN_TILE == SCAN_BLK * SCAN_ITEMS, "scan tile");

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
static_assert(RS_TILE == RS_BLK * RS_ITEMS, "radix tile");

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
  const int tid = threadIdx.x, warp = tid >> 5;
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

// Chunk boundaries for streaming: bounds[t] = the largest row index i with pre[i] <= t * step
// (bounds[0] = 0, bounds[nch] = n), and bpre[t] = pre[bounds[t]]; pre has n + 1 entries and is
// non-decreasing.
__global__ void k_chunk_bounds(const int64_t *pre, int64_t n, int64_t step, int64_t nch, int64_t *bounds,
                               int64_t *bpre) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= nch; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx;
    if (t == 0) idx = 0;
    else if (t == nch) idx = n;
    else {
      const int64_t target = t * step;
      int64_t lo = 0, hi = n + 1;  // first index with pre > target, in [0, n + 1]
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pre[mid] <= target) lo = mid + 1;
        else hi = mid;
      }
      idx = lo - 1 < 0 ? 0 : lo - 1;
    }
    bounds[t] = idx;
    bpre[t] = pre[idx];
  }
}

cudaError_t launch_chunk_bounds(const int64_t *pre, int64_t n, int64_t step, int64_t nch, int64_t *bounds,
                                int64_t *bpre, cudaStream_t s) {
  g_launches++;
  const int64_t blocks = (nch + 1 + 255) / 256;
  k_chunk_bounds<<<(int)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(pre, n, step, nch, bounds, bpre);
  return cudaGetLastError();
}

// Sort-merge join keys: keys[i] = packed (row[kp0], row[kp1]) (kp1 < 0: row[kp0]) of each row.
__global__ void k_join_keys(const int32_t *rows, int32_t w, int32_t kp0, int32_t kp1, int64_t n,
                            unsigned long long *keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *r = rows + i * w;
    const unsigned long long a = (uint32_t)__ldg(r + kp0);
    keys[i] = kp1 >= 0 ? ((a << 32) | (uint32_t)__ldg(r + kp1)) : a;
  }
}

cudaError_t launch_join_keys(const int32_t *rows, int32_t w, int32_t kp0, int32_t kp1, int64_t n,
                             unsigned long long *keys, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_join_keys<<<(int)imin64((n + 255) / 256, 16384), 256, 0, s>>>(rows, w, kp0, kp1, n, keys);
  return cudaGetLastError();
}

// In place: e -> -log(1 - e), the negative log of the fidelity 1 - e.
__global__ void k_neg_log1m(float *w, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = -log1pf(-w[i]);
}

cudaError_t launch_neg_log1m(float *w, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_neg_log1m<<<(int)imin64((n + 255) / 256, 4096), 256, 0, s>>>(w, n);
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
    uint32_t b = score_key(__ldg(sc + i));
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
    uint32_t b = score_key(__ldg(sc + i));
    if (b <= T) out_idx[atomicAdd(ctr, 1ull)] = (int32_t)i;
  }
}

// Direction-aware score of each row (one thread per row): the sum over the pattern's weighted
// slots p -> q of w * edir[slot of f(p) -> f(q) in the data graph's CSR], plus the vertex
// errors of the row's images when qerr is given; FP32, slots in the order given.
__global__ void k_rescore_directed(const int32_t *rows, int64_t n, int32_t np, const int32_t *sp, const int32_t *sq,
                                   const float *sw, int32_t nslots, const int32_t *row_ptr, const int32_t *col_idx,
                                   const float *edir, const float *qerr, float *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t *f = rows + i * np;
    float s = 0.f;
    for (int32_t e = 0; e < nslots; e++) {
      const int32_t u = __ldg(f + __ldg(sp + e)), v = __ldg(f + __ldg(sq + e));
      int32_t lo = __ldg(row_ptr + u), hi = __ldg(row_ptr + u + 1);
      float c = 0.f;
      while (lo < hi) {  // the slot of u -> v (present: the row is an embedding)
        const int32_t mid = (lo + hi) >> 1, x = __ldg(col_idx + mid);
        if (x == v) {
          c = __ldg(edir + mid);
          break;
        }
        if (x < v) lo = mid + 1;
        else hi = mid;
      }
      s += __ldg(sw + e) * c;
    }
    if (qerr)
      for (int32_t u = 0; u < np; u++) s += __ldg(qerr + __ldg(f + u));
    out[i] = s;
  }
}

cudaError_t launch_rescore_directed(const int32_t *rows, int64_t n, int32_t np, const int32_t *sp, const int32_t *sq,
                                    const float *sw, int32_t nslots, const int32_t *row_ptr, const int32_t *col_idx,
                                    const float *edir, const float *qerr, float *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_rescore_directed<<<(int)imin64((n + 255) / 256, 8192), 256, 0, s>>>(rows, n, np, sp, sq, sw, nslots, row_ptr,
                                                                          col_idx, edir, qerr, out);
  return cudaGetLastError();
}

__global__ void k_score_keys(const float *sc, int64_t n, uint32_t *keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = score_key(__ldg(sc + i));
}

cudaError_t launch_score_keys(const float *sc, int64_t n, uint32_t *keys, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  g_launches++;
  k_score_keys<<<(int)imin64((n + 255) / 256, 4096), 256, 0, s>>>(sc, n, keys);
  return cudaGetLastError();
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
    unsigned long long p = 0;
    for (int c = 0; c < w; c++) p += col_term(c, __ldg(row + c));
    hs += dmix64(p + (unsigned long long)(uint32_t)w);
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
