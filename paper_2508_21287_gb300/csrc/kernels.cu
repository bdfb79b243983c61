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

#include "join_device.cuh"
#include "kernels.h"

using namespace dmi;

namespace dmk {

std::atomic<int64_t> g_launches{0};
int64_t launch_count() { return g_launches.load(); }

// ------------------------------------------------------------------ join kernel --------
int join_tile_rows(int w) {
  if (w <= 0) return JOIN_BLK;
  int ws = w | 1;
  int tr = 24576 / (ws * 4);
  tr = tr / 32 * 32;
  if (tr < 32) tr = 32;
  if (tr > JOIN_BLK) tr = JOIN_BLK;
  return tr;
}

static int join_cpt(int n_new) { return n_new <= 4 ? 4 : 1; }

size_t join_smem_bytes(int w, int wo, int tile_rows) {
  (void)wo;
  size_t offs[7];
  return join_smem_layout(tile_rows, w > 0 ? (w | 1) : 1, JOIN_BLK * 4, 2, offs);
}

template <int BLK, int MAXNEW, int CPT, int MODE>
__global__ void __launch_bounds__(BLK, 3) k_join(const __grid_constant__ JoinArgs a, int TR) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_warp[BLK / 32];
  __shared__ unsigned long long s_red[BLK / 32];
  __shared__ long long s_base;
  const bool seed = a.R == nullptr;
  const int ws = a.w > 0 ? (a.w | 1) : 1;
  const JoinSmem S = join_smem(smem, TR, ws, BLK * CPT, 2);
  const int64_t N = seed ? 0 : (a.n_dev ? imin64((int64_t)*a.n_dev, a.in_cap) : a.N);
  const int64_t per = seed ? (int64_t)BLK * CPT : TR;
  const int64_t nt = seed ? (a.seed_hi - a.seed_lo + per - 1) / per : (N + TR - 1) / TR;
  TileOut o;
  o.out = a.out;
  o.outs = a.outs;
  o.out_next = a.out_next;
  o.cap = a.out_cap;
  o.gctr = a.ctr + CTR_ROWS;
  o.lctr = nullptr;
  o.ovf = a.ctr + CTR_OVF;
  o.next_ctr = a.ctr + CTR_NEXT;
  unsigned long long acc_rows = 0, acc_sum = 0, acc_cand = 0;
  if (seed) {
    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
      const int64_t m0 = a.seed_lo + t * per;
      join_tile<BLK, MAXNEW, CPT, MODE>(a, S, TR, 0, false, nullptr, nullptr, 0, m0,
                                        (int)imin64(per, a.seed_hi - m0), o, s_warp, s_red, &s_base, acc_rows,
                                        acc_sum, acc_cand);
    }
  } else {
    // double buffering: the next tile of this block streams into the other buffer (cp.async)
    // while the current one is joined
    int buf = 0;
    int64_t t = blockIdx.x;
    if (t < nt)
      load_tile<BLK, true>(S.tile_buf[0], S.ts_buf[0], a.R + t * TR * a.w, a.Rs ? a.Rs + t * TR : nullptr,
                           (int)imin64(TR, N - t * TR), a.w);
    cp_async_commit();
    for (; t < nt; t += gridDim.x) {
      const int64_t tn = t + gridDim.x;
      if (tn < nt)
        load_tile<BLK, true>(S.tile_buf[buf ^ 1], S.ts_buf[buf ^ 1], a.R + tn * TR * a.w,
                             a.Rs ? a.Rs + tn * TR : nullptr, (int)imin64(TR, N - tn * TR), a.w);
      cp_async_commit();
      cp_async_wait_all_but_one();
      __syncthreads();
      const int64_t r0 = t * TR;
      join_tile<BLK, MAXNEW, CPT, MODE>(a, S, TR, buf, true, a.R + r0 * a.w, a.Rs ? a.Rs + r0 : nullptr,
                                        (int)imin64(TR, N - r0), 0, 0, o, s_warp, s_red, &s_base, acc_rows, acc_sum,
                                        acc_cand);
      buf ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
  }
  unsigned long long tc = block_sum_u64<BLK>(acc_cand, s_red);
  if (threadIdx.x == 0 && tc) atomicAdd(a.ctr + CTR_CAND, tc);
  if (MODE == 1) {
    unsigned long long tr = block_sum_u64<BLK>(acc_rows, s_red);
    unsigned long long ts = block_sum_u64<BLK>(acc_sum, s_red);
    if (threadIdx.x == 0) {
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
