// Persistent batch kernel: count + checksum for many plans on one data graph in one launch.
//
// Work items are root chunks (plan p, rows [lo, hi) of the motif table of p's first slice).
// Each CTA takes the next item from a global counter and runs it depth-first through every
// step of Alg. 1: level j of the CTA's private scratch holds the output of step j for the
// current chunk of level j-1, at most TR input rows at a time, so a level never holds more
// than TR * (largest key group of step j) rows. The last step is counted, not written. No CTA
// ever waits for another; load balance comes from small root chunks taken in order of the
// plans' estimated cost. Join, filter, score and compaction are the same device code as the
// per-step kernel (join_device.cuh). The kernel exists for two block shapes (128 and 256
// threads); a third shape, one walk per warp, is k_batchw (join_warp.cu). The autotuner picks
// the shape and how many CTAs run per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "join_device.cuh"
#include "kernels.h"

namespace dmk {


template <int BATCH_BLK>
__device__ __forceinline__ void batch_tile(const JoinArgs &a, const JoinSmem &S, int TR, const int32_t *src,
                                           int nr, int64_t m0, int seedC, const TileOut &o, int *s_warp,
                                           unsigned long long *s_red, long long *s_base, unsigned long long &ar,
                                           unsigned long long &as, unsigned long long &ac) {
  if (a.mode == 1) {
    if (a.n_new <= 1)
      join_tile<BATCH_BLK, 1, 4, 1>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
    else if (a.n_new <= 4)
      join_tile<BATCH_BLK, 4, 4, 1>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
    else
      join_tile<BATCH_BLK, MAXM, 1, 1>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
  } else {
    if (a.n_new <= 1)
      join_tile<BATCH_BLK, 1, 4, 0>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
    else if (a.n_new <= 4)
      join_tile<BATCH_BLK, 4, 4, 0>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
    else
      join_tile<BATCH_BLK, MAXM, 1, 0>(a, S, TR, 0, false, src, nullptr, nr, m0, seedC, o, s_warp, s_red, s_base, ar, as, ac);
  }
}

__device__ __forceinline__ void load_args(JoinArgs *dst, const JoinArgs *src) {
  const int n = sizeof(JoinArgs) / 4;
  int32_t *d = (int32_t *)dst;
  const int32_t *s = (const int32_t *)src;
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// 128-thread CTAs: up to 5 per SM (at most 102 registers a thread; a few spill), 256-thread CTAs: 2
template <int BATCH_BLK>
__global__ void __launch_bounds__(BATCH_BLK, 640 / BATCH_BLK) k_batch(const __grid_constant__ BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) JoinArgs sa;
  __shared__ int s_warp[BATCH_BLK / 32];
  __shared__ unsigned long long s_red[BATCH_BLK / 32];
  __shared__ long long s_base, s_lctr;
  __shared__ long long s_item;
  __shared__ int64_t n_lvl[MAXSTEPS], cur[MAXSTEPS];

  JoinSmem S = join_smem(smem, P.TR, P.ws_max, BATCH_BLK * 4, 1);
  if (P.bm_words > 0) {
    size_t offs[7];
    S.bm = (unsigned long long *)(smem + join_smem_layout(P.TR, P.ws_max, BATCH_BLK * 4, 1, offs));
    S.bmw = P.bm_words;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.start_ns = globaltimer_ns();
  unsigned char *mine = P.scratch + (int64_t)blockIdx.x * P.cta_bytes;
  TileOut o;
  o.out_next = nullptr;
  o.outs = nullptr;
  o.gctr = nullptr;
  o.lctr = &s_lctr;
  o.ovf = P.ovf;
  o.next_ctr = nullptr;

  while (true) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(P.next_item, 1ull);
    __syncthreads();
    const long long it = s_item;
    if (it >= P.n_items) break;
    const BatchItem item = P.items[it];
    const BatchPlan plan = P.plans[item.plan];
    const int nsteps = plan.n_steps;
    unsigned long long ar = 0, as = 0, ac = 0;

    // step 0: the root chunk's motif rows are the candidates
    load_args(&sa, P.args + plan.args_off);
    if (threadIdx.x == 0) s_lctr = 0;
    __syncthreads();
    o.out = (int32_t *)(mine + P.lvl_off[0]);
    o.cap = P.lvl_cap[0];
    batch_tile<BATCH_BLK>(sa, S, P.TR, nullptr, 0, item.lo, (int)(item.hi - item.lo), o, s_warp, s_red, &s_base, ar, as, ac);
    if (threadIdx.x == 0) {
      n_lvl[0] = s_lctr;
      cur[0] = 0;
    }
    __syncthreads();
    int top = nsteps > 1 ? 0 : -1;
    while (top >= 0) {
      if (top == nsteps - 1 || cur[top] >= n_lvl[top]) {
        top--;
        continue;
      }
      const int j = top + 1;
      load_args(&sa, P.args + plan.args_off + j);
      const int32_t *lv = (const int32_t *)(mine + P.lvl_off[top]);
      const int64_t c0 = cur[top];
      const int nr = (int)imin64(P.TR, n_lvl[top] - c0);
      if (threadIdx.x == 0) s_lctr = 0;
      __syncthreads();
      o.out = (int32_t *)(mine + P.lvl_off[j]);
      o.cap = P.lvl_cap[j];
      batch_tile<BATCH_BLK>(sa, S, P.TR, lv + c0 * sa.w, nr, 0, 0, o, s_warp, s_red, &s_base, ar, as, ac);
      __syncthreads();
      if (threadIdx.x == 0) {
        cur[top] = c0 + nr;
        if (j < nsteps - 1) {
          n_lvl[j] = s_lctr;
          cur[j] = 0;
        }
      }
      __syncthreads();
      if (j < nsteps - 1) top = j;
    }
    unsigned long long tr = block_sum_u64<BATCH_BLK>(ar, s_red);
    unsigned long long ts = block_sum_u64<BATCH_BLK>(as, s_red);
    if (threadIdx.x == 0) {
      if (nsteps == 1 || tr) {
        atomicAdd(P.out + 2 * item.plan, tr);
        atomicAdd(P.out + 2 * item.plan + 1, ts);
      }
      __threadfence();
      if (atomicAdd(P.plan_left + item.plan, ~0ull) == 1ull) P.plan_done[item.plan] = globaltimer_ns();
    }
    __syncthreads();
  }
}

typedef void (*BatchKernel)(BatchParams);

static BatchKernel batch_kernel(int threads) { return threads == 128 ? k_batch<128> : k_batch<256>; }

size_t batch_smem_bytes(int tile_rows, int ws_max, int bm_words, int threads) {
  size_t offs[7];
  return join_smem_layout(tile_rows, ws_max, threads * 4, 1, offs) + (size_t)tile_rows * bm_words * 8;
}

int batch_grid(int tile_rows, int ws_max, int bm_words, int num_sms, int threads, int max_per_sm) {
  size_t smem = batch_smem_bytes(tile_rows, ws_max, bm_words, threads);
  BatchKernel k = batch_kernel(threads);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (per_sm < 1) per_sm = 1;
  if (max_per_sm > 0 && per_sm > max_per_sm) per_sm = max_per_sm;
  return num_sms * per_sm;
}

cudaError_t launch_batch(const BatchParams &p, int grid, int threads, cudaStream_t s) {
  size_t smem = batch_smem_bytes(p.TR, p.ws_max, p.bm_words, threads);
  BatchKernel k = batch_kernel(threads);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  g_launches++;
  k<<<grid, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace dmk
