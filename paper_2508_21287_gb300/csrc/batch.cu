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
// threads); a third shape, one walk per warp, is k_batchw (below). The autotuner picks
// the shape and how many CTAs run per SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "join_device.cuh"
#include "join_warp.cuh"
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

// ---------------------------------------------------------------------------------------
// Persistent batch kernel with one depth-first walk per warp (count + checksum for many plans
// on one data graph; the "warp walk" block shape of dm_match_batch). Every warp takes work
// items (plan, rows of the motif table of its first slice) from the global counter and runs
// each one through the plan's steps on its own: level j of the warp's scratch holds step j's
// output for the current tile (up to 32 rows) of level j - 1, at most 32 x the step's largest
// key group rows, and the last step is counted. A step over one tile is k_joinw's warp tile -- the same
// lookup, candidate walk, checks, staging and 16-byte flush -- so no warp waits for another and
// no block barrier is taken. Level rows are written and read back within the launch, so they
// are read with plain (coherent) loads, never through the read-only cache path.

// 64-entry staging lists: the smaller footprint keeps more walks resident than a longer list
// would save in flushes (the walks are latency-bound). Each walk's shared tile holds
// tile_words words (BatchParams): a step whose rows take s words (join_row_stride) joins
// min(32, tile_words / s) rows a tile, so the few wide steps of a batch take shorter tiles
// instead of every walk reserving 32 rows of the widest.
constexpr int BW_WARPS = BW_WALK_WARPS, BW_BLK = 32 * BW_WARPS, BW_STAGE = 64;

__host__ __device__ __forceinline__ int walk_tile_rows(int tile_words, int w) {
  const int r = tile_words / join_row_stride(w);
  return r < WT ? r : WT;
}

// The warp's tile, checksum terms, scores and staging list (the layout of warp_smem with a
// fixed tile of tile_words words).
__host__ __device__ __forceinline__ size_t walk_head_bytes(int tile_words) {
  size_t b = (size_t)tile_words * 4 + (size_t)WT * 8 + (size_t)WT * 4;
  b = (b + 15) / 16 * 16 + (size_t)BW_STAGE * 12 + (size_t)BW_STAGE * STAGE_NV * 4;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ WarpSmem walk_warp(unsigned char *base, int tile_words) {
  WarpSmem m;
  size_t off = (size_t)tile_words * 4;  // a multiple of 16
  m.rows = (int32_t *)base;
  m.part = (unsigned long long *)(base + off);
  off += (size_t)WT * 8;
  m.rs = (float *)(base + off);
  off += (size_t)WT * 4;
  off = (off + 15) / 16 * 16;
  m.st_r = (int32_t *)(base + off);
  m.st_m = m.st_r + BW_STAGE;
  m.st_s = (float *)(m.st_m + BW_STAGE);
  m.st_nv = (int32_t *)(m.st_s + BW_STAGE);
  return m;
}

struct WalkSmem {
  int32_t *tq;           // MAXW: counted step, 1 + output position of each working column
  int16_t *code;         // MAXW (over tq: a step is either written or counted): packed flush,
                         // output position -> working column / new vertex
  int8_t *npos;          // MAXM: counted step, output position of each new vertex
  int32_t *n_lvl, *cur;  // per level: rows held, rows already joined into the next level
};

__host__ __device__ __forceinline__ size_t walk_warp_bytes(int tile_words, int max_steps) {
  size_t b = walk_head_bytes(tile_words) + (size_t)MAXW * 4 + MAXM;
  b = (b + 15) / 16 * 16 + (size_t)max_steps * 8;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ WalkSmem walk_smem(unsigned char *base, int tile_words, int max_steps) {
  WalkSmem k;
  size_t off = walk_head_bytes(tile_words);  // a multiple of 16
  k.tq = (int32_t *)(base + off);
  k.code = (int16_t *)(base + off);
  off += (size_t)MAXW * 4;
  k.npos = (int8_t *)(base + off);
  off += MAXM;
  off = (off + 15) / 16 * 16;
  k.n_lvl = (int32_t *)(base + off);
  k.cur = k.n_lvl + max_steps;
  return k;
}

// Copy nr rows of a level (row stride rs words: rs = w packed, or a multiple of 4 with 16-byte
// aligned rows) into the warp tile (stride wsv, padding words already -1); plain loads.
__device__ __forceinline__ void walk_load_tile(int32_t *rows, int wsv, const int32_t *src, int nr, int w, int rs) {
  const int lane = threadIdx.x & 31;
  if ((rs & 3) == 0) {  // whole int4s (a padded level keeps its -1 padding)
    const int q = rs >> 2, qs = wsv >> 2, n4 = nr * q;
    const int4 *s4 = (const int4 *)src;
    int4 *d4 = (int4 *)rows;
    int r = lane / q, c = lane - r * q;  // int4 k = r * q + c, advanced with carry
    const int dr = 32 / q, dc = 32 % q;
    for (int k = lane; k < n4; k += 32) {
      d4[r * qs + c] = s4[k];
      r += dr;
      c += dc;
      if (c >= q) {
        c -= q;
        r++;
      }
    }
  } else {
    const int ne = nr * w;
    int r = lane / w, c = lane % w;  // element e = r * w + c, advanced with carry
    const int dr = 32 / w, dc = 32 % w;
    for (int e = lane; e < ne; e += 32) {
      rows[r * wsv + c] = src[e];
      r += dr;
      c += dc;
      if (c >= w) {
        c -= w;
        r++;
      }
    }
  }
}

// Append the warp's n staged survivors to its level buffer (n_out rows so far, cap rows; row
// stride rs_out, or a.wo when packed); rows past cap are dropped and the overflow flag raised.
template <int MAXNEW>
__device__ __forceinline__ void walk_flush(const JoinArgs &a, const WarpSmem &W, const int16_t *code, int wsv, int n,
                                           int32_t *out, int rs_out, int64_t cap, int64_t &n_out,
                                           unsigned long long *ovf) {
  constexpr bool STG = MAXNEW <= STAGE_NV;
  const int64_t base = n_out;
  int Kc = n;
  if (base + n > cap) {
    Kc = (int)imax64(0, cap - base);
    if ((threadIdx.x & 31) == 0) atomicOr(ovf, 1ull);
  }
  n_out = base + n;
  if (STG && rs_out) wwrite_padded<STG ? MAXNEW : 1>(W, wsv, a.w, Kc, out + base * rs_out, rs_out);
  else wwrite<STG>(a, W, code, wsv, Kc, out + base * a.wo, a.wo);
  __syncwarp();
}

// One step of a plan over one tile: nr rows of a level (src, row stride rs_in) or, for the first
// step (src == nullptr), motif rows [m0, m0 + nr) as the candidates. MODE 0 appends the
// survivors to level `out`; MODE 1 (the last step) adds their count and checksum.
// Check one candidate of a step with more than 4 new vertices (or none): each new vertex is read
// from the motif row as the tests reach it, since most candidates fail after a few of them.
__device__ __forceinline__ bool wcheck_lazy(const JoinArgs &a, const WarpSmem &W, int wsv, bool seed, int r, int m) {
  const int32_t *rrow = W.rows + r * wsv;
  const int32_t *trow = a.ix.rows + (int64_t)m * a.ix.mw;
  bool ok = true;
  for (int i = 0; i < a.n_chk; i++) ok &= __ldg(trow + a.chk_mpos[i]) == rrow[a.chk_col[i]];
  if (!seed)
    for (int i = 0; i < a.n_new && ok; i++) ok = !row_has(rrow, a.w, __ldg(trow + a.new_mpos[i]));
  for (int e = 0; e < a.n_be && ok; e++) ok = adjacent(a, join_value(a, rrow, trow, a.be_a[e]), join_value(a, rrow, trow, a.be_b[e]));
  if (ok && a.induced) ok = induced_ok_lazy<MAXM>(a, rrow, trow);
  return ok;
}

template <int MAXNEW, int MODE>
__device__ __forceinline__ void walk_tile(const JoinArgs &a, const WarpSmem &W, const WalkSmem &K,
                                          const int32_t *src, int rs_in, int nr, int64_t m0, int32_t *out, int rs_out,
                                          int64_t cap, int64_t &n_out, unsigned long long *ovf,
                                          unsigned long long &acc_rows, unsigned long long &acc_sum) {
  constexpr bool STG = MAXNEW <= STAGE_NV;
  const int lane = threadIdx.x & 31;
  const bool seed = src == nullptr;
  const int w = a.w, wo = a.wo;
  const int wsv = join_row_stride(w);
  for (int q = lane; q < wo; q += 32) {  // where this step's columns go
    const int col = a.src_col[q];
    if (MODE == 1) {
      if (col < w) K.tq[col] = q + 1;
      else K.npos[col - w] = (int8_t)q;
    } else {
      K.code[q] = (int16_t)(col < w ? col : (0x100 | (col - w)));
    }
  }
  if (lane < nr)  // padding words of the tile rows (row 0 in the first step: read by the padded flush)
    for (int c = w; c < wsv; c++) W.rows[lane * wsv + c] = -1;
  __syncwarp();
  int C;
  int g_start = 0, g_off = 0;
  if (!seed) {
    walk_load_tile(W.rows, wsv, src, nr, w, rs_in);
    __syncwarp();
    int start = 0, len = 0;
    if (lane < nr) {
      const int32_t *row = W.rows + lane * wsv;
      if (MODE == 1) W.part[lane] = row_terms_last(row, w, K.tq);
      ix_lookup(a.ix, row[a.key_col[0]], a.ix.nkeys == 2 ? row[a.key_col[1]] : 0, start, len);
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL_MASK, incl, o);
      if (lane >= o) incl += v;
    }
    C = __shfl_sync(FULL_MASK, incl, 31);
    g_start = start;
    g_off = incl - len;
    __syncwarp();
  } else {
    C = nr;
  }
  const int32_t *mrows = a.ix.rows;
  const int mw = a.ix.mw;
  int nst = 0;
  for (int cb = 0; cb < C; cb += 32) {
    const int c = cb + lane;
    const bool valid = c < C;
    int r = 0, m = 0;
    if (!seed) {
      round_rows(g_start, g_off, cb, C, r, m);
    } else if (valid) {
      m = (int)(m0 + c);
    }
    constexpr int NV = STG ? MAXNEW : 1;  // the lazy check of wide steps keeps no new vertices
    int32_t nv[NV];
    const int32_t *trow = mrows + (int64_t)m * mw;  // row 0 for idle lanes: a valid address
    bool ok;
    if constexpr (STG) {
#pragma unroll
      for (int i = 0; i < MAXNEW; i++) nv[i] = __ldg(trow + a.new_mpos[i]);
      float sc = 0.f;
      ok = valid && wcheck<MAXNEW>(a, W, wsv, seed, r, m, nv, sc);
    } else {
      ok = valid && wcheck_lazy(a, W, wsv, seed, r, m);
    }
    if (MODE == 1) {
      if (ok) {
        unsigned long long p = seed ? 0ull : W.part[r];
        if constexpr (STG) {
#pragma unroll
          for (int i = 0; i < MAXNEW; i++) p += pos_term(K.npos[i] + 1, nv[i]);
        } else {
          for (int i = 0; i < a.n_new; i++) p += pos_term(K.npos[i] + 1, __ldg(trow + a.new_mpos[i]));
        }
        acc_sum += dmix64(p + (unsigned long long)(uint32_t)wo);
        acc_rows++;
      }
    } else {
      const unsigned bal = __ballot_sync(FULL_MASK, ok);
      if (ok) {
        const int pos = nst + __popc(bal & lanemask_lt());
        W.st_r[pos] = r;
        W.st_m[pos] = m;
        if constexpr (STG) {
#pragma unroll
          for (int i = 0; i < MAXNEW; i++) W.st_nv[pos * STAGE_NV + i] = nv[i];
        }
      }
      nst += __popc(bal);
      __syncwarp();
      if (nst > BW_STAGE - 32) {
        walk_flush<MAXNEW>(a, W, K.code, wsv, nst, out, rs_out, cap, n_out, ovf);
        nst = 0;
      }
    }
  }
  if (MODE == 0 && nst > 0) walk_flush<MAXNEW>(a, W, K.code, wsv, nst, out, rs_out, cap, n_out, ovf);
  __syncwarp();  // the next tile overwrites this warp's rows and tables
}

template <int MODE>
__device__ __forceinline__ void walk_step_mode(const JoinArgs &a, const WarpSmem &W, const WalkSmem &K,
                                               const int32_t *src, int rs_in, int nr, int64_t m0, int32_t *out,
                                               int rs_out, int64_t cap, int64_t &n_out, unsigned long long *ovf,
                                               unsigned long long &ar, unsigned long long &as) {
  switch (a.n_new) {
    case 1: walk_tile<1, MODE>(a, W, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 2: walk_tile<2, MODE>(a, W, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 3: walk_tile<3, MODE>(a, W, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 4: walk_tile<4, MODE>(a, W, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    default: walk_tile<MAXM, MODE>(a, W, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as);
  }
}

// Row stride (words) of the level a step writes.
__host__ __device__ __forceinline__ int walk_level_stride(const JoinArgs &a) { return a.rs_out ? a.rs_out : a.wo; }

__global__ void __launch_bounds__(BW_BLK, 14) k_batchw(const __grid_constant__ BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *wbase = smem + (size_t)wid * walk_warp_bytes(P.tile_words, P.max_steps);
  const WarpSmem W = walk_warp(wbase, P.tile_words);
  const WalkSmem K = walk_smem(wbase, P.tile_words, P.max_steps);
  if (blockIdx.x == 0 && threadIdx.x == 0) *P.start_ns = globaltimer_ns();
  unsigned char *mine = P.scratch + ((int64_t)blockIdx.x * BW_WARPS + wid) * P.cta_bytes;
  while (true) {
    long long it = 0;
    if (lane == 0) it = (long long)atomicAdd(P.next_item, 1ull);
    it = __shfl_sync(FULL_MASK, it, 0);
    if (it >= P.n_items) break;
    const BatchItem item = P.items[it];
    const BatchPlan plan = P.plans[item.plan];
    const int S = plan.n_steps;
    const JoinArgs *args = P.args + plan.args_off;
    unsigned long long ar = 0, as = 0;
    {  // first step: the item's motif rows are the candidates, 32 at a time
      const JoinArgs &a0 = args[0];
      int32_t *out = (int32_t *)(mine + P.lvl_off[0]);
      int64_t n_out = 0;
      for (int64_t lo = item.lo; lo < item.hi; lo += 32) {
        const int nr = (int)imin64(32, item.hi - lo);
        if (S == 1)
          walk_step_mode<1>(a0, W, K, nullptr, 0, nr, lo, nullptr, 0, 0, n_out, P.ovf, ar, as);
        else
          walk_step_mode<0>(a0, W, K, nullptr, 0, nr, lo, out, a0.rs_out, P.lvl_cap[0], n_out, P.ovf, ar, as);
      }
      if (lane == 0) {
        K.n_lvl[0] = (int32_t)imin64(n_out, P.lvl_cap[0]);
        K.cur[0] = 0;
      }
      __syncwarp();
    }
    int top = S > 1 ? 0 : -1;
    while (top >= 0) {
      const int cur = K.cur[top], have = K.n_lvl[top];
      if (top == S - 1 || cur >= have) {
        top--;
        continue;
      }
      const int j = top + 1;
      const int nr = min(walk_tile_rows(P.tile_words, args[j].w), have - cur);
      const int rs_in = walk_level_stride(args[top]);
      const int32_t *src = (const int32_t *)(mine + P.lvl_off[top]) + (int64_t)cur * rs_in;
      const JoinArgs &a = args[j];
      int64_t n_out = 0;
      if (j == S - 1)
        walk_step_mode<1>(a, W, K, src, rs_in, nr, 0, nullptr, 0, 0, n_out, P.ovf, ar, as);
      else
        walk_step_mode<0>(a, W, K, src, rs_in, nr, 0, (int32_t *)(mine + P.lvl_off[j]), a.rs_out, P.lvl_cap[j],
                          n_out, P.ovf, ar, as);
      if (lane == 0) {
        K.cur[top] = cur + nr;
        if (j < S - 1) {
          K.n_lvl[j] = (int32_t)imin64(n_out, P.lvl_cap[j]);
          K.cur[j] = 0;
        }
      }
      __syncwarp();
      if (j < S - 1) top = j;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_down_sync(FULL_MASK, ar, o);
      as += __shfl_down_sync(FULL_MASK, as, o);
    }
    if (lane == 0) {
      if (S == 1 || ar) {
        atomicAdd(P.out + 2 * item.plan, ar);
        atomicAdd(P.out + 2 * item.plan + 1, as);
      }
      __threadfence();
      if (atomicAdd(P.plan_left + item.plan, ~0ull) == 1ull) P.plan_done[item.plan] = globaltimer_ns();
    }
    __syncwarp();
  }
}

size_t walk_smem_bytes(int tile_words, int max_steps) {
  return (size_t)BW_WARPS * walk_warp_bytes(tile_words, max_steps);
}

int walk_grid(int tile_words, int max_steps, int num_sms, int max_per_sm) {
  const size_t smem = walk_smem_bytes(tile_words, max_steps);
  cudaFuncSetAttribute(k_batchw, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batchw, BW_BLK, smem);
  if (per_sm < 1) per_sm = 1;
  if (max_per_sm > 0 && per_sm > max_per_sm) per_sm = max_per_sm;
  return num_sms * per_sm;
}

cudaError_t launch_batch_walk(const BatchParams &p, int grid, cudaStream_t s) {
  cudaFuncSetAttribute(k_batchw, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  g_launches++;
  k_batchw<<<grid, BW_BLK, walk_smem_bytes(p.tile_words, p.max_steps), s>>>(p);
  return cudaGetLastError();
}

}  // namespace dmk
