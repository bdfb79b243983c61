// Per-step join kernel, warp-centric: one iteration of Alg. 1 over R with no block barriers.
//
// Every warp owns 32-row tiles of R (the device helpers are in join_warp.cuh): it copies a tile
// into its own slice of shared memory (row stride join_row_stride(w), padding -1) while lane 0
// has the next one prefetched into L2, looks up each row's key group (one row per lane), scans
// the group sizes with shuffles, and walks the candidates 32 at a time (one per lane; a
// candidate finds its tile row by a binary search, with shuffles, over the rows' first-candidate
// offsets held in registers): motif-row loads, extra key equalities, injectivity of the new
// vertices against the whole row with int4 compares, back-edge bitmap tests, FP32 score.
// Survivors are appended to the warp's staging list with a ballot, new vertices included; when
// it fills, and at the end of the tile, the warp reserves its output range with one atomic and
// writes the rows with 16-byte stores (whole int4s of padded rows, 16-byte pieces of packed
// ones). Count mode adds each survivor's checksum instead: the terms of the row's own columns
// are summed once per tile row, so a survivor hashes only its new vertices. Warps never wait for
// each other, so the latency of one warp's dependent loads is hidden by the others.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "join_warp.cuh"
#include "kernels.h"

namespace dmk {

template <int MAXNEW, int MODE>
__global__ void __launch_bounds__(WJ_BLK, 4) k_joinw(const __grid_constant__ JoinArgs a) {
  constexpr bool STG = MAXNEW <= STAGE_NV;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int16_t code[MAXW];
  __shared__ int8_t ipos[MAXW];  // R column -> output position (-1: none)
  __shared__ int8_t npos[MAXM];  // new vertex -> output position
  __shared__ __align__(16) int32_t tq[MAXW];  // counted last step: 1 + output position of column c
  __shared__ unsigned long long s_red[WJ_WARPS];
  const bool seed = a.R == nullptr;
  const int w = a.w, wo = a.wo;
  const int wsv = join_row_stride(w);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const WarpSmem W = warp_smem(smem + (size_t)wid * warp_smem_bytes(wsv), wsv);
  for (int q = threadIdx.x; q < MAXW; q += WJ_BLK) ipos[q] = -1;
  __syncthreads();
  for (int q = threadIdx.x; q < wo; q += WJ_BLK) {
    const int col = a.src_col[q];
    code[q] = (int16_t)(col < w ? col : (0x100 | (col - w)));
    if (col < w) ipos[col] = (int8_t)q;
    else npos[col - w] = (int8_t)q;
    if (MODE == 1 && col < w) tq[col] = q + 1;
  }
  for (int r = lane; r < WT; r += 32)  // padding words never change afterwards
    for (int c = w; c < wsv; c++) W.rows[r * wsv + c] = -1;
  __syncthreads();
  griddep_wait();  // everything above touched shared memory only
  griddep_launch_dependents();
  const int64_t N = seed ? (a.seed_hi - a.seed_lo) : (a.n_dev ? imin64((int64_t)*a.n_dev, a.in_cap) : a.N);
  const int64_t ntiles = (N + WT - 1) / WT;
  const int64_t gw = (int64_t)blockIdx.x * WJ_WARPS + wid, nw = (int64_t)gridDim.x * WJ_WARPS;
  const int32_t *mrows = a.ix.rows;
  const int mw = a.ix.mw;
  unsigned long long acc_rows = 0, acc_sum = 0, acc_cand = 0, nsum = 0;

  for (int64_t t = gw; t < ntiles; t += nw) {
    const int64_t r0 = t * WT;
    const int nr = (int)imin64(WT, N - r0);
    int C;
    int g_start = 0, g_off = 0;  // this lane's tile row: its key group's first motif row and first candidate
    if (!seed) {
      const int rsi = a.rs_in ? a.rs_in : w;  // row stride of R
      const int32_t *src = a.R + r0 * rsi;
      const int ne = nr * w;
      if (lane == 0 && t + nw < ntiles) {  // the warp's next tile: bring it into L2 meanwhile
        const int32_t *nsrc = a.R + (t + nw) * WT * rsi;
        const uint32_t nb = (uint32_t)(imin64(WT, N - (t + nw) * WT) * rsi * 4) & ~15u;
        if (nb && (((uintptr_t)nsrc) & 15) == 0) l2_prefetch(nsrc, nb);
      }
      if (a.rs_in) {
        load_padded_tile(W.rows, wsv, src, nr, rsi);
      } else if ((((uintptr_t)src) & 15) == 0) {  // 16-byte loads; their words go to the padded rows
        const int n4 = ne >> 2;
        int r = (lane * 4) / w, c = lane * 4 - r * w;  // first word 4 * k of the lane, with carry
        const int dr = 128 / w, dc = 128 % w;
        for (int k = lane; k < n4; k += 32) {
          const int4 x = __ldg((const int4 *)src + k);
          int rr = r, cc = c;
          W.rows[rr * wsv + cc] = x.x;
          if (++cc == w) cc = 0, rr++;
          W.rows[rr * wsv + cc] = x.y;
          if (++cc == w) cc = 0, rr++;
          W.rows[rr * wsv + cc] = x.z;
          if (++cc == w) cc = 0, rr++;
          W.rows[rr * wsv + cc] = x.w;
          r += dr;
          c += dc;
          if (c >= w) {
            c -= w;
            r++;
          }
        }
        for (int e = n4 * 4 + lane; e < ne; e += 32) W.rows[(e / w) * wsv + e % w] = __ldg(src + e);
      } else {
        int r = lane / w, c = lane % w;  // element e = r * w + c, advanced with carry
        const int dr = 32 / w, dc = 32 % w;
        for (int e = lane; e < ne; e += 32) {
          W.rows[r * wsv + c] = __ldg(src + e);
          r += dr;
          c += dc;
          if (c >= w) {
            c -= w;
            r++;
          }
        }
      }
      if (a.Rs && lane < nr) W.rs[lane] = __ldg(a.Rs + r0 + lane);
      __syncwarp();
      int start = 0, len = 0;
      if (lane < nr) {
        const int32_t *row = W.rows + lane * wsv;
        if (MODE == 1) W.part[lane] = row_terms_last(row, w, tq);
        ix_lookup(a.ix, row[a.key_col[0]], a.ix.nkeys == 2 ? row[a.key_col[1]] : 0, start, len);
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += v;
      }
      C = __shfl_sync(FULL_MASK, incl, 31);
      g_start = start;
      g_off = incl - len;  // nondecreasing over the lanes; C for lanes past the tile
      __syncwarp();
    } else {
      C = nr;
    }
    acc_cand += lane == 0 ? (unsigned long long)C : 0ull;
    int nst = 0;
    for (int cb = 0; cb < C; cb += 32) {
      const int c = cb + lane;
      const bool valid = c < C;
      int r = 0, m = 0;
      if (!seed) {  // tile row of candidate c: the last row whose first candidate is at or before c
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
          if (__shfl_sync(FULL_MASK, g_off, r + step) <= c) r += step;
        const int ms = __shfl_sync(FULL_MASK, g_start, r), mo = __shfl_sync(FULL_MASK, g_off, r);
        if (valid) m = ms + (c - mo);
        else r = 0;
      } else if (valid) {
        m = (int)(a.seed_lo + r0 + c);
      }
      int32_t nv[MAXNEW];
      const int32_t *trow = mrows + (int64_t)m * mw;  // row 0 for idle lanes: a valid address
#pragma unroll
      for (int i = 0; i < MAXNEW; i++)
        if (i < nnew_of<MAXNEW>(a)) nv[i] = __ldg(trow + a.new_mpos[i]);
      float sc = 0.f;
      const bool ok = valid && wcheck<MAXNEW>(a, W, wsv, seed, r, m, nv, sc);
      if (MODE == 1) {
        if (ok) {
          unsigned long long p = seed ? 0ull : W.part[r];
#pragma unroll
          for (int i = 0; i < MAXNEW; i++)
            if (i < nnew_of<MAXNEW>(a)) p += pos_term(npos[i] + 1, nv[i]);
          acc_sum += dmix64(p + (unsigned long long)(uint32_t)wo);
          acc_rows++;
        }
      } else {
        const unsigned bal = __ballot_sync(FULL_MASK, ok);
        if (ok) {
          const int pos = nst + __popc(bal & lanemask_lt());
          W.st_r[pos] = r;
          W.st_m[pos] = m;
          W.st_s[pos] = sc;
#pragma unroll
          for (int i = 0; i < (STG ? MAXNEW : 0); i++)
            if (i < nnew_of<MAXNEW>(a)) W.st_nv[pos * STAGE_NV + i] = nv[i];
        }
        nst += __popc(bal);
        __syncwarp();
        if (nst > WSTAGE - 32) {
          if (STG && a.rs_out) wflush_padded<STG ? MAXNEW : 1>(a, W, wsv, nst, nsum);
          else wflush<STG>(a, W, code, wsv, nst, nsum);
          nst = 0;
        }
      }
    }
    if (MODE == 0 && nst > 0) {
      if (STG && a.rs_out) wflush_padded<STG ? MAXNEW : 1>(a, W, wsv, nst, nsum);
      else wflush<STG>(a, W, code, wsv, nst, nsum);
    }
    __syncwarp();  // the next tile overwrites this warp's rows
  }
  unsigned long long tc = block_sum_u64<WJ_BLK>(acc_cand, s_red);
  if (threadIdx.x == 0 && tc) atomicAdd(a.ctr + CTR_CAND, tc);
  if (a.out_next) {
    unsigned long long tn = block_sum_u64<WJ_BLK>(nsum, s_red);
    if (threadIdx.x == 0 && tn) atomicAdd(a.ctr + CTR_NEXT, tn);
  }
  if (MODE == 1) {
    unsigned long long tr = block_sum_u64<WJ_BLK>(acc_rows, s_red);
    unsigned long long ts = block_sum_u64<WJ_BLK>(acc_sum, s_red);
    if (threadIdx.x == 0) {
      if (tr) atomicAdd(a.ctr + CTR_ROWS, tr);
      atomicAdd(a.ctr + CTR_SUM, ts);
    }
  }
}

typedef void (*WJoinKernel)(JoinArgs);

// Variants: count or write mode x exactly 1, 2, 3 or 4 new vertices, or any other number (the
// wide variant, which reads it at run time; a step that maps no new vertex goes there too).
static int wjoin_variant(const JoinArgs &a) {
  return (a.mode == 1 ? 0 : 5) + (a.n_new >= 1 && a.n_new <= 4 ? a.n_new - 1 : 4);
}

static WJoinKernel pick_wjoin(const JoinArgs &a) {
  static const WJoinKernel ks[10] = {k_joinw<1, 1>, k_joinw<2, 1>, k_joinw<3, 1>, k_joinw<4, 1>, k_joinw<MAXM, 1>,
                                     k_joinw<1, 0>, k_joinw<2, 0>, k_joinw<3, 0>, k_joinw<4, 0>, k_joinw<MAXM, 0>};
  return ks[wjoin_variant(a)];
}

static size_t wjoin_smem(const JoinArgs &a) { return (size_t)WJ_WARPS * warp_smem_bytes(join_row_stride(a.w)); }

// The dynamic shared-memory limit is a per-device function attribute: set it once for each
// device that launches the kernels (contexts on several threads may race here harmlessly,
// the call is idempotent).
static void set_wjoin_attrs() {
  static std::atomic<unsigned long long> done{0};  // one bit per device ordinal below 64
  int dev = 0;
  cudaGetDevice(&dev);
  const bool cached = dev >= 0 && dev < 64;  // higher ordinals set the attributes on every call
  const unsigned long long bit = cached ? 1ull << dev : 0ull;
  if (cached && (done.load() & bit)) return;
  WJoinKernel ks[] = {k_joinw<1, 1>, k_joinw<2, 1>, k_joinw<3, 1>, k_joinw<4, 1>, k_joinw<MAXM, 1>,
                      k_joinw<1, 0>, k_joinw<2, 0>, k_joinw<3, 0>, k_joinw<4, 0>, k_joinw<MAXM, 0>};
  for (auto k : ks) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (cached) done.fetch_or(bit);
}

int wjoin_grid(const JoinArgs &a, int num_sms) {
  set_wjoin_attrs();
  WJoinKernel k = pick_wjoin(a);
  int64_t rows = a.R == nullptr ? a.seed_hi - a.seed_lo : (a.n_dev ? INT64_MAX / 2 : a.N);
  int64_t blocks_needed = (rows + (int64_t)WT * WJ_WARPS - 1) / ((int64_t)WT * WJ_WARPS);
  // resident blocks per SM for this variant and row stride, asked of the runtime once (the
  // query costs host time on every launch otherwise); every device of the process is taken to
  // be of one architecture
  static std::atomic<int> occ[10][MAXW / 4 + 2];
  const int slot = join_row_stride(a.w) / 4;
  int per_sm = occ[wjoin_variant(a)][slot].load(std::memory_order_relaxed);
  if (per_sm <= 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WJ_BLK, wjoin_smem(a));
    if (per_sm < 1) per_sm = 1;
    occ[wjoin_variant(a)][slot].store(per_sm, std::memory_order_relaxed);
  }
  int64_t g = (int64_t)num_sms * per_sm;
  if (blocks_needed < g) g = blocks_needed;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_wjoin(const JoinArgs &a, int grid, cudaStream_t s, bool pdl) {
  set_wjoin_attrs();
  WJoinKernel k = pick_wjoin(a);
  g_launches++;
  if (pdl) return launch_pdl(k, dim3(grid < 1 ? 1 : grid), dim3(WJ_BLK), wjoin_smem(a), s, a);
  k<<<grid < 1 ? 1 : grid, WJ_BLK, wjoin_smem(a), s>>>(a);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------
// The last two steps of a counted plan in one kernel. Step A (the plan's second-to-last join,
// written in working-column order) and step B (the last join, counted) run back to back on
// every tile: each survivor of A is assembled straight into a shared-memory tile of B rows
// (the A row, then A's new vertices, padded with -1 like any tile), together with the sum of
// its checksum terms (the A row's terms, summed once per A row, plus those of the new
// vertices), and when B's tile cannot take another round of A it is joined and counted as in
// k_joinw's counted step. The table between A and B, the largest of a path-like plan, is
// never written to or read from global memory.

struct FSmem {
  int32_t *rowsA, *rowsB;               // WT x wsA, WT x wsB
  unsigned long long *partA, *partB;    // checksum terms of each A row / B row
};

__host__ __device__ __forceinline__ size_t fused_warp_bytes(int wsA, int wsB) {
  size_t b = (size_t)WT * wsA * 4 + (size_t)WT * wsB * 4;
  b += (size_t)WT * 8 * 2;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ FSmem fused_smem(unsigned char *base, int wsA, int wsB) {
  FSmem m;
  size_t off = 0;
  m.rowsA = (int32_t *)(base + off);
  off += (size_t)WT * wsA * 4;
  m.rowsB = (int32_t *)(base + off);
  off += (size_t)WT * wsB * 4;
  m.partA = (unsigned long long *)(base + off);
  m.partB = m.partA + WT;
  return m;
}

struct FusedArgs {
  JoinArgs a, b;
};

// Look up the key groups of the nr rows of a shared tile (lane = row): g_start = the first motif
// row of the lane's group, g_off = the lane's first candidate (nondecreasing over the lanes; C
// for lanes past the tile). Returns the number of candidates C.
__device__ __forceinline__ int tile_groups(const JoinArgs &a, const int32_t *rows, int ws, int nr, int &g_start,
                                           int &g_off) {
  const int lane = threadIdx.x & 31;
  int start = 0, len = 0;
  if (lane < nr) {
    const int32_t *row = rows + lane * ws;
    ix_lookup(a.ix, row[a.key_col[0]], a.ix.nkeys == 2 ? row[a.key_col[1]] : 0, start, len);
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += v;
  }
  g_start = start;
  g_off = incl - len;
  __syncwarp();  // shared words the lanes wrote before (checksum terms) are read by others next
  return __shfl_sync(FULL_MASK, incl, 31);
}

// Join and count the nb rows of the B tile (step B, its rows' checksum terms in partB).
template <int NB>
__device__ __forceinline__ void count_b_tile(const JoinArgs &b, const FSmem &F, int wsB, int nb, const int32_t *tq,
                                             unsigned long long &acc_rows, unsigned long long &acc_sum,
                                             unsigned long long &acc_cand) {
  const int lane = threadIdx.x & 31;
  int g_start, g_off;
  const int C = tile_groups(b, F.rowsB, wsB, nb, g_start, g_off);
  acc_cand += lane == 0 ? (unsigned long long)C : 0ull;
  WarpSmem W{};
  W.rows = F.rowsB;
  const int w = b.w;
  for (int cb = 0; cb < C; cb += 32) {
    int r, m;
    round_rows(g_start, g_off, cb, C, r, m);
    const bool valid = cb + lane < C;
    int32_t nv[NB];
    const int32_t *trow = b.ix.rows + (int64_t)m * b.ix.mw;
#pragma unroll
    for (int i = 0; i < NB; i++) nv[i] = __ldg(trow + b.new_mpos[i]);
    float sc = 0.f;
    if (valid && wcheck<NB>(b, W, wsB, false, r, m, nv, sc)) {
      unsigned long long p = F.partB[r];
#pragma unroll
      for (int i = 0; i < NB; i++) p += pos_term(tq[w + i], nv[i]);
      acc_sum += dmix64(p + (unsigned long long)(uint32_t)b.wo);
      acc_rows++;
    }
  }
  __syncwarp();  // the B tile is refilled next
}

template <int NA, int NB>
__global__ void __launch_bounds__(WJ_BLK, 4) k_joinf(const __grid_constant__ FusedArgs f) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) int32_t tq[MAXW];  // 1 + B's output position of each B working column
  __shared__ unsigned long long s_red[WJ_WARPS];
  const JoinArgs &a = f.a, &b = f.b;
  const bool seed = a.R == nullptr;
  const int wA = a.w, wB = b.w;  // wB = wA + NA
  const int wsA = join_row_stride(wA), wsB = join_row_stride(wB);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const FSmem F = fused_smem(smem + (size_t)wid * fused_warp_bytes(wsA, wsB), wsA, wsB);
  for (int q = threadIdx.x; q < b.wo; q += WJ_BLK) tq[b.src_col[q]] = q + 1;
  for (int r = lane; r < WT; r += 32) {  // padding words never change afterwards
    for (int c = wA; c < wsA; c++) F.rowsA[r * wsA + c] = -1;
    for (int c = wB; c < wsB; c++) F.rowsB[r * wsB + c] = -1;
  }
  __syncthreads();
  griddep_wait();  // everything above touched shared memory only
  griddep_launch_dependents();
  const int64_t N = seed ? (a.seed_hi - a.seed_lo) : (a.n_dev ? imin64((int64_t)*a.n_dev, a.in_cap) : a.N);
  const int64_t ntiles = (N + WT - 1) / WT;
  const int64_t gw = (int64_t)blockIdx.x * WJ_WARPS + wid, nw = (int64_t)gridDim.x * WJ_WARPS;
  unsigned long long rows_a = 0, cand_a = 0, acc_rows = 0, acc_sum = 0, cand_b = 0;
  WarpSmem W{};
  W.rows = F.rowsA;
  int nb = 0;  // rows in the B tile
  for (int64_t t = gw; t < ntiles; t += nw) {
    const int64_t r0 = t * WT;
    const int nr = (int)imin64(WT, N - r0);
    int C;
    int ga_start = 0, ga_off = 0;
    if (!seed) {
      const int rsi = a.rs_in ? a.rs_in : wA;  // row stride of R
      const int32_t *src = a.R + r0 * rsi;
      if (lane == 0 && t + nw < ntiles) {  // the warp's next tile: bring it into L2 meanwhile
        const int32_t *nsrc = a.R + (t + nw) * WT * rsi;
        const uint32_t nbytes = (uint32_t)(imin64(WT, N - (t + nw) * WT) * rsi * 4) & ~15u;
        if (nbytes && (((uintptr_t)nsrc) & 15) == 0) l2_prefetch(nsrc, nbytes);
      }
      if (a.rs_in) {
        load_padded_tile(F.rowsA, wsA, src, nr, rsi);
      } else {
        int r = lane / wA, c = lane % wA;  // element e = r * wA + c, advanced with carry
        const int dr = 32 / wA, dc = 32 % wA;
        for (int e = lane; e < nr * wA; e += 32) {
          F.rowsA[r * wsA + c] = __ldg(src + e);
          r += dr;
          c += dc;
          if (c >= wA) {
            c -= wA;
            r++;
          }
        }
      }
      __syncwarp();
      if (lane < nr) F.partA[lane] = row_terms_last(F.rowsA + lane * wsA, wA, tq);  // B positions
      C = tile_groups(a, F.rowsA, wsA, nr, ga_start, ga_off);
    } else {
      C = nr;
    }
    cand_a += lane == 0 ? (unsigned long long)C : 0ull;
    for (int cb = 0; cb < C; cb += 32) {
      int r = 0, m = 0;
      if (seed) {
        if (cb + lane < C) m = (int)(a.seed_lo + r0 + cb + lane);
      } else {
        round_rows(ga_start, ga_off, cb, C, r, m);
      }
      const bool valid = cb + lane < C;
      int32_t nv[NA];
      const int32_t *trow = a.ix.rows + (int64_t)m * a.ix.mw;
#pragma unroll
      for (int i = 0; i < NA; i++) nv[i] = __ldg(trow + a.new_mpos[i]);
      float sc = 0.f;
      const bool ok = valid && wcheck<NA>(a, W, wsA, seed, r, m, nv, sc);
      const unsigned bal = __ballot_sync(FULL_MASK, ok);
      const int K = __popc(bal);
      if (nb + K > WT) {  // B's tile is full: join and count it first
        count_b_tile<NB>(b, F, wsB, nb, tq, acc_rows, acc_sum, cand_b);
        nb = 0;
      }
      if (ok) {  // the survivor's row in B's tile: the A row, then A's new vertices
        const int slot = nb + __popc(bal & lanemask_lt());
        int32_t *d = F.rowsB + slot * wsB;
        unsigned long long p = seed ? 0ull : F.partA[r];
        if (!seed) {
          const int4 *s4 = (const int4 *)(F.rowsA + r * wsA);
          int4 *d4 = (int4 *)d;
          for (int c4 = 0; c4 < (wA + 3) >> 2; c4++) d4[c4] = s4[c4];  // -1 beyond wA, overwritten below
        }
#pragma unroll
        for (int i = 0; i < NA; i++) {
          d[wA + i] = nv[i];
          p += pos_term(tq[wA + i], nv[i]);
        }
        F.partB[slot] = p;
      }
      nb += K;
      rows_a += lane == 0 ? (unsigned long long)K : 0ull;
      __syncwarp();  // B's tile is read next
    }
    __syncwarp();  // the next tile overwrites this warp's A rows
  }
  if (nb > 0) count_b_tile<NB>(b, F, wsB, nb, tq, acc_rows, acc_sum, cand_b);
  unsigned long long t0 = block_sum_u64<WJ_BLK>(rows_a, s_red);
  unsigned long long t1 = block_sum_u64<WJ_BLK>(cand_a, s_red);
  unsigned long long t2 = block_sum_u64<WJ_BLK>(cand_b, s_red);
  unsigned long long t3 = block_sum_u64<WJ_BLK>(acc_rows, s_red);
  unsigned long long t4 = block_sum_u64<WJ_BLK>(acc_sum, s_red);
  if (threadIdx.x == 0) {
    if (t0) atomicAdd(a.ctr + CTR_ROWS, t0);
    if (t1) atomicAdd(a.ctr + CTR_CAND, t1);
    if (t2) atomicAdd(b.ctr + CTR_CAND, t2);
    if (t3) atomicAdd(b.ctr + CTR_ROWS, t3);
    atomicAdd(b.ctr + CTR_SUM, t4);
  }
}

typedef void (*FJoinKernel)(FusedArgs);

static FJoinKernel pick_fused(int na, int nb) {
  static const FJoinKernel ks[4][4] = {
      {k_joinf<1, 1>, k_joinf<1, 2>, k_joinf<1, 3>, k_joinf<1, 4>},
      {k_joinf<2, 1>, k_joinf<2, 2>, k_joinf<2, 3>, k_joinf<2, 4>},
      {k_joinf<3, 1>, k_joinf<3, 2>, k_joinf<3, 3>, k_joinf<3, 4>},
      {k_joinf<4, 1>, k_joinf<4, 2>, k_joinf<4, 3>, k_joinf<4, 4>}};
  return ks[na - 1][nb - 1];
}

static size_t fused_smem(const JoinArgs &a, const JoinArgs &b) {
  return (size_t)WJ_WARPS * fused_warp_bytes(join_row_stride(a.w), join_row_stride(b.w));
}

bool fused_ok(const JoinArgs &a, const JoinArgs &b) {
  return a.mode == 0 && b.mode == 1 && a.n_new >= 1 && a.n_new <= 4 && b.n_new >= 1 && b.n_new <= 4 &&
         b.w == a.w + a.n_new && a.wo == b.w && b.R == nullptr && !a.scored && !b.scored && a.n_shards <= 1 &&
         fused_smem(a, b) <= 200 * 1024;
}

cudaError_t launch_fused(const JoinArgs &a, const JoinArgs &b, int num_sms, cudaStream_t s, bool pdl) {
  FJoinKernel k = pick_fused(a.n_new, b.n_new);
  const size_t smem = fused_smem(a, b);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, WJ_BLK, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t rows = a.R == nullptr ? a.seed_hi - a.seed_lo : (a.n_dev ? INT64_MAX / 2 : a.N);
  int64_t g = (int64_t)num_sms * per_sm, need = (rows + (int64_t)WT * WJ_WARPS - 1) / ((int64_t)WT * WJ_WARPS);
  if (need < g) g = need;
  if (g < 1) g = 1;
  FusedArgs fa;
  fa.a = a;
  fa.b = b;
  g_launches++;
  if (pdl) return launch_pdl(k, dim3((unsigned)g), dim3(WJ_BLK), smem, s, fa);
  k<<<(unsigned)g, WJ_BLK, smem, s>>>(fa);
  return cudaGetLastError();
}

}  // namespace dmk
