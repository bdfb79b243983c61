// Per-step join kernel, warp-centric: one iteration of Alg. 1 over R with no block barriers.
//
// Every warp owns 32-row tiles of R: it copies a tile into its own slice of shared memory
// (row stride join_row_stride(w), padding -1), looks up each row's key group (one row per lane),
// scans the group sizes with shuffles, and walks the candidates 32 at a time (one per lane; a
// candidate finds its tile row by a binary search, with shuffles, over the rows' first-candidate
// offsets held in registers): motif-row loads, extra key equalities, injectivity of the new
// vertices against the whole row
// with int4 compares, back-edge bitmap tests, FP32 score. Survivors are appended to the warp's
// staging list with a ballot, new vertices included; when it fills, and at the end of the
// tile, the warp reserves its output range with one atomic and writes the rows element by
// element from shared memory, lanes on consecutive words. Count mode adds each survivor's
// checksum instead: the terms of the row's own columns are summed once per tile row, so a
// survivor hashes only its new vertices. Warps never wait for each other, so the latency of
// one warp's dependent loads is hidden by the others.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "join_device.cuh"
#include "kernels.h"

namespace dmk {

constexpr int WJ_BLK = 256, WJ_WARPS = WJ_BLK / 32, WT = 32, WSTAGE = 96, STAGE_NV = 4;

struct WarpSmem {
  int32_t *rows;              // WT x wsv
  unsigned long long *part;   // WT checksum partial sums (count mode)
  float *rs;                  // WT scores
  int32_t *st_r, *st_m;       // WSTAGE survivors: tile row, motif row
  float *st_s;                // WSTAGE scores
  int32_t *st_nv;             // WSTAGE x STAGE_NV new vertices
};

// NST: entries of the staging list (WSTAGE in k_joinw)
template <int NST = WSTAGE>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int wsv) {
  size_t b = (size_t)WT * wsv * 4;
  b += (size_t)WT * 8 + (size_t)WT * 4;
  b = (b + 15) / 16 * 16;
  b += (size_t)NST * 12 + (size_t)NST * STAGE_NV * 4;
  return (b + 15) / 16 * 16;
}

template <int NST = WSTAGE>
__device__ __forceinline__ WarpSmem warp_smem(unsigned char *base, int wsv) {
  WarpSmem m;
  size_t off = 0;
  m.rows = (int32_t *)(base + off);
  off += (size_t)WT * wsv * 4;
  m.part = (unsigned long long *)(base + off);
  off += (size_t)WT * 8;
  m.rs = (float *)(base + off);
  off += (size_t)WT * 4;
  off = (off + 15) / 16 * 16;
  m.st_r = (int32_t *)(base + off);
  m.st_m = m.st_r + NST;
  m.st_s = (float *)(m.st_m + NST);
  m.st_nv = (int32_t *)(m.st_s + NST);
  return m;
}

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16); the data
// stays in global memory, nothing waits for it.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Whether any of the four ids of x equals one of nv[0 .. NN), folded into hit: the compares
// accumulate into one predicate (setp with .or), one instruction a compare.
template <int NN>
__device__ __forceinline__ bool any_eq4(bool hit, const int4 x, const int32_t *nv) {
  uint32_t r;
  if (NN == 1)
    asm("{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
        " setp.eq.or.s32 p, %2, %6, p;\n setp.eq.or.s32 p, %3, %6, p;\n"
        " setp.eq.or.s32 p, %4, %6, p;\n setp.eq.or.s32 p, %5, %6, p;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r) : "r"((uint32_t)hit), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w), "r"(nv[0]));
  else if (NN == 2)
    asm("{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
        " setp.eq.or.s32 p, %2, %6, p;\n setp.eq.or.s32 p, %3, %6, p;\n"
        " setp.eq.or.s32 p, %4, %6, p;\n setp.eq.or.s32 p, %5, %6, p;\n"
        " setp.eq.or.s32 p, %2, %7, p;\n setp.eq.or.s32 p, %3, %7, p;\n"
        " setp.eq.or.s32 p, %4, %7, p;\n setp.eq.or.s32 p, %5, %7, p;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r) : "r"((uint32_t)hit), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w), "r"(nv[0]), "r"(nv[1]));
  else if (NN == 3)
    asm("{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
        " setp.eq.or.s32 p, %2, %6, p;\n setp.eq.or.s32 p, %3, %6, p;\n"
        " setp.eq.or.s32 p, %4, %6, p;\n setp.eq.or.s32 p, %5, %6, p;\n"
        " setp.eq.or.s32 p, %2, %7, p;\n setp.eq.or.s32 p, %3, %7, p;\n"
        " setp.eq.or.s32 p, %4, %7, p;\n setp.eq.or.s32 p, %5, %7, p;\n"
        " setp.eq.or.s32 p, %2, %8, p;\n setp.eq.or.s32 p, %3, %8, p;\n"
        " setp.eq.or.s32 p, %4, %8, p;\n setp.eq.or.s32 p, %5, %8, p;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r) : "r"((uint32_t)hit), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w), "r"(nv[0]), "r"(nv[1]), "r"(nv[2]));
  else
    asm("{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n"
        " setp.eq.or.s32 p, %2, %6, p;\n setp.eq.or.s32 p, %3, %6, p;\n"
        " setp.eq.or.s32 p, %4, %6, p;\n setp.eq.or.s32 p, %5, %6, p;\n"
        " setp.eq.or.s32 p, %2, %7, p;\n setp.eq.or.s32 p, %3, %7, p;\n"
        " setp.eq.or.s32 p, %4, %7, p;\n setp.eq.or.s32 p, %5, %7, p;\n"
        " setp.eq.or.s32 p, %2, %8, p;\n setp.eq.or.s32 p, %3, %8, p;\n"
        " setp.eq.or.s32 p, %4, %8, p;\n setp.eq.or.s32 p, %5, %8, p;\n"
        " setp.eq.or.s32 p, %2, %9, p;\n setp.eq.or.s32 p, %3, %9, p;\n"
        " setp.eq.or.s32 p, %4, %9, p;\n setp.eq.or.s32 p, %5, %9, p;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"((uint32_t)hit), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w), "r"(nv[0]), "r"(nv[1]), "r"(nv[2]), "r"(nv[3]));
  return r != 0;
}

// Number of new vertices of a step: exactly MAXNEW in the variants for 1 to 4 (so the loops over
// them unroll without runtime guards), read from the arguments in the wide variant.
template <int MAXNEW>
__device__ __forceinline__ int nnew_of(const JoinArgs &a) {
  return MAXNEW <= STAGE_NV ? MAXNEW : a.n_new;
}

// New vertex i (uniform over the warp) of a candidate, from the preloaded registers.
template <int MAXNEW>
__device__ __forceinline__ int32_t pick_nv(const int32_t (&nv)[MAXNEW], int i) {
  int32_t v = nv[0];
#pragma unroll
  for (int k = 1; k < MAXNEW; k++)
    if (i == k) v = nv[k];
  return v;
}

// Check one candidate against row r of the warp tile (new vertices preloaded).
template <int MAXNEW>
__device__ __forceinline__ bool wcheck(const JoinArgs &a, const WarpSmem &W, int wsv, bool seed, int r, int m,
                                       const int32_t (&nv)[MAXNEW], float &sc) {
  const int32_t *rrow = W.rows + r * wsv;
  const int32_t *trow = a.ix.rows + (int64_t)m * a.ix.mw;
  const int nn = nnew_of<MAXNEW>(a);
  bool ok = true;
  if (seed && a.n_shards > 1) ok = (uint32_t)nv[0] % (uint32_t)a.n_shards == (uint32_t)a.shard;
  for (int i = 0; i < a.n_chk; i++) ok &= __ldg(trow + a.chk_mpos[i]) == rrow[a.chk_col[i]];
  if (ok && !seed) {  // FilterOverlappingNodes: one pass over the row for all new vertices
    const int4 *r4 = (const int4 *)rrow;
    bool hit = false;
#pragma unroll 2
    for (int c4 = 0; c4 < (a.w + 3) >> 2; c4++) {
      const int4 x = r4[c4];
      if (MAXNEW <= STAGE_NV) {
        hit = any_eq4<MAXNEW>(hit, x, nv);
      } else {
#pragma unroll
        for (int i = 0; i < MAXNEW; i++)
          if (i < nn) hit |= (x.x == nv[i]) | (x.y == nv[i]) | (x.z == nv[i]) | (x.w == nv[i]);
      }
    }
    ok = !hit;
  }
  sc = 0.f;
  if (a.scored) {
    sc = (!seed && a.Rs) ? W.rs[r] : 0.f;
    if (a.ix.score) sc += __ldg(a.ix.score + m);
    if (a.qerr) {
#pragma unroll
      for (int i = 0; i < MAXNEW; i++)
        if (i < nn) sc += __ldg(a.qerr + nv[i]);
    }
  }
  for (int e = 0; e < a.n_be && ok; e++) {
    const int ca = a.be_a[e], cb = a.be_b[e];
    int32_t va, vb;
    if (MAXNEW <= STAGE_NV) {  // new vertices from the registers
      va = ca < a.w ? rrow[ca] : pick_nv<MAXNEW>(nv, ca - a.w);
      vb = cb < a.w ? rrow[cb] : pick_nv<MAXNEW>(nv, cb - a.w);
    } else {
      va = join_value(a, rrow, trow, ca);
      vb = join_value(a, rrow, trow, cb);
    }
    ok = adjacent(a, va, vb);
    if (ok && a.scored && a.eerr) sc += edge_weight(a, va, vb);
  }
  if (ok && a.induced) ok = induced_ok<MAXNEW>(a, rrow, nv);
  if (sc > a.prune) ok = false;
  return ok;
}

// Sum of the checksum terms of a tile row in a counted last step, where every working column
// is an output column: tq[c] = 1 + the output position of column c (int4-aligned, padded), so
// one 16-byte read gives the positions of four columns; two accumulators keep eight terms
// independent per iteration.
__device__ __forceinline__ unsigned long long row_terms_last(const int32_t *row, int w, const int32_t *tq) {
  const int4 *r4 = (const int4 *)row;
  const int4 *q4 = (const int4 *)tq;
  unsigned long long p0 = 0, p1 = 0;
  const int nq = w >> 2;
  int c4 = 0;
  for (; c4 + 1 < nq; c4 += 2) {
    const int4 x = r4[c4], y = r4[c4 + 1], qx = q4[c4], qy = q4[c4 + 1];
    p0 += pos_term(qx.x, x.x) +
          pos_term(qx.y, x.y);
    p1 += pos_term(qx.z, x.z) +
          pos_term(qx.w, x.w);
    p0 += pos_term(qy.x, y.x) +
          pos_term(qy.y, y.y);
    p1 += pos_term(qy.z, y.z) +
          pos_term(qy.w, y.w);
  }
  if (c4 < nq) {
    const int4 x = r4[c4], qx = q4[c4];
    p0 += pos_term(qx.x, x.x) +
          pos_term(qx.y, x.y);
    p1 += pos_term(qx.z, x.z) +
          pos_term(qx.w, x.w);
  }
  for (int c = 4 * nq; c < w; c++) p0 += pos_term(tq[c], row[c]);
  return p0 + p1;
}

// Copy nr rows of a padded table (stride rs = 4q words, 16-byte aligned rows, padding -1) into a
// warp tile (stride wsv >= rs, a multiple of 4): whole int4s; the tile's words past rs keep
// their -1.
__device__ __forceinline__ void load_padded_tile(int32_t *rows, int wsv, const int32_t *src, int nr, int rs) {
  const int lane = threadIdx.x & 31;
  const int q = rs >> 2, qs = wsv >> 2, n4 = nr * q;
  const int4 *s4 = (const int4 *)src;
  int4 *d4 = (int4 *)rows;
  if (qs == q) {
    for (int k = lane; k < n4; k += 32) d4[k] = __ldg(s4 + k);
  } else {
    int r = lane / q, c = lane - r * q;  // int4 k = r * q + c, advanced with carry
    const int dr = 32 / q, dc = 32 % q;
    for (int k = lane; k < n4; k += 32) {
      d4[r * qs + c] = __ldg(s4 + k);
      r += dr;
      c += dc;
      if (c >= q) {
        c -= q;
        r++;
      }
    }
  }
}

// Word q of staged survivor s's output row. code[q] < 0x100: working column of the R row; else
// 0x100 | index of the new vertex (read from the staging area when STG, else from the motif row).
template <bool STG>
__device__ __forceinline__ int32_t out_word(const JoinArgs &a, const WarpSmem &W, const int16_t *code, int wsv, int s,
                                            int q) {
  const int cd = code[q];
  if (cd < 0x100) return W.rows[W.st_r[s] * wsv + cd];
  if (STG) return W.st_nv[s * STAGE_NV + (cd & 0xff)];
  return __ldg(a.ix.rows + (int64_t)W.st_m[s] * a.ix.mw + a.new_mpos[cd & 0xff]);
}

// Reserve the output range of n staged survivors (one atomic); returns its first row and sets Kc
// to the rows that fit the output (the overflow flag is raised for the rest). Writes the
// survivors' scores and next-step candidate counts.
__device__ __forceinline__ long long wreserve(const JoinArgs &a, const WarpSmem &W, int wsv, int n, int &Kc,
                                              unsigned long long &nsum) {
  const int lane = threadIdx.x & 31;
  long long base = 0;
  if (lane == 0) base = (long long)atomicAdd(a.ctr + CTR_ROWS, (unsigned long long)n);
  base = __shfl_sync(FULL_MASK, base, 0);
  Kc = n;
  if (base + n > a.out_cap) {
    Kc = (int)imax64(0, a.out_cap - base);
    if (lane == 0) atomicOr(a.ctr + CTR_OVF, 1ull);
  }
  const int32_t *mrows = a.ix.rows;
  const int mw = a.ix.mw;
  for (int i = lane; i < Kc; i += 32) {
    if (a.outs) a.outs[base + i] = W.st_s[i];
    if (a.out_next) {
      const int32_t *rrow = W.rows + W.st_r[i] * wsv;
      const int32_t *trow = mrows + (int64_t)W.st_m[i] * mw;
      int32_t st, ln;
      ix_lookup(a.nx, join_value(a, rrow, trow, a.nx_key_col[0]),
                a.nx.nkeys == 2 ? join_value(a, rrow, trow, a.nx_key_col[1]) : 0, st, ln);
      a.out_next[base + i] = ln;
      nsum += (unsigned long long)ln;
    }
  }
  return base;
}

// Write Kc staged survivors into a padded table at dst (row stride rs = 4 q4 words, the rows
// 16-byte aligned): output int4 k of survivor s is int4 k of its tile row (the row's w words,
// then -1 padding) with the survivor's new vertices put at positions w .. w + NN - 1; int4s
// past the tile row are -1. Lanes write consecutive int4s.
template <int NN>
__device__ __forceinline__ void wwrite_padded(const WarpSmem &W, int wsv, int w, int Kc, int32_t *dst_rows, int rs) {
  const int lane = threadIdx.x & 31;
  const int q4 = rs >> 2, wq = wsv >> 2;
  int4 *dst = (int4 *)dst_rows;
  const int n4 = Kc * q4;
  int s = lane / q4, k = lane - s * q4;  // int4 e = s * q4 + k, advanced with carry
  const int ds = 32 / q4, dk = 32 % q4;
  for (int e = lane; e < n4; e += 32) {
    int4 v = make_int4(-1, -1, -1, -1);
    if (k < wq) v = *(const int4 *)(W.rows + W.st_r[s] * wsv + 4 * k);
    const int p = 4 * k - w;  // new-vertex index of v.x
    if (p > -4 && p < NN) {
      const int32_t *nvs = W.st_nv + s * STAGE_NV;
      if (p >= 0) v.x = nvs[p];
      if (p + 1 >= 0 && p + 1 < NN) v.y = nvs[p + 1];
      if (p + 2 >= 0 && p + 2 < NN) v.z = nvs[p + 2];
      if (p + 3 < NN) v.w = nvs[p + 3];
    }
    dst[e] = v;
    s += ds;
    k += dk;
    if (k >= q4) {
      k -= q4;
      s++;
    }
  }
}

// Write Kc staged survivors as packed rows of wo words at dst (word q of a row from code[q]):
// consecutive 16-byte pieces from the first 16-byte boundary, scalar head and tail.
template <bool STG>
__device__ __forceinline__ void wwrite(const JoinArgs &a, const WarpSmem &W, const int16_t *code, int wsv, int Kc,
                                       int32_t *dst, int wo) {
  const int lane = threadIdx.x & 31;
  const int ne = Kc * wo;
  const int h = min((int)((4 - (((uintptr_t)dst >> 2) & 3)) & 3), ne);  // words before a 16-byte boundary
  if (lane < h) dst[lane] = out_word<STG>(a, W, code, wsv, lane / wo, lane % wo);
  const int n4 = (ne - h) >> 2;
  int4 *d4 = (int4 *)(dst + h);
  int s = (h + 4 * lane) / wo, q = h + 4 * lane - s * wo;  // word h + 4 * k of the lane, with carry
  const int ds = 128 / wo, dq = 128 % wo;
  for (int k = lane; k < n4; k += 32) {
    int4 v;
    int ss = s, qq = q;
    v.x = out_word<STG>(a, W, code, wsv, ss, qq);
    if (++qq == wo) qq = 0, ss++;
    v.y = out_word<STG>(a, W, code, wsv, ss, qq);
    if (++qq == wo) qq = 0, ss++;
    v.z = out_word<STG>(a, W, code, wsv, ss, qq);
    if (++qq == wo) qq = 0, ss++;
    v.w = out_word<STG>(a, W, code, wsv, ss, qq);
    d4[k] = v;
    s += ds;
    q += dq;
    if (q >= wo) {
      q -= wo;
      s++;
    }
  }
  for (int e = h + 4 * n4 + lane; e < ne; e += 32) dst[e] = out_word<STG>(a, W, code, wsv, e / wo, e % wo);
}

// Flush the warp's staged survivors into the step's output (one atomic reservation).
template <int NN>
__device__ __forceinline__ void wflush_padded(const JoinArgs &a, const WarpSmem &W, int wsv, int n,
                                              unsigned long long &nsum) {
  int Kc;
  const long long base = wreserve(a, W, wsv, n, Kc, nsum);
  wwrite_padded<NN>(W, wsv, a.w, Kc, a.out + base * a.rs_out, a.rs_out);
  __syncwarp();
}

template <bool STG>
__device__ __forceinline__ void wflush(const JoinArgs &a, const WarpSmem &W, const int16_t *code, int wsv, int n,
                                       unsigned long long &nsum) {
  int Kc;
  const long long base = wreserve(a, W, wsv, n, Kc, nsum);
  wwrite<STG>(a, W, code, wsv, Kc, a.out + base * a.wo, a.wo);
  __syncwarp();
}

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

// Candidate c = cb + lane of a tile: its tile row r (the last row whose first candidate is at or
// before c, found by binary search over the lanes' g_off) and its motif row m; 0 and 0 past C.
__device__ __forceinline__ void round_rows(int g_start, int g_off, int cb, int C, int &r, int &m) {
  const int c = cb + (threadIdx.x & 31);
  r = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1)
    if (__shfl_sync(FULL_MASK, g_off, r + step) <= c) r += step;
  const int ms = __shfl_sync(FULL_MASK, g_start, r), mo = __shfl_sync(FULL_MASK, g_off, r);
  m = 0;
  if (c < C) m = ms + (c - mo);
  else r = 0;
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

// ---------------------------------------------------------------------------------------
// Persistent batch kernel with one depth-first walk per warp (count + checksum for many plans
// on one data graph; the "warp walk" block shape of dm_match_batch). Every warp takes work
// items (plan, rows of the motif table of its first slice) from the global counter and runs
// each one through the plan's steps on its own: level j of the warp's scratch holds step j's
// output for the current 32-row tile of level j - 1 (at most 32 x the step's largest key group
// rows), and the last step is counted. A step over one tile is k_joinw's warp tile -- the same
// lookup, candidate walk, checks, staging and 16-byte flush -- so no warp waits for another and
// no block barrier is taken. Level rows are written and read back within the launch, so they
// are read with plain (coherent) loads, never through the read-only cache path.

// 64-entry staging lists: the smaller footprint keeps more walks resident than a longer list
// would save in flushes (the walks are latency-bound)
constexpr int BW_WARPS = BW_WALK_WARPS, BW_BLK = 32 * BW_WARPS, BW_STAGE = 64;

struct WalkSmem {
  int32_t *tq;           // MAXW: counted step, 1 + output position of each working column
  int16_t *code;         // MAXW (over tq: a step is either written or counted): packed flush,
                         // output position -> working column / new vertex
  int8_t *npos;          // MAXM: counted step, output position of each new vertex
  int32_t *n_lvl, *cur;  // per level: rows held, rows already joined into the next level
};

__host__ __device__ __forceinline__ size_t walk_warp_bytes(int ws_max, int max_steps) {
  size_t b = warp_smem_bytes<BW_STAGE>(ws_max) + (size_t)MAXW * 4 + MAXM;
  b = (b + 15) / 16 * 16 + (size_t)max_steps * 8;
  return (b + 15) / 16 * 16;
}

__device__ __forceinline__ WalkSmem walk_smem(unsigned char *base, int ws_max, int max_steps) {
  WalkSmem k;
  size_t off = warp_smem_bytes<BW_STAGE>(ws_max);  // a multiple of 16
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
__device__ __forceinline__ void walk_tile(const JoinArgs &a, unsigned char *wbase, const WalkSmem &K,
                                          const int32_t *src, int rs_in, int nr, int64_t m0, int32_t *out, int rs_out,
                                          int64_t cap, int64_t &n_out, unsigned long long *ovf,
                                          unsigned long long &acc_rows, unsigned long long &acc_sum) {
  constexpr bool STG = MAXNEW <= STAGE_NV;
  const int lane = threadIdx.x & 31;
  const bool seed = src == nullptr;
  const int w = a.w, wo = a.wo;
  const int wsv = join_row_stride(w);
  const WarpSmem W = warp_smem<BW_STAGE>(wbase, wsv);
  for (int q = lane; q < wo; q += 32) {  // where this step's columns go
    const int col = a.src_col[q];
    if (MODE == 1) {
      if (col < w) K.tq[col] = q + 1;
      else K.npos[col - w] = (int8_t)q;
    } else {
      K.code[q] = (int16_t)(col < w ? col : (0x100 | (col - w)));
    }
  }
  for (int c = w; c < wsv; c++) W.rows[lane * wsv + c] = -1;  // padding words of the 32 tile rows
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
__device__ __forceinline__ void walk_step_mode(const JoinArgs &a, unsigned char *wbase, const WalkSmem &K,
                                               const int32_t *src, int rs_in, int nr, int64_t m0, int32_t *out,
                                               int rs_out, int64_t cap, int64_t &n_out, unsigned long long *ovf,
                                               unsigned long long &ar, unsigned long long &as) {
  switch (a.n_new) {
    case 1: walk_tile<1, MODE>(a, wbase, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 2: walk_tile<2, MODE>(a, wbase, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 3: walk_tile<3, MODE>(a, wbase, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    case 4: walk_tile<4, MODE>(a, wbase, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as); break;
    default: walk_tile<MAXM, MODE>(a, wbase, K, src, rs_in, nr, m0, out, rs_out, cap, n_out, ovf, ar, as);
  }
}

// Row stride (words) of the level a step writes.
__host__ __device__ __forceinline__ int walk_level_stride(const JoinArgs &a) { return a.rs_out ? a.rs_out : a.wo; }

__global__ void __launch_bounds__(BW_BLK, 14) k_batchw(const __grid_constant__ BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *wbase = smem + (size_t)wid * walk_warp_bytes(P.ws_max, P.max_steps);
  const WalkSmem K = walk_smem(wbase, P.ws_max, P.max_steps);
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
          walk_step_mode<1>(a0, wbase, K, nullptr, 0, nr, lo, nullptr, 0, 0, n_out, P.ovf, ar, as);
        else
          walk_step_mode<0>(a0, wbase, K, nullptr, 0, nr, lo, out, a0.rs_out, P.lvl_cap[0], n_out, P.ovf, ar, as);
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
      const int nr = min(32, have - cur);
      const int rs_in = walk_level_stride(args[top]);
      const int32_t *src = (const int32_t *)(mine + P.lvl_off[top]) + (int64_t)cur * rs_in;
      const JoinArgs &a = args[j];
      int64_t n_out = 0;
      if (j == S - 1)
        walk_step_mode<1>(a, wbase, K, src, rs_in, nr, 0, nullptr, 0, 0, n_out, P.ovf, ar, as);
      else
        walk_step_mode<0>(a, wbase, K, src, rs_in, nr, 0, (int32_t *)(mine + P.lvl_off[j]), a.rs_out, P.lvl_cap[j],
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

size_t walk_smem_bytes(int ws_max, int max_steps) { return (size_t)BW_WARPS * walk_warp_bytes(ws_max, max_steps); }

int walk_grid(int ws_max, int max_steps, int num_sms, int max_per_sm) {
  const size_t smem = walk_smem_bytes(ws_max, max_steps);
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
  k_batchw<<<grid, BW_BLK, walk_smem_bytes(p.ws_max, p.max_steps), s>>>(p);
  return cudaGetLastError();
}

}  // namespace dmk
