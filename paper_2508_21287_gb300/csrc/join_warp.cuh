// Warp-tile join machinery shared by the per-step join kernel (k_joinw, join_warp.cu) and the
// warp form of the persistent batch kernel (k_batchw, batch.cu): one warp joins a 32-row tile of
// R held in its own slice of shared memory, one row per lane for the key lookup and one
// candidate per lane for the checks, and stages its survivors for coalesced 16-byte writes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "join_device.cuh"

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

}  // namespace dmk
