// Launchers of the library's sm_103a kernels (kernels.cu). All take the stream to run on;
// none synchronises. Sizes are in elements unless the name says bytes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "dm_internal.h"

namespace dmk {

// Launch with programmatic dependent launch: the kernel may be scheduled while the previous
// kernel in the stream is finishing; it must execute griddep_wait() (join_device.cuh) before
// touching global memory that the previous kernel reads or writes. Used only where the
// previous stream operation is itself a kernel of the same chain.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Number of kernels this library has launched from the calling thread so far (a context's
// calls run on the calling thread, so per-call differences stay exact when several threads
// drive their own contexts at once).
int64_t launch_count();
extern thread_local int64_t g_launches;

// Fused join step of Alg. 1 (InnerJoin + FilterOverlappingNodes + back-edge filter + score
// + compaction, or count + checksum in the last step), warp-centric (join_warp.cu). The grid
// fills the GPU at the kernel's occupancy, or covers the rows of R when they are fewer.
// pdl: launched with programmatic dependent launch (the previous stream operation must be a
// kernel of the same chain).
cudaError_t launch_wjoin(const dmi::JoinArgs &a, int grid, cudaStream_t s, bool pdl = false);
// One full wave for a launch that reads its input row count on the device (n_dev), else the
// blocks its rows need, at most one wave.
int wjoin_grid(const dmi::JoinArgs &a, int num_sms);
// The last two steps of a counted plan in one kernel (join_warp.cu): a = the second-to-last
// step (writes, identity column order), b = the last (counted); b's rows are a's survivors,
// which never reach global memory (b.R is ignored). Counts go to a.ctr (a's survivors and
// candidates) and b.ctr (the count, checksum and b's candidates). fused_ok tells whether the
// pair qualifies (1 to 4 new vertices each, no scores, no shards, shared memory fits).
bool fused_ok(const dmi::JoinArgs &a, const dmi::JoinArgs &b);
cudaError_t launch_fused(const dmi::JoinArgs &a, const dmi::JoinArgs &b, int num_sms, cudaStream_t s, bool pdl);

// Data-graph preparation.
cudaError_t launch_csr_to_m2(const int32_t *row_ptr, const int32_t *col_idx, const float *eerr,
                             int32_t V, int64_t nnz, int32_t *rows, float *score, cudaStream_t s);
cudaError_t launch_vertex_table(int32_t V, int32_t *rows, float *score, cudaStream_t s);
cudaError_t launch_bitmap(const int32_t *row_ptr, const int32_t *col_idx, int32_t V, int64_t nnz,
                          int32_t words, unsigned long long *adj, cudaStream_t s);

// Exclusive scan of n values into out[0..n], out[n] = total. tmp must hold
// scan_tmp_elems(n) int64 values: per level of the scan over tile sums, the sums and their scan.
constexpr int SCAN_BLK = 256, SCAN_ITEMS = 8, SCAN_TILE = 2048;
constexpr int64_t scan_tmp_elems(int64_t n) {
  return (n + SCAN_TILE - 1) / SCAN_TILE <= 1
             ? 1
             : 2 * ((n + SCAN_TILE - 1) / SCAN_TILE) + 1 + scan_tmp_elems((n + SCAN_TILE - 1) / SCAN_TILE);
}
cudaError_t scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
cudaError_t scan_i32(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);

// One stable LSD pass: perm_out = perm_in stably sorted by the 8-bit digit
// (key >> shift) & 255 of key = keys[perm_in[i] * stride]. hist must hold
// radix_hist_elems(n) int64, tmp scan_tmp_elems(radix_hist_elems(n)).
constexpr int RS_BLK = 256, RS_ITEMS = 8, RS_TILE = 2048;
constexpr int64_t radix_hist_elems(int64_t n) { return 256 * ((n + RS_TILE - 1) / RS_TILE); }
cudaError_t radix_pass(const uint32_t *keys, int64_t stride, const int32_t *perm_in,
                       int32_t *perm_out, int64_t n, int shift, int64_t *hist, int64_t *hist_scan,
                       int64_t *tmp, cudaStream_t s);
cudaError_t launch_iota(int32_t *p, int64_t n, cudaStream_t s);
// In place: w[i] = -log(1 - w[i]) (error rate -> negative log fidelity).
cudaError_t launch_neg_log1m(float *w, int64_t n, cudaStream_t s);
// Packed join keys of a table's rows: (row[kp0] << 32) | row[kp1], or row[kp0] when kp1 < 0.
cudaError_t launch_join_keys(const int32_t *rows, int32_t w, int32_t kp0, int32_t kp1, int64_t n,
                             unsigned long long *keys, cudaStream_t s);
// Streaming chunk boundaries over a prefix array pre[0..n] (non-decreasing): bounds[t] is the
// largest i with pre[i] <= t * step for 0 < t < nch, bounds[0] = 0, bounds[nch] = n; bpre[t] =
// pre[bounds[t]]. Both outputs hold nch + 1 entries.
cudaError_t launch_chunk_bounds(const int64_t *pre, int64_t n, int64_t step, int64_t nch, int64_t *bounds,
                                int64_t *bpre, cudaStream_t s);
cudaError_t launch_gather_rows(const int32_t *in, const float *ins, const int32_t *perm, int64_t n,
                               int32_t w, int32_t *out, float *outs, cudaStream_t s);

// Motif-table indices.
cudaError_t launch_offsets_direct(const int32_t *rows, int32_t mw, int32_t kpos, int64_t n,
                                  int32_t V, int32_t *offsets, cudaStream_t s);
cudaError_t launch_hash_build(const int32_t *rows, int32_t mw, int32_t kp0, int32_t kp1, int64_t n,
                              dmi::HashSlot *slots, uint32_t log2cap, unsigned long long *ctr,
                              cudaStream_t s);

// Top-k support: histogram of the 8-bit digit at `shift` of the scores' order-preserving keys, over the
// scores whose keys agree with `prefix` on `pmask`; and compaction of indices with key <= T.
cudaError_t launch_score_hist(const float *sc, int64_t n, uint32_t prefix, uint32_t pmask, int shift,
                              unsigned long long *hist, cudaStream_t s);
cudaError_t launch_select_le(const float *sc, int64_t n, uint32_t T, int32_t *out_idx,
                             unsigned long long *ctr, cudaStream_t s);
// Direction-aware scores (Sec. 5.4 footnote): out[i] = sum_e sw[e] * edir[slot of
// rows[i][sp[e]] -> rows[i][sq[e]]] (+ sum_u qerr[rows[i][u]] when qerr is set), FP32.
cudaError_t launch_rescore_directed(const int32_t *rows, int64_t n, int32_t np, const int32_t *sp, const int32_t *sq,
                                    const float *sw, int32_t nslots, const int32_t *row_ptr, const int32_t *col_idx,
                                    const float *edir, const float *qerr, float *out, cudaStream_t s);
// keys[i] = order-preserving unsigned key of sc[i] (the bits of both functions above are
// these keys, not the raw FP32 bits).
cudaError_t launch_score_keys(const float *sc, int64_t n, uint32_t *keys, cudaStream_t s);

// Sum over rows of the checksum hash H(row) into ctr[CTR_SUM] (count = n).
cudaError_t launch_hash_rows(const int32_t *rows, int64_t n, int32_t w, unsigned long long *ctr, cudaStream_t s);

// Canonical row order by comparison sort (sort.cu): *perm_out (inside tmp) receives the
// row indices in ascending lexicographic order; ids are below 2^bits. tmp holds
// msort_tmp_bytes(n) bytes.
int64_t msort_tmp_bytes(int64_t n);
// Tables of at most msort_into_max_rows() rows: the canonical order written straight into
// out_rows / out_scores (nullable) in three launches (key packing with the optional checksum,
// tile sort, rank scatter, the last on at most max_blocks blocks); tmp as for msort_rows.
int64_t msort_into_max_rows();
cudaError_t msort_rows_into(const int32_t *rows, const float *scores, int64_t n, int32_t w, int bits, void *tmp,
                            int32_t *out_rows, float *out_scores, unsigned long long *sum, int max_blocks,
                            cudaStream_t s);
// When sum is set, the row checksums (sum of H(row), as the count-mode join) are added to it.
cudaError_t msort_rows(const int32_t *rows, int64_t n, int32_t w, int bits, void *tmp, int32_t **perm_out,
                       unsigned long long *sum, cudaStream_t s);

// The min(k, n) smallest (score key, row index) of a canonically sorted table, k <= 1024,
// gathered into orows / osc in that order. tmp holds topk_tmp_bytes(n) bytes.
int64_t topk_tmp_bytes(int64_t n);
cudaError_t topk_sorted(const int32_t *rows, const float *sc, int64_t n, int32_t w, int32_t k, void *tmp,
                        int32_t *orows, float *osc, cudaStream_t s);

// Images (sort.cu): sort the ids inside each row in place; then, on canonically sorted rows,
// keep the first row of every run of equal rows (pos[n] receives the number kept; flag holds n
// ints, pos n + 1, tmp scan_tmp_elems(n)).
cudaError_t images_prepare(int32_t *rows, int64_t n, int32_t w, cudaStream_t s);
cudaError_t unique_rows(const int32_t *rows, int64_t n, int32_t w, int32_t *flag, int64_t *pos, int64_t *tmp,
                        int32_t *out, cudaStream_t s);

// Persistent batch kernel (batch.cu).
struct BatchPlan {
  int32_t n_steps;
  int32_t args_off;  // index of the plan's first step in BatchParams::args
};
struct BatchItem {
  int32_t plan;
  int32_t pad;
  int64_t lo, hi;    // rows of the first slice's motif table
};
struct BatchParams {
  const dmi::JoinArgs *args;
  const BatchPlan *plans;
  const BatchItem *items;
  int64_t n_items;
  unsigned long long *next_item;  // work counter (zeroed before the launch)
  unsigned long long *out;        // count, checksum per plan (zeroed before the launch)
  unsigned long long *ovf;
  unsigned char *scratch;         // grid * cta_bytes (warp walks: one cta_bytes slice per warp)
  int64_t cta_bytes;
  int64_t lvl_off[dmi::MAXSTEPS]; // byte offset of level j inside a CTA's scratch
  int64_t lvl_cap[dmi::MAXSTEPS]; // rows level j can hold
  int TR;                         // rows per tile
  int ws_max;                     // shared-memory row stride covering every step
  int bm_words;                   // > 0: per tile row, a bitmap of its ids (ids < 64 * bm_words) for
                                  // the injectivity test of steps with many new vertices
  unsigned long long *plan_left;  // work items still open per plan (set before the launch)
  unsigned long long *plan_done;  // GPU global-timer time at which each plan's last item ended
  unsigned long long *start_ns;   // GPU global-timer time at the start of the launch
  int max_steps;                  // warp walks: the most steps of a plan (per-warp level state)
  int tile_words;                 // warp walks: words of each walk's shared tile (a multiple of 4)
};
// threads: 128 or 256 per CTA. batch_grid: SMs x resident CTAs per SM (at most max_per_sm when
// it is > 0).
size_t batch_smem_bytes(int tile_rows, int ws_max, int bm_words, int threads);
int batch_grid(int tile_rows, int ws_max, int bm_words, int num_sms, int threads, int max_per_sm);
cudaError_t launch_batch(const BatchParams &p, int grid, int threads, cudaStream_t s);
// The same batch with one depth-first walk per warp (k_batchw, 64-thread CTAs): tiles of up to
// 32 rows (TR = 32; a step of row stride s takes min(32, tile_words / s)), the levels of each warp
// in its own cta_bytes slice of scratch, rows of level j of stride args[j].rs_out (padded,
// working-column order) or args[j].wo. walk_grid: SMs x resident CTAs per SM (at most max_per_sm
// when it is > 0); BW_WALK_WARPS warps a CTA. BW_WALK_TILE_STRIDE: the row stride (words) that a
// walk's tile holds 32 rows of.
constexpr int BW_WALK_WARPS = 2, BW_WALK_TILE_STRIDE = 28;
size_t walk_smem_bytes(int tile_words, int max_steps);
int walk_grid(int tile_words, int max_steps, int num_sms, int max_per_sm);
cudaError_t launch_batch_walk(const BatchParams &p, int grid, cudaStream_t s);

// Cardinality model (mlp.cu): flat FP32 parameters, BF16 tensor-core forward / backward.
int64_t mlp_param_count();
int64_t mlp_work_bytes(int rows);
// Word of the work buffer that the forward/backward pass sets when a tensor-core wait ran out
// (the pass's outputs are then invalid); zeroed at the start of every pass.
unsigned *mlp_error_flag(void *work, int rows);
cudaError_t mlp_forward_backward(const float *params, const float *X, const float *target, int rows, int n_valid,
                                 float *y, float *grads, float *loss, void *work, cudaStream_t s);
cudaError_t mlp_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr, int step,
                     cudaStream_t s);

}  // namespace dmk
