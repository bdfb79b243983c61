/*
 * dm.h - C ABI of the GB300 (sm_103a) Delta-Motif embedding-enumeration library.
 *
 * Problem (Sec. 3.1 of "Delta-Motif: Parallel Subgraph Isomorphism via Tabular Operations
 * for Scalable Layout Selection", arXiv 2508.21287): given an undirected, simple, connected
 * data graph G_d and pattern graph G_p, enumerate every injective map f : V_p -> V_d such
 * that each pattern edge {u, v} maps onto a data edge {f(u), f(v)}. The library follows the
 * method's reading of that statement (Alg. 1 with the overlap filter of Sec. 3.2): edges
 * must be preserved, non-edges need not be (monomorphisms); dm_plan_opts.induced = 1 adds the
 * non-edge condition of the literal statement.
 *
 * Method (Sec. 3.2-3.3, Alg. 1, Alg. 2): the pattern is decomposed into motif slices (paths,
 * cycles, stars, ...); the embeddings Res(M) of each motif in G_d are tables of vertex-id
 * tuples, built once per data graph; the result is assembled by joining the tables on the
 * pattern vertices that slices share and filtering rows whose mapped vertices repeat.
 * All of it runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions for every call:
 *   - Return value: DM_OK (0) or a negative DM_E_* code; dm_strerror() names it. On error
 *     no output argument is written unless stated.
 *   - Vertex ids are int32, 0-based. CSR: row_ptr has n+1 entries, row_ptr[0] = 0,
 *     col_idx[row_ptr[u] .. row_ptr[u+1]) lists the neighbours of u, sorted ascending,
 *     no duplicates; every edge appears in both directions. Self-loops are dropped on load
 *     (Res(M2) excludes them, Sec. 3.3).
 *   - Input arrays are host memory owned by the caller; the library copies what it keeps.
 *   - Calls on one dm_ctx must not run concurrently from several host threads.
 *   - All device work of a context runs on its stream (dm_set_stream), in order.
 */
#ifndef DM_H
#define DM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes ---- */
#define DM_OK 0
#define DM_E_INVAL (-1)        /* bad argument or malformed CSR (asymmetric, unsorted, duplicate, out of range) */
#define DM_E_DISCONNECTED (-2) /* pattern or data graph not connected (Sec. 3.1 assumes connected graphs) */
#define DM_E_NOMEM (-3)        /* device or host allocation failed, or the memory budget is too small */
#define DM_E_CAPACITY (-4)     /* projected work or rows exceed the plan's cap (dm_plan_opts.max_rows) */
#define DM_E_TIMEOUT (-5)      /* a bounded wait (about a second) of the model's tensor-core matmul ran out */
#define DM_E_CUDA (-6)         /* a CUDA runtime call failed */
#define DM_E_CANCELLED (-7)    /* the chunk callback returned non-zero */
#define DM_E_NOTFOUND (-8)     /* unknown graph handle or motif id */

/* ------------------------------------------------------------------ handles --------- */
typedef struct dm_ctx dm_ctx;
typedef struct dm_plan_s dm_plan_t; /* plan handle (the call that makes one is dm_plan) */
typedef int32_t dm_graph;

/* ------------------------------------------------------------------ motifs ---------- */
/* Motif ids (naming of Sec. 3.1: M_k is a path on k vertices, "-O" a cycle, "-1" one
 * branch). Vertex order of each motif is fixed: paths 0-1-...-(k-1); cycles 0-1-...-(k-1)-0;
 * M4-1 has centre 0 and leaves 1, 2, 3; M6-2O is the 2 x 3 grid 0-1-2 / 3-4-5 with rungs
 * 0-3, 1-4, 2-5; M18-O-6 is the 12-cycle 0..11 plus pendant vertex 12 + i/2 on each even
 * cycle vertex i. */
#define DM_MOTIF_PATH(k) (k)           /* k = 2..24: M_k, M2 is a single edge */
#define DM_MOTIF_CYCLE(k) (100 + (k))  /* k = 3..24: M_{k-O} */
#define DM_MOTIF_M4_1 201              /* claw K_{1,3} */
#define DM_MOTIF_M6_2O 202             /* two 4-cycles sharing an edge (2 x 3 grid) */
#define DM_MOTIF_M18_O_6 203           /* 12-cycle with a pendant on every other vertex */

/* ------------------------------------------------------------------ plan options ---- */
#define DM_ORDER_PAPER 0      /* Sec. 3.2: largest motif first, first match found */
#define DM_ORDER_HEURISTIC 1  /* greedy: smallest estimated intermediate table next */
#define DM_ORDER_LEARNED 2    /* cheapest of several candidate plans under the trained cardinality model (heuristic order if none) */

#define DM_JOIN_AUTO 0
#define DM_JOIN_HASH 1        /* probe a per-key index of the motif table (direct offsets for one key,
                                 open-addressing hash of the packed 64-bit key for two) */
#define DM_JOIN_SORTMERGE 2   /* sort the intermediate table by its key columns each step and find each
                                 row's group by binary search in the motif table's sorted packed keys
                                 (no offsets or hash table; plans with it always stream step by step) */

typedef struct dm_plan_opts {
    const int32_t *motifs; /* motif ids to decompose with (M2 is always added); NULL = preset by data-graph degree */
    int32_t n_motifs;
    int32_t order;          /* DM_ORDER_* */
    int32_t join_algo;      /* DM_JOIN_* */
    int32_t induced;        /* 0 = embeddings preserve pattern edges (monomorphisms, Alg. 1 as given);
                               1 = also non-edges: pattern vertices that are not adjacent map to
                               data vertices that are not adjacent (the literal "iff" of Sec. 3.1) */
    int64_t chunk_rows;     /* 0 = from the memory budget; else the row cap of one intermediate chunk */
    int64_t max_rows;       /* 0 = unlimited; else DM_E_CAPACITY once a step's candidate rows exceed it */
} dm_plan_opts;

/* ------------------------------------------------------------------ context --------- */

/* Create a context on CUDA device `device`. No counterpart in the paper (its tables live in a
 * dataframe library's memory pool): a context owns a stream, counters and the device memory
 * of its graphs and tables. mem_budget_bytes bounds the device memory the intermediate tables
 * of one dm_match may hold (0 = half of the free memory at creation); larger results are
 * streamed in chunks (depth-first over the join steps). Errors: DM_E_INVAL (out NULL),
 * DM_E_CUDA (no such device, or stream/event creation failed), DM_E_NOMEM. */
int dm_create(dm_ctx **out, int device, uint64_t mem_budget_bytes);

/* Release every graph, motif table and buffer of the context (no counterpart in the paper).
 * Waits for the context's stream first. The handle is invalid afterwards. DM_E_INVAL for
 * NULL. */
int dm_destroy(dm_ctx *ctx);

/* Run subsequent device work on `stream` (a cudaStream_t; NULL = the context's own stream). */
int dm_set_stream(dm_ctx *ctx, void *stream);

/* Change the memory budget of later calls (bytes; 0 = half of the free memory now). */
int dm_set_budget(dm_ctx *ctx, uint64_t mem_budget_bytes);

/* ------------------------------------------------------------------ data graph ------ */

/* Load a data graph (Sec. 3.1). edge_err (nullable) is aligned with col_idx: the error of
 * the directed slot, equal on both directions of an edge. qubit_err (nullable) has n
 * entries. Weights must be finite (NaN or infinity: DM_E_INVAL). Error rates are >= 0 in the
 * paper's use (Sec. 5.4); negative weights are accepted, but then dm_score_topk cannot prune
 * rows by their partial score and keeps every row until the end (slower, same answer).
 * The graph, its adjacency bitmap and its Res(M2) table (Sec. 3.3) stay resident
 * on the device until dm_destroy. Errors: DM_E_INVAL for malformed CSR or weights,
 * DM_E_DISCONNECTED if G_d is not connected; on any error no graph is registered and nothing
 * stays allocated. */
int dm_load_data_graph(dm_ctx *ctx, int32_t n_vertices, const int32_t *row_ptr,
                       const int32_t *col_idx, const float *edge_err, const float *qubit_err,
                       dm_graph *out);

/* Score forms of a loaded graph (Sec. 5.4 ranks layouts by the product of the fidelities
 * 1 - e of the mapped edges and qubits):
 *   DM_SCORE_ERROR_SUM    the score of a row is the sum of its error rates e (the first-order,
 *                         log-domain form of the product; dm_load_data_graph uses it);
 *   DM_SCORE_LOG_FIDELITY the score is the sum of -log(1 - e) = -log(product of fidelities):
 *                         exactly the product's order, and exp(-score) is the layout fidelity.
 * Lower is better in both. */
#define DM_SCORE_ERROR_SUM 0
#define DM_SCORE_LOG_FIDELITY 1

/* dm_load_data_graph with a score form. With DM_SCORE_LOG_FIDELITY every error rate must lie
 * in [0, 1) (else DM_E_INVAL); the device keeps -log(1 - e) per edge slot and qubit. */
int dm_load_data_graph_ex(dm_ctx *ctx, int32_t n_vertices, const int32_t *row_ptr,
                          const int32_t *col_idx, const float *edge_err, const float *qubit_err,
                          int32_t score_form, dm_graph *out);

/* Res(M) of one motif on a loaded graph (Alg. 2 builds it by the same join-and-filter
 * loop). Writes min(cap, count) rows of k = motif size ints (row-major, host memory, in
 * canonical ascending order) to out_rows (nullable) and the count and k to out_n / out_k. */
int dm_motif_table(dm_ctx *ctx, dm_graph g, int32_t motif_id, int32_t *out_rows, int64_t cap,
                   int64_t *out_n, int32_t *out_k);

/* ------------------------------------------------------------------ plans ----------- */

/* Decompose a pattern into motif slices (Sec. 3.2) against a loaded data graph and fix the
 * join order. opts may be NULL. Errors: DM_E_INVAL (malformed CSR, n_p outside 1..128),
 * DM_E_DISCONNECTED (pattern not connected). The plan owns copies of the pattern. */
int dm_plan(dm_ctx *ctx, dm_graph g, int32_t n_p, const int32_t *p_row_ptr,
            const int32_t *p_col_idx, const dm_plan_opts *opts, dm_plan_t **out);

/* Release a plan made by dm_plan, dm_plan_batch or dm_plan_candidates (no counterpart in
 * the paper; host memory only, no device work). NULL is accepted. */
void dm_plan_free(dm_plan_t *plan);

/* dm_plan (the decomposition and join order of Sec. 3.2) for n_patterns patterns at once,
 * no counterpart in the paper as a batch (pattern i: n_p[i] vertices, CSR p_row_ptr[i] /
 * p_col_idx[i]), the same options for all: motif tables are prepared on the calling thread,
 * the decompositions run on host threads, and with DM_ORDER_LEARNED every candidate of every
 * pattern is costed in one model evaluation. Plans equal those of dm_plan pattern by pattern;
 * out (n_patterns entries, caller-owned array) receives them, each to be released with
 * dm_plan_free. On error nothing is returned (out[i] = NULL for all i) and the status is that
 * of the first failing pattern. */
int dm_plan_batch(dm_ctx *ctx, dm_graph g, int32_t n_patterns, const int32_t *n_p,
                  const int32_t *const *p_row_ptr, const int32_t *const *p_col_idx,
                  const dm_plan_opts *opts, dm_plan_t **out);

/* The candidate decompositions that DM_ORDER_LEARNED chooses from (Sec. 3.2 decomposition
 * with the paper's order and with the greedy heuristic order, over the motif set and, unless
 * opts->motifs is given, over sets adding a larger motif typical of the topology or two
 * paths of about half the pattern). Each is a runnable plan with that order fixed; running
 * them is how a caller logs training steps for every shape the learned planner may pick.
 * Writes up to max_out handles to out (the caller frees each with dm_plan_free) and returns
 * the number of candidates, or a negative error (as dm_plan). out may be NULL when
 * max_out is 0. The paper has no counterpart (its order is fixed by hand). */
int32_t dm_plan_candidates(dm_ctx *ctx, dm_graph g, int32_t n_p, const int32_t *p_row_ptr,
                           const int32_t *p_col_idx, const dm_plan_opts *opts, dm_plan_t **out,
                           int32_t max_out);

/* Flat description of a plan, for inspection and tests. Writes up to buf_len int32 words:
 *   [n_steps, then per step: motif_id, k, slice[0..k-1] (pattern vertex of each motif
 *    position), n_keys, n_backedges, backedge pairs (2 words each, pattern vertex ids)]
 * and returns the number of words needed (or a negative error). */
int32_t dm_plan_describe(const dm_plan_t *plan, int32_t *buf, int32_t buf_len);

/* Host-only decomposition (Sec. 3.2) of a pattern with a motif set, without a data graph
 * or a GPU: same output format as dm_plan_describe. order DM_ORDER_PAPER is the paper's
 * rule; the estimate-driven orders see unit table sizes here. Returns the words needed, or
 * DM_E_INVAL / DM_E_DISCONNECTED / DM_E_NOTFOUND (unknown motif id). */
int32_t dm_decompose(int32_t n_p, const int32_t *p_row_ptr, const int32_t *p_col_idx,
                     const int32_t *motifs, int32_t n_motifs, int32_t order, int32_t *buf,
                     int32_t buf_len);

/* ------------------------------------------------------------------ matching -------- */
#define DM_ALL 0            /* materialise every embedding */
#define DM_COUNT 1          /* count + checksum only */
#define DM_DEVICE_ROWS 0x10 /* flag: the callback gets device pointers instead of host copies */

/* Chunk callback of DM_ALL. rows: nrows x n_cols int32, row-major, row r = (f(0), ...,
 * f(n_p - 1)) indexed by pattern vertex; scores: nrows FP32 layout scores, or NULL when the
 * graph has no error weights. Buffers belong to the library and are valid only during the
 * call. Returning non-zero stops the match with DM_E_CANCELLED. */
typedef int (*dm_chunk_cb)(void *user, const int32_t *rows, const float *scores, int64_t nrows,
                           int32_t n_cols);

/* Enumerate Emb(G_p, G_d) with the plan (Alg. 1).
 *   DM_ALL: rows are delivered through cb in ascending canonical (lexicographic) order when
 *     the whole result fits the memory budget; otherwise each delivered chunk is sorted and
 *     chunks follow the depth-first order of the streamed join.
 *   DM_COUNT: nothing is delivered; cb may be NULL.
 * out_count / out_checksum (nullable) receive |Emb| and the checksum: the sum mod 2^64 over
 * rows of H(row) = mix64(n_p + sum_j mix64(((j + 1) << 32) | f(j))), sums mod 2^64, mix64 the
 * SplitMix64 finaliser. The library's own digest (the paper has none); it binds each vertex
 * id to its pattern position and does not depend on row order.
 * Scores (when the graph has error weights) are the sum of edge errors over pattern edges
 * plus vertex errors, FP32 (Sec. 5.4, log-domain form of the fidelity product). */
int dm_match(dm_ctx *ctx, const dm_plan_t *plan, int mode, dm_chunk_cb cb, void *user,
             uint64_t *out_count, uint64_t *out_checksum);

/* One shard of dm_match(DM_COUNT) (Alg. 1 over a slice of its first table R_0; the paper
 * runs one GPU): the count and checksum of the embeddings whose image of the plan's first
 * slice vertex (dm_plan_describe: step 0, slice[0]) is congruent to shard modulo n_shards.
 * The shards 0 .. n_shards - 1 partition Emb: their counts and checksums sum (mod 2^64) to
 * dm_match's, so GPUs that each run one shard combine their results with one 2 x u64 sum.
 * Each shard reads the whole motif table of the first step and keeps its rows; the later
 * steps see only the shard's rows. DM_E_INVAL unless 0 <= shard < n_shards. */
int dm_match_shard(dm_ctx *ctx, const dm_plan_t *plan, int32_t shard, int32_t n_shards,
                   uint64_t *out_count, uint64_t *out_checksum);

/* Count + checksum for n_plans plans on the same data graph in one persistent launch
 * (captured in a CUDA graph). Each plan is Alg. 1 (Sec. 3.2) as in dm_match; running many
 * plans in one launch has no counterpart in the paper (it answers one pattern at a time).
 * mode must be DM_COUNT (else DM_E_INVAL). out_counts / out_checksums have n_plans entries
 * (caller-owned host arrays). Results are identical to dm_match(DM_COUNT) on each plan alone.
 * Errors: DM_E_INVAL (plans on different graphs, NULL arguments), DM_E_NOMEM, DM_E_CUDA. */
int dm_match_batch(dm_ctx *ctx, const dm_plan_t *const *plans, int32_t n_plans, int mode,
                   uint64_t *out_counts, uint64_t *out_checksums);

/* Configuration of the last dm_match_batch, as picked by the autotuner (no counterpart in
 * the paper): tile rows per CTA step, root rows per work item, CTAs of the persistent launch,
 * how many plans (those whose predicted largest table exceeds heavy_rows) ran step by step
 * over the whole GPU after the persistent launch instead of inside it, the block shape
 * (threads per CTA, 128 or 256, and resident CTAs per SM; 32 = one depth-first walk per warp,
 * two warps a CTA, 32-row tiles) and the load factor of the two-key hash indices the joins
 * probed. Every output pointer may be NULL. DM_E_INVAL if the context
 * has run no batch. */
int dm_batch_config(dm_ctx *ctx, int32_t *tile_rows, int64_t *root_chunk, int32_t *grid,
                    int32_t *n_stepwise, double *heavy_rows, int32_t *threads_per_cta,
                    int32_t *ctas_per_sm, double *hash_load_factor);

/* Completion time of each plan of the last dm_match_batch (all plans taken to arrive
 * together), in ms: for plans in the persistent launch, from the launch's start to the end
 * of the plan's last work item (GPU global timer); for plans run step by step, from the
 * start of the call to their end (host clock). n must equal that call's n_plans. */
int dm_batch_latency(dm_ctx *ctx, double *out_ms, int32_t n);

/* Tuning knobs: autotune (1 = on the first dm_match_batch of a new set of plans, time the
 * candidate configurations and keep the fastest: tile rows x root chunk, the split between
 * the persistent launch and step-by-step execution, the block shape (and the root chunk again
 * for a changed shape), then the two-key hash
 * load factor among 0.25, 0.5 and 0.75, a coordinate search; the chosen load factor stays
 * the context's for later calls), hash_load_factor (fill of two-key hash indices,
 * 0 < f <= 0.95; changing it drops those indices, which are rebuilt when a plan next runs),
 * heavy_rows (without autotuning: plans whose predicted largest table exceeds it run step by
 * step; <= 0 = none). */
int dm_set_tuning(dm_ctx *ctx, int autotune, double hash_load_factor, double heavy_rows);

/* on = 1: counted matches (DM_COUNT, dm_match_shard) on the device-driven path run their
 * plan's last two joins as one kernel when both map 1 to 4 new vertices: the survivors of the
 * second-to-last join are joined and counted in shared memory, so the table between the two
 * joins (the largest of a path-like plan) is never written to or read from device memory.
 * on = 0 (the default) runs every join as its own launch (Alg. 1 step by step). Results are
 * identical either way. No counterpart in the paper (its joins are library calls). */
int dm_set_fusion(dm_ctx *ctx, int on);

/* Block shape of dm_match_batch when autotuning is off (no counterpart in the paper):
 * threads_per_cta 128 or 256 (every CTA walks its work items through the plan's steps in
 * tiles of the tuned row count), or 32 (every warp walks its own work items in 32-row tiles,
 * with no block barrier; two warps a CTA), and ctas_per_sm resident CTAs per SM (0 = as many
 * as fit). DM_E_INVAL otherwise. Takes effect at the next dm_match_batch. */
int dm_set_batch_shape(dm_ctx *ctx, int32_t threads_per_cta, int32_t ctas_per_sm);

/* The k best layouts (Sec. 5.4): the min(k, |Emb|) embeddings with the smallest (score,
 * row) key, in that order. out_rows: k x n_p int32 host buffer; out_scores: k floats
 * (nullable); out_n receives the number written. Needs edge weights (DM_E_INVAL if none).
 * When every weight of the graph is >= 0, rows whose partial score already exceeds the
 * current k-th best are dropped inside the joins (a partial score is then a lower bound of
 * the full one); with a negative weight nothing is pruned. The answer is the same either way. */
int dm_score_topk(dm_ctx *ctx, const dm_plan_t *plan, int32_t k, int32_t *out_rows,
                  float *out_scores, int32_t *out_n);

/* Direction-aware layout scores (Sec. 5.4, its footnote on directed two-qubit gates: layouts
 * are enumerated on the undirected coupling graph and the direction of each gate is handled
 * afterwards). e_dir has row_ptr[n] floats aligned with the graph's col_idx: e_dir[slot of
 * u -> v] is the cost of a two-qubit gate run from u to v (the native direction's error, or
 * that error plus the cost of turning the gate around); it need not be symmetric and must be
 * finite (else DM_E_INVAL). The library keeps a device copy with the graph, replacing any
 * earlier one, until dm_destroy. DM_E_NOTFOUND for an unknown graph. */
int dm_load_directed_errors(dm_ctx *ctx, dm_graph g, const float *e_dir);

/* The k best layouts by their direction-aware score: score(f) = sum over the pattern's slots
 * p -> q of w_dir[slot] * e_dir(f(p) -> f(q)), plus the graph's vertex errors of the images
 * when it has them; FP32. w_dir (host, finite, aligned with the plan's pattern col_idx) is the
 * circuit's number of gates run from p to q (0 for none; any weight works). The embeddings
 * are those of dm_match (every one is scored after the joins; nothing is pruned by a partial
 * score), then ranked as in dm_score_topk by (score, row). Needs dm_load_directed_errors on
 * the plan's graph first (else DM_E_INVAL). out_rows: k x n_p int32 host buffer; out_scores:
 * k floats (nullable); out_n receives the number written. */
int dm_score_topk_directed(dm_ctx *ctx, const dm_plan_t *plan, const float *w_dir, int32_t k,
                           int32_t *out_rows, float *out_scores, int32_t *out_n);

/* DM_ALL and top-k from one pass of the joins: every embedding goes through cb exactly as
 * in dm_match, and the k best (score, row) rows are written to out_rows / out_scores as in
 * dm_score_topk. Needs edge weights. */
int dm_match_topk(dm_ctx *ctx, const dm_plan_t *plan, int mode, dm_chunk_cb cb, void *user,
                  int32_t k, int32_t *out_rows, float *out_scores, int32_t *out_n,
                  uint64_t *out_count, uint64_t *out_checksum);

/* ------------------------------------------------------------------ learned planner --- */
/* No counterpart in the paper (which notes that motif choice and ordering matter, Sec. 5.2):
 * a 3-layer MLP (32 -> 128 -> 128 -> 1, ReLU; BF16 matmuls on the fifth-generation tensor
 * cores, tcgen05, with FP32 accumulation in tensor memory) predicts, for a candidate join
 * step, the log growth of the intermediate
 * table, log(1 + rows after) - log(1 + rows before). DM_ORDER_LEARNED plans are the cheapest,
 * under the model's predicted cardinalities, of several candidate decompositions (the
 * paper's rule and the greedy heuristic order, with the given motif set, with motifs
 * typical of the topology, and with two half-length paths for patterns of 16+ vertices; see
 * dm_plan_candidates); without a trained model they use the heuristic order.
 * The output set never depends on the order. Feature vectors are DM_MODEL_FEATURES floats
 * (dm_plan_estimates / dm_step_log give them); parameters are FP32, flat, in the order
 * W1[128][32] b1[128] W2[128][128] b2[128] w3[128] b3, followed by the 32 input means and
 * 32 input standard deviations used to standardise the features. The calls that run the
 * model (dm_model_train, dm_model_predict, dm_model_grad, and planning in the learned order)
 * return DM_E_TIMEOUT if a matmul's bounded wait for its tensor-core work ran out (the results
 * of that call are then discarded). */
#define DM_MODEL_FEATURES 32

/* Fresh He-uniform weights from a SplitMix64 stream seeded by `seed`; forgets training. */
int dm_model_init(dm_ctx *ctx, uint64_t seed);

/* Train on n (features, log growth) samples with Adam (mini-batches of `batch` >= 16,
 * `epochs` passes, learning rate lr, shuffling seeded by `seed`), all on the GPU.
 * out_loss (nullable) receives the mean squared error of each epoch. */
int dm_model_train(dm_ctx *ctx, const float *feats, const float *targets, int32_t n, int32_t epochs,
                   int32_t batch, float lr, uint64_t seed, float *out_loss);

/* Predicted log growth of n feature vectors (host in, host out). */
int dm_model_predict(dm_ctx *ctx, const float *feats, int32_t n, float *out);

/* One forward + backward pass on raw (already standardised) inputs, for checking the
 * kernels: predictions, the gradient of the mean squared error (flat, parameter order) and
 * the loss. targets may be NULL (forward only). */
int dm_model_grad(dm_ctx *ctx, const float *feats, const float *targets, int32_t n, float *out_pred,
                  float *out_grads, float *out_loss);

/* Parameters + standardisation (n_floats receives the count); set them back (checkpoint). */
int dm_model_weights(dm_ctx *ctx, float *out, int64_t *n_floats);
int dm_model_set_weights(dm_ctx *ctx, const float *w, int64_t n_floats);

/* The (features, observed log growth) samples logged by every dm_match so far: up to cap of
 * them are copied out, out_n receives how many exist, clear != 0 empties the log. */
int dm_step_log(dm_ctx *ctx, float *feats, float *targets, int64_t cap, int64_t *out_n, int clear);

/* Predicted cost of a plan (bytes its joins write, plus a fixed per-step overhead) and its
 * largest predicted intermediate table, from the trained model for DM_ORDER_LEARNED plans
 * and from the independence heuristic otherwise. */
int dm_plan_cost(const dm_plan_t *plan, double *cost, double *max_rows);

/* Predicted rows after each step of a plan (the chain of predicted log growths it was costed
 * with: the trained model's for DM_ORDER_LEARNED plans, the independence heuristic's
 * otherwise). Writes up to cap values and returns the number of steps (or DM_E_INVAL). */
int32_t dm_plan_predicted_rows(const dm_plan_t *plan, double *rows, int32_t cap);

/* The model inputs of a plan's steps (cap rows of DM_MODEL_FEATURES) and the independence
 * heuristic's log growth of each; returns the number of steps. */
int dm_plan_estimates(const dm_plan_t *plan, float *feats, float *heur_growth, int32_t cap);

/* ------------------------------------------------------------------ serving ---------- */
/* Layout-query server (Sec. 5.4's layout selection as a service; the paper has no serving
 * loop): top-k requests are taken in arrival order by n_slots worker slots, each with its own
 * context and CUDA stream, so requests admitted while others run overlap on the GPU. A
 * request is admitted when a slot is free and its projected join memory (planner estimates of
 * the two largest consecutive tables) fits the pool shared by all in-flight requests; it is
 * answered with DM_E_CAPACITY when the projection exceeds the pool or max_rows, or when a
 * step's candidate rows exceed max_rows while it runs. Results equal dm_score_topk on the
 * same plan alone. Every graph is loaded into every slot. */
typedef struct dm_server dm_server;
typedef struct dm_server_opts {
    int32_t n_slots;            /* concurrent requests (default 4, at most 64) */
    uint64_t mem_budget_bytes;  /* pool for projected join memory (0 = 16 GiB) */
    int64_t max_rows;           /* work cap per request step (0 = none) */
    int32_t order;              /* DM_ORDER_* of request plans */
    const int32_t *motifs;      /* motif set of request plans (NULL = presets) */
    int32_t n_motifs;
} dm_server_opts;
typedef struct dm_server_stats {
    int64_t submitted, completed, rejected, failed, queued, in_flight;
    uint64_t pool_used, pool_total;
    int64_t max_running;  /* most requests inside their device work at one time (host view) */
    int64_t overlapped;   /* requests whose device interval (CUDA events on the slot's stream,
                             timed against one reference event) intersected another request's */
} dm_server_stats;

int dm_server_create(dm_server **out, int device, const dm_server_opts *opts);
/* Load a data graph into every slot (no request may be queued or running); same arguments
 * and errors as dm_load_data_graph. */
int dm_server_load_graph(dm_server *s, int32_t n_vertices, const int32_t *row_ptr,
                         const int32_t *col_idx, const float *edge_err, const float *qubit_err,
                         dm_graph *out);
/* Install trained model parameters (dm_model_weights layout) in every slot. */
int dm_server_set_model(dm_server *s, const float *w, int64_t n_floats);
/* Enqueue a top-k request (pattern CSR copied; the arrival time is now); out_id identifies it. */
int dm_server_submit(dm_server *s, dm_graph g, int32_t n_p, const int32_t *p_row_ptr,
                     const int32_t *p_col_idx, int32_t k, uint64_t *out_id);
/* Block until request `id` is answered: rows (k x n_p) and scores (k) as dm_score_topk,
 * n_out rows written, status (DM_OK or a DM_E_* code), latency = answer time - arrival,
 * queue = start of its device work - arrival (ms). Each id can be waited for once. */
int dm_server_wait(dm_server *s, uint64_t id, int32_t *rows, float *scores, int32_t *n_out,
                   int32_t *status, double *latency_ms, double *queue_ms);
int dm_server_stats_get(dm_server *s, dm_server_stats *out);
/* Finish the queued requests, stop the workers, release every slot. */
int dm_server_destroy(dm_server *s);

/* ------------------------------------------------------------------ no-allocation sort */
/* No counterpart in the paper: a library service for callers that cannot allocate device
 * memory when they need it (cudaMalloc/cudaFree synchronise the device, which a latency-bound
 * serving thread cannot afford; a framework's caching allocator may hold nearly all device
 * memory; some callers are only handed pre-reserved buffers).
 *
 * Sorts n rows of w int32 ids (row-major, device memory) into ascending lexicographic order
 * (column 0 most significant), writing rows_out (n x w, device) and, when scores_in is not
 * NULL, the scores carried along to scores_out (n floats, device). Every id must be below
 * 2^bits (1 <= bits <= 31). Inputs and outputs are caller-owned and must not overlap.
 * The temporaries live in one fixed device array of the library (about 10.5 MB, held by
 * every GPU that loads the library until exit); nothing is allocated or freed.
 * Limits: n <= DM_SORT_STATIC_MAX_ROWS (else DM_E_CAPACITY), 1 <= w <= 64 (else DM_E_INVAL).
 * Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream) and the call
 * returns without waiting. Every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, host-side); the first lookup on a device may load the
 * library's device code there, so make the first call on each device before any stream
 * capture. All calls share the one array: calls whose work overlaps on the GPU (other streams,
 * other host threads) race and corrupt each other's results; serialise them. */
#define DM_SORT_STATIC_MAX_ROWS (1 << 20)
int dm_sort_rows_static(const int32_t *rows_in, const float *scores_in, int64_t n, int32_t w,
                        int32_t bits, int32_t *rows_out, float *scores_out, void *stream);

/* The distinct vertex sets covered by the embeddings (the image of each map, ids ascending),
 * in ascending lexicographic order: automorphic copies of a layout collapse into one
 * (|images| x |Aut(G_p)| = |Emb|). Writes min(cap, count) sets of n_p ints to out_sets
 * (host, nullable) and the count to out_n. */
int dm_images(dm_ctx *ctx, const dm_plan_t *plan, int32_t *out_sets, int64_t cap, int64_t *out_n);

/* ------------------------------------------------------------------ statistics ------ */
#define DM_MAX_STEPS 128
typedef struct dm_stats {
    int32_t n_steps;                  /* join steps of the last dm_match / dm_score_topk */
    int64_t rows[DM_MAX_STEPS];       /* rows of the intermediate table after each step */
    int64_t candidates[DM_MAX_STEPS]; /* joined rows before filtering, per step */
    int64_t chunks;                   /* join launches (> n_steps when streaming) */
    int64_t max_rows;                 /* largest intermediate table held at once */
    double join_ms;                   /* device time of the join kernels (CUDA events) */
    int64_t join_launches;
    double join_bytes;                /* algorithmic bytes of the join launches */
    double total_ms;                  /* host wall time of the call */
    int64_t kernel_launches;          /* launches of the library's own kernels during the call */
} dm_stats;

/* Statistics of the last dm_match / dm_score_topk on this context. Device timings are
 * collected only after dm_enable_timing(ctx, 1). */
int dm_get_stats(dm_ctx *ctx, dm_stats *out);
int dm_enable_timing(dm_ctx *ctx, int on);

/* Many independent layout queries at once (no counterpart in the paper: a host-side runner
 * for callers with a batch of queries, each too small to fill the GPU alone). Query i
 * (0 <= i < n_q) is the pattern (n_p[i], p_row_ptr[i], p_col_idx[i]); it is planned with opts
 * (nullable) and answered exactly as dm_plan + dm_match_topk(mode, k) would answer it alone.
 * Context ctxs[t] (0 <= t < n_ctx, distinct contexts on one device, each with the same data
 * graph loaded as gids[t]) is driven by its own host thread; the threads take queries in
 * index order, so queries on different contexts overlap on the GPU. Outputs per query:
 * out_rows[i] (k x n_p[i] int32 host buffer, required), out_scores[i] (k floats; out_scores
 * or an entry may be NULL), out_n[i], and, where the arrays are not NULL, out_counts[i],
 * out_checksums[i] and out_status[i] (DM_OK or the query's error). cb, if not NULL, receives
 * every query's rows as dm_match_topk's callback would, plus the query index; it is called
 * from the worker threads and must be thread-safe. out_stats (nullable): the dm_stats fields
 * chunks, join_ms, join_launches, join_bytes and kernel_launches summed over the queries,
 * max_rows their maximum, total_ms the wall time of the call (n_steps 0). Returns DM_OK, or
 * the status of the lowest-numbered failing query (the others still run). */
typedef int (*dm_query_cb)(void *user, int32_t query, const int32_t *rows, const float *scores,
                           int64_t nrows, int32_t n_cols);
int dm_match_topk_queries(dm_ctx *const *ctxs, const dm_graph *gids, int32_t n_ctx, int32_t n_q,
                          const int32_t *n_p, const int32_t *const *p_row_ptr,
                          const int32_t *const *p_col_idx, const dm_plan_opts *opts, int mode,
                          dm_query_cb cb, void *user, int32_t k, int32_t *const *out_rows,
                          float *const *out_scores, int32_t *out_n, uint64_t *out_counts,
                          uint64_t *out_checksums, int32_t *out_status, dm_stats *out_stats);

/* Name of a DM_* status code, a static string (no counterpart in the paper). */
const char *dm_strerror(int code);

/* Text of the last CUDA failure seen by the context (empty if none); owned by the context. */
const char *dm_last_error(dm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DM_H */
