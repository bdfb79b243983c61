"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Embedding sets are compared bit-exactly in canonical order (integer work); FP32 layout scores
within 1e-5 relative of the FP64 oracle (the sum has at most ~150 non-negative terms, so FP32
recursive summation stays below 150 * 2^-24 ~ 9e-6 relative); top-k by position with the
tie rule of the library's reading (rows equal except inside the 1e-5 band around the k-th).
"""
import numpy as np
import pytest

import oracle
from paper_2508_21287_gb300 import inputs as I

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(0)
    yield c
    c.close()


def _rows_equal(a, b):
    assert a.shape == b.shape, (a.shape, b.shape)
    assert np.array_equal(a, b)


def check_all(ctx, gid, g, p, motifs=None, order=0, chunk_rows=0, scores=True, join_algo=0, induced=False,
              score_form=0):
    plan = ctx.plan(gid, p, motifs=motifs, order=order, chunk_rows=chunk_rows, join_algo=join_algo,
                    induced=induced)
    rows, sc, cnt, cs = plan.all()
    ref = oracle.enumerate(g, p, induced=induced)
    if chunk_rows:
        rows = rows[np.lexsort(rows.T[::-1])] if len(rows) else rows
    _rows_equal(rows, ref.rows)
    assert cnt == ref.count and cs == ref.checksum
    c2, cs2 = plan.count()
    assert c2 == ref.count and cs2 == ref.checksum
    if scores and g.edge_err is not None and ref.count:
        want = oracle.scores(g, p, rows, form=score_form)
        np.testing.assert_allclose(sc, want, rtol=RTOL, atol=0)
    return ref


def check_topk(ctx, gid, g, p, k, score_form=0, **kw):
    plan = ctx.plan(gid, p, **kw)
    rows, scores = plan.topk(k)
    assert_topk(g, p, oracle.enumerate(g, p).rows, rows, scores, k, score_form)


def assert_topk(g, p, allrows, rows, scores, k, score_form=0):
    """rows/scores are a correct top-k of the embeddings allrows (oracle order): scores equal the
    oracle's k best within RTOL, and every row scoring clearly below the k-th one is present."""
    m = min(k, len(allrows))
    assert rows.shape == (m, p.n)
    if m == 0:
        return
    s = oracle.scores(g, p, allrows, form=score_form)
    order = oracle.topk(allrows, s, k)
    np.testing.assert_allclose(scores, s[order], rtol=RTOL, atol=0)
    pos = {tuple(r): i for i, r in enumerate(allrows.tolist())}
    idx = [pos.get(tuple(r)) for r in rows.tolist()]
    assert None not in idx and len(set(idx)) == m
    np.testing.assert_allclose(s[idx], scores, rtol=RTOL, atol=0)
    kth = s[order[-1]]
    must = {i for i in np.nonzero(s < kth * (1 - RTOL))[0].tolist()}
    assert must <= set(idx)


# ------------------------------------------------------------------ 6x6 grid (tiny) -------
@pytest.mark.parametrize("motifs", [None, [2], [4, 2], [3], [104], [201], [104, 106], [202, 4]])
def test_grid6x6_path5_cycle4(ctx, motifs):
    g = I.grid(6, 6)
    gid = ctx.load(g)
    r = check_all(ctx, gid, g, I.path(5), motifs=motifs)
    assert r.count == 1712
    r = check_all(ctx, gid, g, I.cycle(4), motifs=motifs)
    assert r.count == 200


def test_grid6x6_brute_force(ctx):
    g = I.grid(6, 6)
    gid = ctx.load(g)
    plan = ctx.plan(gid, I.path(5))
    rows, _, cnt, _ = plan.all()
    _rows_equal(rows, oracle.brute_force(g, I.path(5)).rows)


# ------------------------------------------------------------------ motif tables ----------
def _motif_graph(mid):
    if 2 <= mid <= 16:
        return I.path(mid)
    if 103 <= mid <= 116:
        return I.cycle(mid - 100)
    if mid == 201:
        return I.star(3)
    if mid == 202:
        return I.grid(2, 3)
    if mid == 203:
        edges = [(i, (i + 1) % 12) for i in range(12)] + [(i, 12 + i // 2) for i in range(0, 12, 2)]
        return I.from_edges(18, edges)
    raise KeyError(mid)


@pytest.mark.parametrize("mid", [2, 3, 4, 5, 7, 103, 104, 106, 112, 201, 202, 203])
def test_motif_tables(ctx, mid):
    for g in (I.grid(5, 6), I.heavy_hex(2, 3), I.random_regular3(40, 3)):
        gid = ctx.load(g)
        got = ctx.motif_table(gid, mid)
        want = oracle.enumerate(g, _motif_graph(mid)).rows
        _rows_equal(got, want)


# ------------------------------------------------------------------ heavy-hex ~160 ---------
@pytest.fixture(scope="module")
def hh(ctx):
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=7, qubits=True)
    return g, ctx.load(g)


@pytest.mark.parametrize("seed", range(10))
def test_c2_patterns_all_scores(ctx, hh, seed):
    g, gid = hh
    check_all(ctx, gid, g, I.c2_pattern(seed))
    for n in (10, 20, 30):
        check_all(ctx, gid, g, I.sub_patch(g, n, seed))


@pytest.mark.parametrize("seed", range(6))
def test_c2_top100(ctx, hh, seed):
    g, gid = hh
    check_topk(ctx, gid, g, I.sub_patch(g, 12 + 3 * seed, seed), 100)
    check_topk(ctx, gid, g, I.path(8 + seed), 100)


@pytest.mark.parametrize("k_path,k", [(14, 100), (14, 1), (14, 1024), (18, 100), (22, 1024), (22, 7)])
def test_topk_single_block_and_tiled(ctx, hh, k_path, k):
    # 10856 rows take the single-block select, 31448 and 84724 the tile passes
    g, gid = hh
    check_topk(ctx, gid, g, I.path(k_path), k)


@pytest.mark.parametrize("seed", range(4))
def test_match_topk_one_pass(ctx, hh, B, seed):
    g, gid = hh
    p = I.layout_query(g, seed)
    plan = ctx.plan(gid, p)
    got = []
    rows_k, sc_k, cnt, cs = B.dm_match_topk(ctx.h, plan.h, B.DM_ALL, lambda r, s: got.append((r, s)) and 0, 100, p.n)
    ref = oracle.enumerate(g, p)
    rows = np.concatenate([r for r, _ in got])
    scores = np.concatenate([s for _, s in got])
    _rows_equal(rows, ref.rows)
    assert cnt == ref.count and cs == ref.checksum
    s = oracle.scores(g, p, ref.rows)
    np.testing.assert_allclose(scores, s, rtol=RTOL, atol=0)
    order = oracle.topk(ref.rows, s, 100)
    np.testing.assert_allclose(sc_k, s[order], rtol=RTOL, atol=0)
    st = B.dm_get_stats(ctx.h)
    assert st["kernel_launches"] > 0 and st["join_launches"] == st["chunks"]


@pytest.mark.parametrize("chunk_rows", [0, 700])
def test_match_topk_device_rows_and_streamed(ctx, hh, B, chunk_rows):
    # the benchmark's call (device rows) and a streamed result (several flushes): the top-k and
    # the checksum are the oracle's either way
    g, gid = hh
    for seed in (4, 5):
        p = I.layout_query(g, seed)
        plan = ctx.plan(gid, p, chunk_rows=chunk_rows)
        seen = []
        rows_k, sc_k, cnt, cs = B.dm_match_topk(ctx.h, plan.h, B.DM_ALL | B.DM_DEVICE_ROWS,
                                                lambda r, s, m, n: seen.append(m) and 0, 100, p.n)
        ref = oracle.enumerate(g, p)
        assert cnt == ref.count == sum(seen) and cs == ref.checksum
        s = oracle.scores(g, p, ref.rows)
        order = oracle.topk(ref.rows, s, 100)
        np.testing.assert_allclose(sc_k, s[order], rtol=RTOL, atol=0)
        assert rows_k.shape == (min(100, ref.count), p.n)


def test_many_queries_over_several_contexts(ctx, hh, B):
    # the multi-context runner answers each query exactly as one dm_match_topk call alone;
    # host rows (with the query index) and device rows both reach the callback
    g, gid = hh
    qs = [I.layout_query(g, s) for s in range(12)]
    pats = [(q.n, q.row_ptr, q.col_idx) for q in qs]
    ctxs = [B.Context(0) for _ in range(3)]
    try:
        gids = [c.load(g) for c in ctxs]
        got = {}
        res, st = B.dm_match_topk_queries([c.h for c in ctxs], gids, pats, 100,
                                          cb=lambda i, r, s: got.setdefault(i, []).append((r, s)) and 0)
        launches = 0
        for i, (q, (rows_k, sc_k, cnt, cs, status)) in enumerate(zip(qs, res)):
            assert status == B.DM_OK
            plan = ctx.plan(gid, q)
            one = []
            r1, s1, c1, cs1 = B.dm_match_topk(ctx.h, plan.h, B.DM_ALL, lambda r, s: one.append((r, s)) and 0, 100, q.n)
            launches += B.dm_get_stats(ctx.h)["kernel_launches"]
            assert (cnt, cs) == (c1, cs1)
            assert np.array_equal(rows_k, r1) and np.array_equal(sc_k, s1)
            rows = np.concatenate([r for r, _ in got[i]])
            assert np.array_equal(rows, np.concatenate([r for r, _ in one]))
            assert np.array_equal(np.concatenate([s for _, s in got[i]]), np.concatenate([s for _, s in one]))
            if i < 4:
                ref = oracle.enumerate(g, q, rows=False)
                assert (cnt, cs) == (ref.count, ref.checksum)
        assert st["kernel_launches"] >= launches > 0 and st["join_launches"] > 0
        seen = {}
        res2, _ = B.dm_match_topk_queries([c.h for c in ctxs], gids, pats, 7, mode=B.DM_ALL | B.DM_DEVICE_ROWS,
                                          cb=lambda i, r, s, m, n: seen.__setitem__(i, seen.get(i, 0) + m) and 0)
        for i, (rows_k, sc_k, cnt, cs, status) in enumerate(res2):
            assert status == B.DM_OK and cnt == res[i][2] == seen.get(i, 0) and cs == res[i][3]
            assert np.array_equal(rows_k, res[i][0][:7])
        res3, _ = B.dm_match_topk_queries([ctxs[0].h], gids[:1], pats[:3], 5)  # one context, no callback
        assert [x[2:4] for x in res3] == [x[2:4] for x in res[:3]]
        res0, st0 = B.dm_match_topk_queries([c.h for c in ctxs], gids, [], 5)
        assert res0 == [] and st0["kernel_launches"] == 0
        with pytest.raises(B.DMError):
            B.dm_match_topk_queries([ctxs[0].h, ctxs[0].h], gids[:2], pats[:2], 5)
    finally:
        for c in ctxs:
            c.close()


def test_topk_more_than_count_and_no_embeddings(ctx, hh, B):
    g, gid = hh
    check_topk(ctx, gid, g, I.cycle(12), 1000)      # 576 < k
    check_topk(ctx, gid, g, I.cycle(8), 10)         # girth 12: none
    ug = I.heavy_hex(2, 2)
    ugid = ctx.load(ug)
    with pytest.raises(B.DMError):
        ctx.plan(ugid, I.path(4)).topk(5)           # no weights loaded


@pytest.mark.parametrize("k", [10, 16, 24, 30])
def test_heavy_hex_paths(ctx, hh, k):
    g, gid = hh
    r = check_all(ctx, gid, g, I.path(k), scores=k <= 16)
    assert r.count == {10: 3696, 16: 18528, 24: 138648, 30: 548048}.get(k, r.count)


# ------------------------------------------------------------------ orders, chunks ---------
@pytest.mark.parametrize("order", [0, 1])
def test_orders_agree(ctx, hh, order):
    g, gid = hh
    for s in range(4):
        check_all(ctx, gid, g, I.sub_patch(g, 18, 100 + s), order=order)
        check_all(ctx, gid, g, I.random_tree(14, s), order=order)


@pytest.mark.parametrize("chunk_rows", [64, 1000, 20000])
def test_chunked_streaming(ctx, hh, chunk_rows):
    g, gid = hh
    check_all(ctx, gid, g, I.path(16), chunk_rows=chunk_rows, scores=False)
    check_all(ctx, gid, g, I.sub_patch(g, 25, 3), chunk_rows=chunk_rows)


def test_small_budget_streams(B, hh):
    g, _ = hh
    with B.Context(0, mem_budget_bytes=2 << 20) as c:
        gid = c.load(g)
        plan = c.plan(gid, I.path(20))
        cnt, cs = plan.count()
        ref = oracle.enumerate(g, I.path(20), rows=False)
        assert cnt == ref.count and cs == ref.checksum
        rows, _, cnt2, cs2 = plan.all()
        assert cnt2 == ref.count and cs2 == ref.checksum
        assert c.stats()["chunks"] > c.stats()["n_steps"]


@pytest.mark.parametrize("n", [24, 36])
def test_long_cycle_two_key_path_join(ctx, hh, n):
    # a cycle as two half-length path slices joined on both end vertices (hashed 2-key index)
    g, gid = hh
    check_all(ctx, gid, g, I.cycle(n), motifs=sorted({(n + 1) // 2 + 1, n // 2 + 1}, reverse=True) + [4])


def test_cycle40_half_paths_count(ctx):
    g = I.heavy_hex(12, 6)
    gid = ctx.load(g)
    plan = ctx.plan(gid, I.cycle(40), motifs=[21, 4])
    assert [s["motif"] for s in plan.describe()][:2] == [21, 21]
    cnt, cs = plan.count()
    ref = oracle.enumerate(g, I.cycle(40), rows=False, threads=8)
    assert cnt == ref.count == 402240 and cs == ref.checksum


@pytest.mark.parametrize("motifs", [None, [104], [4, 2], [202, 4]])
def test_sort_merge_join_grid(ctx, B, motifs):
    # the sort-merge join (R sorted by its key columns, motif groups found in the sorted packed
    # keys) gives the same rows, scores and checksums as the oracle, for one- and two-key joins
    g = I.lognormal_weights(I.grid(6, 6), seed=5)
    gid = ctx.load(g)
    for p in (I.path(5), I.cycle(4), I.grid(2, 3), I.random_tree(9, 4)):
        check_all(ctx, gid, g, p, motifs=motifs, join_algo=B.DM_JOIN_SORTMERGE)


@pytest.mark.parametrize("seed", range(3))
def test_sort_merge_join_heavy_hex(ctx, hh, B, seed):
    g, gid = hh
    check_all(ctx, gid, g, I.layout_query(g, seed), join_algo=B.DM_JOIN_SORTMERGE)
    check_all(ctx, gid, g, I.cycle(24), motifs=[13, 4], join_algo=B.DM_JOIN_SORTMERGE)
    plan = ctx.plan(gid, I.path(12 + seed), join_algo=B.DM_JOIN_SORTMERGE, chunk_rows=500)
    ref = oracle.enumerate(g, I.path(12 + seed), rows=False)
    assert plan.count() == (ref.count, ref.checksum)


@pytest.mark.parametrize("motifs", [None, [2], [4, 2], [104], [202, 4]])
def test_induced_matching_grid(ctx, motifs):
    # induced embeddings (non-adjacent pattern vertices on non-adjacent data vertices): the
    # oracle's induced enumeration, itself pinned by brute force and closed forms
    g = I.lognormal_weights(I.grid(6, 6), seed=9)
    gid = ctx.load(g)
    for p in (I.path(4), I.path(6), I.cycle(4), I.star(4), I.grid(2, 3), I.random_tree(8, 2), I.cycle(8)):
        check_all(ctx, gid, g, p, motifs=motifs, induced=True)


@pytest.mark.parametrize("seed", range(4))
def test_induced_matching_heavy_hex_and_random(ctx, hh, B, seed):
    g, gid = hh
    check_all(ctx, gid, g, I.layout_query(g, seed), induced=True)
    check_all(ctx, gid, g, I.sub_patch(g, 14 + seed, seed), induced=True, join_algo=B.DM_JOIN_SORTMERGE)
    r = I.random_regular3(40, seed)
    rg = ctx.load(r)
    for p in (I.path(5), I.cycle(5), I.random_tree(7, seed)):
        check_all(ctx, rg, r, p, induced=True, scores=False)
        plan = ctx.plan(rg, p, induced=True, chunk_rows=7)
        ref = oracle.enumerate(r, p, induced=True)
        assert plan.count() == (ref.count, ref.checksum)


def test_log_fidelity_scores(ctx, B):
    # scores as -log(product of fidelities 1 - e): FP32 sums of -log1p(-e) against FP64
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=21, qubits=True)
    gid = ctx.load(g, score_form=B.DM_SCORE_LOG_FIDELITY)
    for seed in range(4):
        check_all(ctx, gid, g, I.layout_query(g, seed), score_form=1)
        check_topk(ctx, gid, g, I.layout_query(g, 10 + seed), 50, score_form=1)
    check_topk(ctx, gid, g, I.path(18), 100, score_form=1)  # the selection-first top-k
    bad = I.lognormal_weights(I.grid(3, 3), seed=2)
    bad.edge_err = bad.edge_err.copy()
    bad.edge_err[:] = 1.0
    with pytest.raises(B.DMError) as e:
        ctx.load(bad, score_form=B.DM_SCORE_LOG_FIDELITY)
    assert e.value.code == B.DM_E_INVAL


# ------------------------------------------------------------------ larger heavy-hex -------
@pytest.mark.parametrize("m,n", [(12, 15), (27, 28)])
def test_scaling_counts(ctx, m, n):
    g = I.heavy_hex(m, n)
    gid = ctx.load(g)
    for p in (I.path(8), I.path(16), I.path(24), I.sub_patch(g, 12, 1), I.sub_patch(g, 25, 2), I.sub_patch(g, 40, 3)):
        plan = ctx.plan(gid, p)
        cnt, cs = plan.count()
        ref = oracle.enumerate(g, p, rows=False, threads=8)
        assert cnt == ref.count and cs == ref.checksum


def test_scaling_rows_heavy_hex_27x28(ctx):
    # every embedding row, not only count and checksum, at the scaling workload's middle size
    # (V = 3999): the device-driven chain with its 16-byte-padded intermediate tables, then the
    # canonical sort, against the oracle's rows element by element
    g = I.heavy_hex(27, 28)
    gid = ctx.load(g)
    for p in (I.path(16), I.path(20), I.sub_patch(g, 30, 4)):
        rows, _, cnt, cs = ctx.plan(gid, p).all()
        ref = oracle.enumerate(g, p, threads=16)
        assert cnt == ref.count > 0 and cs == ref.checksum
        _rows_equal(rows, ref.rows)


def test_largest_heavy_hex_p24(ctx):
    g = I.heavy_hex(53, 59)
    gid = ctx.load(g)
    plan = ctx.plan(gid, I.path(24))
    cnt, cs = plan.count()
    ref = oracle.enumerate(g, I.path(24), rows=False, threads=16)
    assert cnt == ref.count and cs == ref.checksum


def test_c3_benchmark_queries_match_oracle(ctx, B):
    # the benchmark's default workload at full size: heavy-hex 53x59 and its 32 seeded queries,
    # each planned and counted as bench.py times them (one context, the device-driven chain of
    # join launches with padded intermediate tables), unfused and with the last two joins fused;
    # every count and checksum equals the oracle's
    import bench
    g, pats = bench.workload(0, bench.BATCH, "c3")
    gid = ctx.load(g)
    try:
        for p in pats:
            ref = oracle.enumerate(g, p, rows=False, threads=16)
            plan = ctx.plan(gid, p)
            for fuse in (0, 1):
                B.dm_set_fusion(ctx.h, fuse)
                assert plan.count() == (ref.count, ref.checksum), (p.n, fuse)
                st = ctx.stats()
                assert st["chunks"] == st["n_steps"]  # one device-driven chain, no streaming
    finally:
        B.dm_set_fusion(ctx.h, 0)


def test_c2_benchmark_queries_match_oracle(B):
    # the C2 benchmark step as bench.py times it: its 32 seeded layout queries on the weighted
    # heavy-hex 4x6 graph, over 8 contexts, every embedding with its score and the top-100 of
    # each; rows, scores, count, checksum and top-100 all agree with the oracle
    import bench
    g, pats = bench.workload(0, bench.BATCH, "c2")
    ctxs = [B.Context(0) for _ in range(8)]
    try:
        gids = [c.load(g) for c in ctxs]
        got = {}
        res, _ = B.dm_match_topk_queries([c.h for c in ctxs], gids, [(q.n, q.row_ptr, q.col_idx) for q in pats],
                                         bench.K_TOP, cb=lambda i, r, s: got.setdefault(i, []).append((r, s)) and 0)
        for i, (q, (rows_k, sc_k, cnt, cs, status)) in enumerate(zip(pats, res)):
            assert status == B.DM_OK
            ref = oracle.enumerate(g, q)
            assert (cnt, cs) == (ref.count, ref.checksum)
            rows = np.concatenate([r for r, _ in got[i]]) if i in got else np.zeros((0, q.n), np.int32)
            scores = np.concatenate([s for _, s in got[i]]) if i in got else np.zeros(0, np.float32)
            _rows_equal(rows, ref.rows)
            np.testing.assert_allclose(scores, oracle.scores(g, q, ref.rows), rtol=RTOL, atol=0)
            assert_topk(g, q, ref.rows, rows_k, sc_k, bench.K_TOP)
    finally:
        for c in ctxs:
            c.close()


def test_streaming_far_beyond_the_budget_is_consistent(ctx, B):
    # a 37-vertex path in heavy-hex 53x59: billions of embeddings, intermediate tables of
    # hundreds of GB streamed depth-first in budget-sized chunks; two budgets (different
    # chunkings) must give the same count and order-independent checksum
    g = I.heavy_hex(53, 59)
    gid = ctx.load(g)
    plan = ctx.plan(gid, I.path(37))
    got = []
    try:
        for budget in (24 << 30, 8 << 30):
            B.dm_set_budget(ctx.h, budget)
            got.append(plan.count())
            st = ctx.stats()
            assert st["chunks"] > 2 * st["n_steps"]
    finally:
        B.dm_set_budget(ctx.h, 0)
    assert got[0] == got[1] and got[0][0] > 10 ** 9


def test_patterns_beyond_64_vertices(ctx, B):
    # 91- and 106-vertex heavy-hex patches in larger heavy-hex graphs (rigid: few placements),
    # and random connected 80- and 100-vertex sub-patches of the 4485-vertex heavy-hex
    for (a, b), (c, d) in (((3, 7), (2, 6)), ((4, 6), (3, 5))):
        g, p = I.heavy_hex(a, b), I.heavy_hex(c, d)
        assert p.n > 64
        check_all(ctx, ctx.load(g), g, p, scores=False)
    g = I.heavy_hex(25, 34)
    gid = ctx.load(g)
    for n, seed in ((80, 1), (100, 1), (100, 2)):
        p = I.sub_patch(g, n, seed)
        ref = oracle.enumerate(g, p, rows=False, threads=16)
        # the greedy order keeps the intermediate tables near the result size at this scale
        # (the paper's order streams hundreds of millions of rows on some of them)
        assert ctx.plan(gid, p, order=B.DM_ORDER_HEURISTIC).count() == (ref.count, ref.checksum)


# ------------------------------------------------------------------ other graphs -----------
def _er(n, p1000, seed):
    rng = I.SplitMix64(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.below(1000) < p1000]
    edges += [(i, i + 1) for i in range(n - 1)]  # keep it connected
    return I.from_edges(n, edges)


@pytest.mark.parametrize("seed", range(8))
def test_dense_random_graphs(ctx, seed):
    g = _er(12, 350, seed)
    gid = ctx.load(g)
    pats = [I.complete(3), I.complete(4), I.cycle(5), I.random_tree(6, seed), I.cycle_with_chords(6, seed)]
    for p in pats:
        for motifs in (None, [2], [103], [4], [104, 3]):
            check_all(ctx, gid, g, p, motifs=motifs)


def test_regular3_and_grid32(ctx):
    g = I.random_regular3(256, 5)
    gid = ctx.load(g)
    for p in (I.path(7), I.cycle(6), I.random_tree(9, 2)):
        check_all(ctx, gid, g, p, scores=False)
    g = I.grid(12, 12)
    gid = ctx.load(g)
    for p in (I.path(7), I.cycle(8), I.subdivided_grid(2, 2), I.grid(2, 3)):
        check_all(ctx, gid, g, p, scores=False)


def test_relabelled_data_graph(ctx):
    g = I.heavy_hex(3, 3)
    rng = I.SplitMix64(9)
    perm = list(range(g.n))
    rng.shuffle(perm)
    h = I.relabel(g, perm)
    p = I.sub_patch(g, 15, 4)
    a = ctx.plan(ctx.load(g), p).all()[0]
    b = ctx.plan(ctx.load(h), p).all()[0]
    mapped = np.asarray(perm, dtype=np.int32)[a]
    mapped = mapped[np.lexsort(mapped.T[::-1])]
    _rows_equal(mapped, b)


# ------------------------------------------------------------------ images (dedup) ---------
@pytest.mark.parametrize("pat", [I.path(6), I.cycle(12), I.star(3), I.random_tree(9, 4), I.grid(2, 3)])
def test_images_dedup(ctx, B, pat):
    g = I.grid(7, 7) if pat.name == "grid2x3" else I.heavy_hex(3, 4)
    gid = ctx.load(g)
    plan = ctx.plan(gid, pat)
    got = B.dm_images(ctx.h, plan.h, pat.n)
    ref = oracle.enumerate(g, pat)
    want = oracle.images(ref.rows)
    _rows_equal(got, want)
    assert len(got) * oracle.automorphisms(pat) == ref.count


# ------------------------------------------------------------------ edge cases -------------
def test_edge_cases(ctx, B):
    g = I.lognormal_weights(I.grid(4, 4), seed=1)
    gid = ctx.load(g)
    one = I.from_edges(1, [])
    check_all(ctx, gid, g, one)                                   # every vertex
    check_all(ctx, gid, g, I.path(2))                              # = 2|E|
    assert check_all(ctx, gid, g, I.path(17)).count == 0          # larger than the graph
    assert check_all(ctx, gid, g, I.complete(3)).count == 0       # no triangles in a grid
    two = I.from_edges(4, [(0, 1), (2, 3)])
    with pytest.raises(B.DMError) as e:
        ctx.plan(gid, two)
    assert e.value.code == B.DM_E_DISCONNECTED
    with pytest.raises(B.DMError) as e:
        B.dm_load_data_graph(ctx.h, 3, [0, 1, 2, 2], [1, 0], None, None)  # 0-1 plus isolated 2
    assert e.value.code == B.DM_E_DISCONNECTED
    with pytest.raises(B.DMError) as e:
        B.dm_load_data_graph(ctx.h, 2, [0, 1, 1], [1], None, None)        # asymmetric
    assert e.value.code == B.DM_E_INVAL
    with pytest.raises(B.DMError) as e:
        B.dm_load_data_graph(ctx.h, 2, [0, 2, 3], [1, 1, 0], None, None)  # duplicate edge
    assert e.value.code == B.DM_E_INVAL
    # self-loops are dropped on load (Res(M2) excludes them)
    sl = B.dm_load_data_graph(ctx.h, 3, [0, 2, 5, 6], [0, 1, 0, 1, 2, 1], None, None)
    assert ctx.motif_table(sl, 2).tolist() == [[0, 1], [1, 0], [1, 2], [2, 1]]


def test_capacity_cap(ctx, B, hh):
    g, gid = hh
    plan = ctx.plan(gid, I.path(20), max_rows=1000)
    with pytest.raises(B.DMError) as e:
        plan.count()
    assert e.value.code == B.DM_E_CAPACITY


def test_callback_cancel(ctx, B, hh):
    g, gid = hh
    plan = ctx.plan(gid, I.path(6))
    with pytest.raises(B.DMError) as e:
        B.dm_match(ctx.h, plan.h, B.DM_ALL, lambda r, s: 1)
    assert e.value.code == B.DM_E_CANCELLED


# ------------------------------------------------------------------ weight preconditions ---
def _with_negative_edges(g, frac_seed: int, value: float = -0.02):
    """A copy of g whose every third undirected edge (in a seeded order) weighs `value`."""
    import copy
    h = copy.deepcopy(g)
    edges = h.edges()
    rng = I.SplitMix64(frac_seed)
    neg = {e for e in edges if rng.below(3) == 0}
    for u in range(h.n):
        for k in range(h.row_ptr[u], h.row_ptr[u + 1]):
            v = int(h.col_idx[k])
            if (min(u, v), max(u, v)) in neg:
                h.edge_err[k] = value
    return h


@pytest.mark.parametrize("chunk_rows", [0, 64])
@pytest.mark.parametrize("case", ["hh3x4", "hh4x6_p18"])
def test_negative_weights_topk_is_exact(ctx, B, chunk_rows, case):
    # Sec. 5.4 ranks layouts by a sum of weights. With a negative weight a row's partial score
    # is no lower bound of its final score, so the joins must not drop rows by partial score
    # (the streamed plan, chunk_rows 64, is where a pruning join would lose rows), and every
    # selection must order negative scores by value (the single-block select, the tile passes
    # and, for k > 1024, the radix select with the stable score sort). FP32 sums are compared
    # with the FP64 oracle within 1e-5 of the sum of the terms' magnitudes (the error bound of
    # a recursive sum of mixed signs).
    if case == "hh3x4":
        base = I.lognormal_weights(I.heavy_hex(3, 4), seed=21, qubits=False)
        pats, ks = (I.path(9), I.sub_patch(base, 14, 3)), (1, 10, 50)
    else:
        base = I.lognormal_weights(I.heavy_hex(4, 6), seed=22, qubits=False)
        pats, ks = (I.path(18),), (7, 1100)
    g = _with_negative_edges(base, 99)
    assert (g.edge_err < 0).any() and (g.edge_err > 0).any()
    gid = ctx.load(g)
    gabs = _with_negative_edges(base, 99, value=0.02)
    for p in pats:
        allrows = oracle.enumerate(g, p).rows
        s = oracle.scores(g, p, allrows)
        mag = oracle.scores(gabs, p, allrows)  # sum of |terms| per row
        assert (s < 0).any()
        for k in ks:
            plan = ctx.plan(gid, p, chunk_rows=chunk_rows)
            rows, scores = plan.topk(k)
            m = min(k, len(allrows))
            assert rows.shape == (m, p.n)
            pos = {tuple(r): i for i, r in enumerate(allrows.tolist())}
            idx = [pos.get(tuple(r)) for r in rows.tolist()]
            assert None not in idx and len(set(idx)) == m
            tol = RTOL * mag[idx]
            assert np.all(np.abs(scores - s[idx]) <= tol)
            order = oracle.topk(allrows, s, k)
            band = RTOL * mag.max()
            assert np.all(np.abs(scores - s[order]) <= band)
            assert np.all(np.diff(scores) >= 0)
            kth = s[order[-1]]
            must = set(np.nonzero(s < kth - band)[0].tolist())
            assert must <= set(idx)


def test_non_finite_weights_rejected_and_not_registered(ctx, B):
    # weights must be finite; a graph that fails to load takes no handle and holds nothing
    g = I.lognormal_weights(I.heavy_hex(2, 3), seed=5)
    gid0 = ctx.load(g)
    for bad in (np.nan, np.inf, -np.inf):
        h = I.lognormal_weights(I.heavy_hex(2, 3), seed=5)
        h.edge_err = h.edge_err.copy()
        h.edge_err[3] = bad
        with pytest.raises(B.DMError) as e:
            ctx.load(h)
        assert e.value.code == B.DM_E_INVAL
    q = I.lognormal_weights(I.heavy_hex(2, 3), seed=5, qubits=True)
    q.qubit_err = q.qubit_err.copy()
    q.qubit_err[0] = np.nan
    with pytest.raises(B.DMError):
        ctx.load(q)
    gid1 = ctx.load(g)
    assert gid1 == gid0 + 1
    r = check_all(ctx, gid1, g, I.path(6))
    assert r.count > 0


# ------------------------------------------------------------------ R_0 shards -------------
@pytest.mark.parametrize("n_shards", [2, 3, 7])
def test_r0_shards_partition_the_embeddings(ctx, B, hh, n_shards):
    # each shard of the first table is the oracle's part (image of the shard vertex modulo the
    # shard count), and the shards' counts and checksums sum (mod 2^64) to the whole
    g, gid = hh
    m64 = (1 << 64) - 1
    for p, kw in ((I.path(14), {}), (I.sub_patch(g, 20, 4), {}), (I.path(12), {"chunk_rows": 500})):
        plan = ctx.plan(gid, p, **kw)
        v0 = plan.describe()[0]["slice"][0]
        rows = oracle.enumerate(g, p).rows
        tot_c, tot_s = 0, 0
        for sh in range(n_shards):
            c, s = B.dm_match_shard(ctx.h, plan.h, sh, n_shards)
            part = rows[rows[:, v0] % n_shards == sh]
            assert (c, s) == (len(part), oracle.checksum(part))
            tot_c, tot_s = tot_c + c, (tot_s + s) & m64
        assert (tot_c, tot_s) == plan.count()
    with pytest.raises(B.DMError):
        B.dm_match_shard(ctx.h, plan.h, 3, 3)


# ------------------------------------------------------------------ fused last two joins ----
@pytest.mark.parametrize("graph", ["hh", "grid", "rr3"])
def test_fused_last_two_joins_equal_unfused_and_oracle(ctx, B, hh, graph):
    # a counted plan's last two joins run as one kernel (the table between them stays in
    # shared memory); counts and checksums must equal the step-by-step run and the oracle,
    # also when the pair starts at the seed step (two-step plans) and with back-edges
    if graph == "hh":
        g, gid = hh
        pats = [I.path(7), I.path(10), I.path(13), I.path(22), I.cycle(12), I.sub_patch(g, 16, 2),
                I.sub_patch(g, 25, 9), I.layout_query(g, 3)]
    elif graph == "grid":
        g = I.grid(9, 9)
        gid = ctx.load(g)
        pats = [I.path(5), I.path(8), I.cycle(4), I.cycle(8), I.grid(2, 3), I.sub_patch(g, 9, 1)]
    else:
        g = I.random_regular3(200, 7)
        gid = ctx.load(g)
        pats = [I.path(6), I.path(9), I.star(3), I.random_tree(8, 5), I.sub_patch(g, 10, 4)]
    for p in pats:
        plan = ctx.plan(gid, p)
        ref = oracle.enumerate(g, p, rows=False, threads=8)
        B.dm_set_fusion(ctx.h, True)
        fused = plan.count()
        B.dm_set_fusion(ctx.h, False)
        plain = plan.count()
        B.dm_set_fusion(ctx.h, True)
        assert fused == plain == (ref.count, ref.checksum), p.name
