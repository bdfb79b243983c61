"""Persistent batch kernel (dm_match_batch) against the oracle and against dm_match alone.

One launch runs count + checksum for every plan; each plan's result must equal its own
single-plan run and the oracle's, for uneven plan sizes, plans with no embedding, two-key
(hash-indexed) joins, every autotuned launch shape and a changed hash load factor.
"""
import numpy as np
import pytest

import oracle
from paper_2508_21287_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


def _run(B, ctx, gid, pats, **kw):
    plans = [B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx, **kw) for p in pats]
    counts, sums = B.dm_match_batch(ctx.h, plans, B.DM_COUNT)
    single = [B.dm_match(ctx.h, pl, B.DM_COUNT) for pl in plans]
    for pl in plans:
        B.dm_plan_free(pl)
    return counts, sums, single


def _run_shape(B, ctx, gid, pats, threads):
    """_run with a fixed block shape (autotuning off); also returns the batch's configuration."""
    B.dm_set_batch_shape(ctx.h, threads, 1 if threads == 256 else 0)
    try:
        counts, sums, single = _run(B, ctx, gid, pats)
        return counts, sums, B.dm_batch_config(ctx.h)
    finally:
        B.dm_set_batch_shape(ctx.h, 256, 0)


def _check(g, pats, counts, sums, single):
    for p, c, s, (c1, s1) in zip(pats, counts.tolist(), sums.tolist(), single):
        ref = oracle.enumerate(g, p, rows=False, threads=8)
        assert (c, s) == (ref.count, ref.checksum), p.name
        assert (c1, s1) == (c, s)


def test_batch_mixed_heavy_hex(B):
    g = I.heavy_hex(12, 6)
    pats = [I.mixed_pattern(s, 5, 40) for s in range(60)]
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        counts, sums, single = _run(B, ctx, gid, pats)
        _check(g, pats, counts, sums, single)
        cfg = B.dm_batch_config(ctx.h)
        assert cfg["tile_rows"] in (32, 64, 128) and cfg["root_chunk"] in (4, 16, 64)
        # the autotuner also picked a block shape and a two-key hash load factor
        assert cfg["threads_per_cta"] in (32, 128, 256) and cfg["ctas_per_sm"] >= 1
        assert cfg["hash_load_factor"] in (0.25, 0.5, 0.75)
        # the same plans again: the cached device image and graph are replayed
        counts2, sums2, _ = _run(B, ctx, gid, pats)
        assert np.array_equal(counts, counts2) and np.array_equal(sums, sums2)
        # every block shape and load factor gives the oracle's counts and checksums
        for th, lf in ((128, 0.25), (256, 0.75), (32, 0.5)):
            B.dm_set_tuning(ctx.h, autotune=False, hash_load_factor=lf)
            counts3, sums3, cfg3 = _run_shape(B, ctx, gid, pats, th)
            assert np.array_equal(counts, counts3) and np.array_equal(sums, sums3)
            assert cfg3["hash_load_factor"] == lf and cfg3["threads_per_cta"] == th
            if th == 32:  # warp walks take 32-row tiles
                assert cfg3["tile_rows"] == 32


def test_batch_candidate_plans_with_wide_steps(B):
    # every candidate plan of long cycles and mixed patterns: half-length path slices map up
    # to 19 new vertices a step, tested in per-row id bitmaps inside the CTA batch kernel and
    # read lazily from the motif rows by the warp walks
    g = I.heavy_hex(12, 6)
    pats = [I.cycle(n) for n in (24, 30, 36, 39, 40)] + [I.mixed_pattern(s, 16, 40) for s in range(20)]
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        plans, owner = [], []
        for i, p in enumerate(pats):
            for pl in B.dm_plan_candidates(ctx.h, gid, p.n, p.row_ptr, p.col_idx):
                plans.append(pl)
                owner.append(i)
        assert any(max(s["motif"] for s in B.dm_plan_describe(pl)) > 8 for pl in plans)
        refs = [oracle.enumerate(g, p, rows=False, threads=8) for p in pats]
        for shape in (None, 32, 256):  # autotuned, warp walks, 256-thread CTAs
            if shape is not None:  # plans predicted above 2^20 rows run step by step, as tuned
                B.dm_set_tuning(ctx.h, autotune=False, hash_load_factor=0.5, heavy_rows=1048576.0)
                B.dm_set_batch_shape(ctx.h, shape, 0)
            counts, sums = B.dm_match_batch(ctx.h, plans, B.DM_COUNT)
            if shape is not None:
                assert B.dm_batch_config(ctx.h)["threads_per_cta"] == shape
            for i, c, s in zip(owner, counts.tolist(), sums.tolist()):
                assert (c, s) == (refs[i].count, refs[i].checksum), (pats[i].name, shape)
        for pl in plans:
            B.dm_plan_free(pl)


@pytest.mark.parametrize("shape", [None, 32])  # autotuned, warp walks
def test_batch_sort_merge_plans(B, shape):
    g = I.heavy_hex(12, 6)
    pats = [I.mixed_pattern(s, 5, 30) for s in range(30)] + [I.cycle(24)]
    with B.Context(0) as ctx:
        if shape is not None:
            B.dm_set_tuning(ctx.h, False, 0.5)
            B.dm_set_batch_shape(ctx.h, shape, 0)
        gid = ctx.load(g)
        counts, sums, single = _run(B, ctx, gid, pats, join_algo=B.DM_JOIN_SORTMERGE)
        _check(g, pats, counts, sums, single)


def test_c4_full_batch_matches_oracle(B):
    # the benchmark's whole C4 batch (512 patterns of 5-40 vertices on heavy-hex 12x6) in one
    # persistent launch, with paper plans and with the cheapest candidate plan of each pattern
    import sys
    import os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    g, pats = bench.workload(0, 512, "c4")
    refs = [oracle.enumerate(g, p, rows=False, threads=16) for p in pats]
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        paper = [B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx) for p in pats]
        cheap = []
        for p in pats:
            cands = B.dm_plan_candidates(ctx.h, gid, p.n, p.row_ptr, p.col_idx)
            best = min(range(len(cands)), key=lambda i: B.dm_plan_cost(cands[i])[0])
            cheap.append(cands[best])
            for i, c in enumerate(cands):
                if i != best:
                    B.dm_plan_free(c)
        for plans in (paper, cheap):
            counts, sums = B.dm_match_batch(ctx.h, plans, B.DM_COUNT)
            for p, r, c, s in zip(pats, refs, counts.tolist(), sums.tolist()):
                assert (c, s) == (r.count, r.checksum), p.name
        # both kernel forms on their own: CTA walks and warp walks
        B.dm_set_tuning(ctx.h, autotune=False, hash_load_factor=0.5)
        for shape in (256, 32):
            B.dm_set_batch_shape(ctx.h, shape, 0)
            for plans in (paper, cheap):
                counts, sums = B.dm_match_batch(ctx.h, plans, B.DM_COUNT)
                for p, r, c, s in zip(pats, refs, counts.tolist(), sums.tolist()):
                    assert (c, s) == (r.count, r.checksum), (p.name, shape)
        for pl in paper + cheap:
            B.dm_plan_free(pl)


@pytest.mark.parametrize("shape", [256, 32])  # CTA walks, warp walks
def test_batch_paths_and_patches(B, shape):
    g = I.heavy_hex(8, 9)
    pats = [I.path(k) for k in (2, 3, 4, 7, 12, 20, 28)] + [I.sub_patch(g, n, n) for n in (5, 15, 25, 40)]
    pats += [I.from_edges(1, [])]  # single vertex: one-step plan
    pats += [I.star(3), I.cycle(12)]  # patterns that are motifs themselves: one-step plans
    with B.Context(0) as ctx:
        gid = ctx.load(g)
        B.dm_set_tuning(ctx.h, False, 0.5)
        B.dm_set_batch_shape(ctx.h, shape, 0)
        counts, sums, single = _run(B, ctx, gid, pats)
        _check(g, pats, counts, sums, single)
        lat = B.dm_batch_latency(ctx.h, len(pats))
        assert np.all(lat >= 0)
        # the heaviest plans step by step, the rest in the persistent launch: same results
        B.dm_set_tuning(ctx.h, False, 0.5, heavy_rows=5000.0)
        counts2, sums2, _ = _run(B, ctx, gid, pats)
        cfg = B.dm_batch_config(ctx.h)
        assert cfg["stepwise_plans"] > 0 and cfg["threads_per_cta"] == shape
        assert np.array_equal(counts, counts2) and np.array_equal(sums, sums2)


@pytest.mark.parametrize("lf,shape", [(0.25, None), (0.9, None), (0.5, 32), (0.5, 128)])
def test_batch_two_key_joins_on_grid(B, lf, shape):
    g = I.grid(10, 10)
    pats = [I.cycle(4), I.cycle(6), I.cycle(8), I.grid(2, 3), I.grid(3, 3), I.subdivided_grid(2, 2),
            I.random_tree(7, 1), I.path(6)]
    with B.Context(0) as ctx:
        B.dm_set_tuning(ctx.h, shape is None, lf)  # None: autotuned
        if shape is not None:
            B.dm_set_batch_shape(ctx.h, shape, 0)
        gid = ctx.load(g)
        counts, sums, single = _run(B, ctx, gid, pats, motifs=[104, 106, 202, 2])
        _check(g, pats, counts, sums, single)


@pytest.mark.parametrize("shape", [256, 32])  # CTA walks, warp walks
def test_batch_induced_plans(B, shape):
    # the literal reading of Sec. 3.1 (induced = 1): every step also rejects rows whose new
    # vertices are adjacent to columns their pattern vertices are not adjacent to
    cases = [(I.grid(7, 7), [I.path(k) for k in (3, 4, 6, 9)] + [I.cycle(4), I.cycle(8), I.star(3),
                                                              I.grid(2, 3), I.random_tree(8, 2)]),
             (I.heavy_hex(6, 5), [I.path(k) for k in (5, 12, 18)] + [I.sub_patch(I.heavy_hex(6, 5), 14, 1)])]
    with B.Context(0) as ctx:
        B.dm_set_tuning(ctx.h, False, 0.5)
        B.dm_set_batch_shape(ctx.h, shape, 0)
        for g, pats in cases:
            gid = ctx.load(g)
            plans = [B.dm_plan(ctx.h, gid, p.n, p.row_ptr, p.col_idx, induced=True) for p in pats]
            counts, sums = B.dm_match_batch(ctx.h, plans, B.DM_COUNT)
            assert B.dm_batch_config(ctx.h)["threads_per_cta"] == shape
            for p, pl, c, s_ in zip(pats, plans, counts.tolist(), sums.tolist()):
                ref = oracle.enumerate(g, p, induced=True, rows=False, threads=8)
                assert (c, s_) == (ref.count, ref.checksum), (p.name, shape)
                assert B.dm_match(ctx.h, pl, B.DM_COUNT) == (c, s_)
            for pl in plans:
                B.dm_plan_free(pl)


def test_batch_rejects_mixed_graphs_and_modes(B):
    with B.Context(0) as ctx:
        a = ctx.load(I.grid(3, 3))
        b = ctx.load(I.grid(4, 4))
        p = I.path(3)
        pa = B.dm_plan(ctx.h, a, p.n, p.row_ptr, p.col_idx)
        pb = B.dm_plan(ctx.h, b, p.n, p.row_ptr, p.col_idx)
        with pytest.raises(B.DMError):
            B.dm_match_batch(ctx.h, [pa, pb], B.DM_COUNT)
        with pytest.raises(B.DMError):
            B.dm_match_batch(ctx.h, [pa], B.DM_ALL)
        B.dm_plan_free(pa)
        B.dm_plan_free(pb)
