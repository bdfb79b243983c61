"""Direction-aware layout scores (Sec. 5.4, its footnote on directed two-qubit gates) through
the C ABI, against the FP64 oracle.

The embedding set is the undirected one; every embedding is re-scored with per-direction
device costs times per-direction gate counts. FP32 sums of non-negative terms are compared with
the FP64 oracle within 1e-5 relative: the patterns here have at most 30 vertices and ~36
edges, so a row's score has at most ~100 terms (72 weighted slots and 30 vertex errors), and a
recursive FP32 sum of n non-negative terms (each rounded once) is within about n * 2^-24
~ 6e-6 of the exact value; the top-k rows follow the tie rule of the undirected top-k tests.
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


def _check(allrows, s, rows, scores, k, n):
    m = min(k, len(allrows))
    assert rows.shape == (m, n)
    if m == 0:
        return
    order = oracle.topk(allrows, s, k)
    np.testing.assert_allclose(scores, s[order], rtol=RTOL, atol=0)
    pos = {tuple(r): i for i, r in enumerate(allrows.tolist())}
    idx = [pos.get(tuple(r)) for r in rows.tolist()]
    assert None not in idx and len(set(idx)) == m
    np.testing.assert_allclose(s[idx], scores, rtol=RTOL, atol=0)
    kth = s[order[-1]]
    assert set(np.nonzero(s < kth * (1 - RTOL))[0].tolist()) <= set(idx)


@pytest.mark.parametrize("chunk_rows", [0, 300])
def test_directed_topk_matches_oracle(ctx, B, chunk_rows):
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=31, qubits=True)
    e_dir = I.directed_errors(g, seed=32)
    gid = ctx.load(g)
    B.dm_load_directed_errors(ctx.h, gid, e_dir)
    pats = [I.layout_query(g, s) for s in range(4)] + [I.path(12), I.sub_patch(g, 20, 7)]
    for i, p in enumerate(pats):
        w = I.gate_directions(p, 100 + i)
        allrows = oracle.enumerate(g, p).rows
        s = oracle.scores_directed(g, e_dir, p, w, allrows)
        plan = ctx.plan(gid, p, chunk_rows=chunk_rows)
        for k in (1, 10, 100):
            rows, scores = B.dm_score_topk_directed(ctx.h, plan.h, w, k, p.n)
            _check(allrows, s, rows, scores, k, p.n)


def test_directed_with_symmetric_costs_equals_undirected_topk(ctx, B):
    # symmetric costs and one gate per pattern edge (lower to higher vertex): the direction-aware
    # ranking is the undirected one of dm_score_topk
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=33, qubits=True)
    gid = ctx.load(g)
    B.dm_load_directed_errors(ctx.h, gid, g.edge_err)
    for s_ in range(3):
        p = I.sub_patch(g, 14 + 3 * s_, s_)
        w = np.array([1.0 if a < int(p.col_idx[k]) else 0.0 for a in range(p.n)
                      for k in range(p.row_ptr[a], p.row_ptr[a + 1])], dtype=np.float32)
        plan = ctx.plan(gid, p)
        rows_d, sc_d = B.dm_score_topk_directed(ctx.h, plan.h, w, 50, p.n)
        rows_u, sc_u = plan.topk(50)
        np.testing.assert_allclose(sc_d, sc_u, rtol=RTOL, atol=0)
        allrows = oracle.enumerate(g, p).rows
        _check(allrows, oracle.scores(g, p, allrows), rows_d, sc_d, 50, p.n)


def test_directed_argument_checks(ctx, B):
    g = I.lognormal_weights(I.heavy_hex(2, 3), seed=34)
    gid = ctx.load(g)
    p = I.path(5)
    plan = ctx.plan(gid, p)
    w = np.ones(len(p.col_idx), dtype=np.float32)
    with pytest.raises(B.DMError) as e:  # no directed costs loaded for this graph
        B.dm_score_topk_directed(ctx.h, plan.h, w, 5, p.n)
    assert e.value.code == B.DM_E_INVAL
    bad = I.directed_errors(g, 1)
    bad[2] = np.nan
    with pytest.raises(B.DMError) as e:
        B.dm_load_directed_errors(ctx.h, gid, bad)
    assert e.value.code == B.DM_E_INVAL
    B.dm_load_directed_errors(ctx.h, gid, I.directed_errors(g, 1))
    w[0] = np.inf
    with pytest.raises(B.DMError) as e:
        B.dm_score_topk_directed(ctx.h, plan.h, w, 5, p.n)
    assert e.value.code == B.DM_E_INVAL
