"""Layout-query server: answers equal the oracle's and results alone; overlap; admission.

Requests are submitted faster than they complete, so several are in flight on different
slots (streams) at once and later ones are admitted as slots and pool memory free up. Every
answer must be exactly the dm_score_topk answer for the same pattern on a lone context (the
per-row FP32 score does not depend on scheduling, and ties break on the row), and the top-k
of the FP64 oracle (Sec. 5.4 scores) within 1e-5 relative, with the tie band of check_topk."""
import numpy as np
import pytest

import oracle
from paper_2508_21287_gb300 import inputs as I

RTOL = 1e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


def _graphs():
    return [I.lognormal_weights(I.heavy_hex(4, 6), seed=1, qubits=True),
            I.lognormal_weights(I.grid(8, 8), seed=2),
            I.lognormal_weights(I.random_regular3(128, 3), seed=3)]


def test_results_in_the_mix_equal_results_alone(B):
    graphs = _graphs()
    reqs = []
    for s in range(48):
        gi = s % 3
        g = graphs[gi]
        p = I.mixed_pattern(s, 5, 9) if s % 2 else I.sub_patch(g, 5 + s % 6, s)
        reqs.append((gi, p))
    srv = B.dm_server_create(0, n_slots=4, mem_budget_bytes=8 << 30)
    try:
        gids = [B.dm_server_load_graph(srv, g.n, g.row_ptr, g.col_idx, g.edge_err, g.qubit_err) for g in graphs]
        ids = [B.dm_server_submit(srv, gids[gi], p.n, p.row_ptr, p.col_idx, 10) for gi, p in reqs]
        answers = [B.dm_server_wait(srv, rid, 10, p.n) for rid, (gi, p) in zip(ids, reqs)]
        st = B.dm_server_stats_get(srv)
    finally:
        B.dm_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["rejected"] == 0 and st["failed"] == 0
    with B.Context(0) as ctx:
        lone = [ctx.load(g) for g in graphs]
        for (gi, p), a in zip(reqs, answers):
            assert a["status"] == 0
            rows, scores = ctx.plan(lone[gi], p).topk(10)
            assert np.array_equal(a["rows"], rows)
            assert np.array_equal(a["scores"], scores)
            assert a["latency_ms"] >= a["queue_ms"] >= 0


def test_work_cap_rejects_and_others_complete(B):
    g = I.lognormal_weights(I.grid(16, 16), seed=5)
    big = I.path(40)            # astronomically many embeddings on a grid
    small = I.path(4)
    srv = B.dm_server_create(0, n_slots=2, mem_budget_bytes=4 << 30, max_rows=200000)
    try:
        gid = B.dm_server_load_graph(srv, g.n, g.row_ptr, g.col_idx, g.edge_err)
        r_big = B.dm_server_submit(srv, gid, big.n, big.row_ptr, big.col_idx, 10)
        r_small = B.dm_server_submit(srv, gid, small.n, small.row_ptr, small.col_idx, 10)
        a_big = B.dm_server_wait(srv, r_big, 10, big.n)
        a_small = B.dm_server_wait(srv, r_small, 10, small.n)
        st = B.dm_server_stats_get(srv)
    finally:
        B.dm_server_destroy(srv)
    assert a_big["status"] == B.DM_E_CAPACITY
    assert a_small["status"] == 0 and len(a_small["rows"]) == 10
    assert st["rejected"] == 1 and st["completed"] == 1


def _check_oracle_topk(g, p, rows, scores, k):
    allrows = oracle.enumerate(g, p).rows
    m = min(k, len(allrows))
    assert rows.shape == (m, p.n)
    if m == 0:
        return
    s = oracle.scores(g, p, allrows)
    order = oracle.topk(allrows, s, k)
    np.testing.assert_allclose(scores, s[order], rtol=RTOL, atol=0)
    pos = {tuple(r): i for i, r in enumerate(allrows.tolist())}
    idx = [pos.get(tuple(r)) for r in rows.tolist()]
    assert None not in idx and len(set(idx)) == m
    np.testing.assert_allclose(s[idx], scores, rtol=RTOL, atol=0)
    kth = s[order[-1]]
    assert set(np.nonzero(s < kth * (1 - RTOL))[0].tolist()) <= set(idx)


def test_serving_answers_equal_the_oracle_and_overlap_on_the_device(B):
    # the serving configuration's three device-resident graphs (heavy-hex 4x6, grid 32x32,
    # random 3-regular V=2048) with patterns small enough for the oracle; all requests are
    # submitted at once, so slots run concurrently and later requests wait for admission
    graphs = [I.lognormal_weights(I.heavy_hex(4, 6), seed=11, qubits=True),
              I.lognormal_weights(I.grid(32, 32), seed=12),
              I.lognormal_weights(I.random_regular3(2048, 13), seed=13)]
    reqs = []
    for s in range(36):
        gi = s % 3
        g = graphs[gi]
        p = I.mixed_pattern(40000 + s, 5, 8) if s % 2 else I.sub_patch(g, 5 + s % 5, s)
        reqs.append((gi, p))
    srv = B.dm_server_create(0, n_slots=6, mem_budget_bytes=32 << 30)  # no work cap: all must finish
    try:
        gids = [B.dm_server_load_graph(srv, g.n, g.row_ptr, g.col_idx, g.edge_err, g.qubit_err) for g in graphs]
        ids = [B.dm_server_submit(srv, gids[gi], p.n, p.row_ptr, p.col_idx, 10) for gi, p in reqs]
        answers = [B.dm_server_wait(srv, rid, 10, p.n) for rid, (gi, p) in zip(ids, reqs)]
        st = B.dm_server_stats_get(srv)
    finally:
        B.dm_server_destroy(srv)
    assert [a["status"] for a in answers] == [0] * len(reqs)
    assert st["completed"] == len(reqs) and st["rejected"] == 0 and st["failed"] == 0
    # requests really ran at the same time: on the host and on the GPU timeline
    assert st["max_running"] > 1
    assert st["overlapped"] > 0
    for (gi, p), a in zip(reqs, answers):
        assert a["status"] == 0
        _check_oracle_topk(graphs[gi], p, a["rows"], a["scores"], 10)
