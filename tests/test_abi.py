"""CPU tests of the C ABI: the library loads, exports every symbol include/dm.h declares,
and the host-only planner follows the decomposition rules of Sec. 3.2. No GPU calls."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2508_21287_gb300 import build
    build.build()
    from paper_2508_21287_gb300 import binding
    return binding


def _declared():
    src = open(os.path.join(ROOT, "include", "dm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dm_[a-z_]+)\s*\(", src)) - {"dm_chunk_cb"})


def test_library_exports_every_declared_symbol(B):
    nm = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dm_\w+)", nm))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    # the binding wraps each of them under the same name
    assert set(declared) <= set(B.exported_symbols())
    for d in declared:
        assert hasattr(B, d)


def test_strerror(B):
    assert B.dm_strerror(0) == "ok"
    assert "connected" in B.dm_strerror(B.DM_E_DISCONNECTED)


def test_six_cycle_example(B):
    # Sec. 3.2: a 6-cycle decomposed with M4 gives two path slices sharing their two end
    # vertices, i.e. join constraints that pair the ends of S_0 with the ends of S_1.
    from paper_2508_21287_gb300 import inputs as I
    c6 = I.cycle(6)
    d = B.dm_decompose(6, c6.row_ptr, c6.col_idx, [4])
    assert [s["motif"] for s in d] == [4, 4]
    s0, s1 = d[0]["slice"], d[1]["slice"]
    shared = set(s0) & set(s1)
    assert len(shared) == 2 and d[1]["n_keys"] == 2
    assert {s0[0], s0[3]} == shared and {s1[0], s1[3]} == shared
    assert set(s0) | set(s1) == set(range(6))


@pytest.mark.parametrize("n", [16, 31, 40, 46])
def test_long_cycle_as_two_half_paths(B, n):
    # the 6-cycle example scaled up: with paths of about half the cycle in the motif set the
    # cycle is one path slice joined with a second path on both end vertices
    from paper_2508_21287_gb300 import inputs as I
    c = I.cycle(n)
    a, b = n // 2 + 1, (n + 1) // 2 + 1
    d = B.dm_decompose(n, c.row_ptr, c.col_idx, sorted({a, b}, reverse=True) + [4])
    assert [s["motif"] for s in d] == [b, a]
    assert d[1]["n_keys"] == 2 and not d[0]["backedges"] and not d[1]["backedges"]
    assert set(d[0]["slice"]) | set(d[1]["slice"]) == set(range(n))


@pytest.mark.parametrize("seed", range(8))
def test_m2_only_iterations_equal_edge_count(B, seed):
    # Sec. 4.2: with M2 alone the number of join-and-filter iterations equals |E_p|; here a
    # covering M2 slice or a back-edge check per pattern edge.
    from paper_2508_21287_gb300 import inputs as I
    for p in (I.random_tree(6 + seed, seed), I.cycle_with_chords(8 + seed, seed), I.subdivided_grid(2, 2 + seed % 3)):
        d = B.dm_decompose(p.n, p.row_ptr, p.col_idx, [2])
        assert all(s["motif"] == 2 for s in d)
        assert len(d) + sum(len(s["backedges"]) for s in d) == p.n_edges
        assert len(d) == p.n - 1


@pytest.mark.parametrize("motifs", [[4], [3], [104, 106], [201], [112, 4], [202], [203, 4]])
def test_decomposition_covers_every_edge_once(B, motifs):
    from paper_2508_21287_gb300 import inputs as I
    pats = [I.heavy_hex(1, 2), I.grid(3, 4), I.random_tree(15, 1), I.cycle(12), I.subdivided_grid(2, 3)]
    for p in pats:
        d = B.dm_decompose(p.n, p.row_ptr, p.col_idx, motifs)
        covered = []
        mapped = set()
        for i, s in enumerate(d):
            from paper_2508_21287_gb300.binding import _lib  # noqa: F401
            sl = s["slice"]
            if i > 0:
                assert set(sl) & mapped, "a later slice must overlap the mapped set"
                assert s["n_keys"] == len(set(sl) & mapped)
            mapped |= set(sl)
            covered += [tuple(sorted(e)) for e in s["backedges"]]
        # each slice edge + back-edge covers a pattern edge; count them through the motif shapes
        assert mapped == set(range(p.n))
        edges = set(p.edges())
        assert set(covered) <= edges


def test_decompose_rejects_bad_input(B):
    from paper_2508_21287_gb300 import inputs as I
    two = I.from_edges(4, [(0, 1), (2, 3)])
    with pytest.raises(B.DMError) as e:
        B.dm_decompose(4, two.row_ptr, two.col_idx, [2])
    assert e.value.code == B.DM_E_DISCONNECTED
    with pytest.raises(B.DMError):
        B.dm_decompose(3, [0, 1, 2, 2], [1, 0], [2])  # asymmetric? 0-1 only; vertex 2 isolated -> disconnected
    with pytest.raises(B.DMError) as e:
        B.dm_decompose(2, [0, 1, 1], [1], [2])  # edge 0->1 without 1->0
    assert e.value.code == B.DM_E_INVAL
    with pytest.raises(B.DMError) as e:
        p = I.path(3)
        B.dm_decompose(3, p.row_ptr, p.col_idx, [999])
    assert e.value.code == B.DM_E_NOTFOUND


def test_plan_batch_checks_arguments_without_a_device(B):
    from paper_2508_21287_gb300 import inputs as I
    p = I.path(3)
    with pytest.raises(B.DMError) as e:
        B.dm_plan_batch(None, 0, [(p.n, p.row_ptr, p.col_idx)])
    assert e.value.code == B.DM_E_INVAL


def test_query_runner_checks_arguments_without_a_device(B):
    import ctypes
    from paper_2508_21287_gb300 import inputs as I
    p = I.path(3)
    fake = ctypes.c_void_p(0x1000)
    with pytest.raises(B.DMError) as e:  # one context given twice: refused before any use
        B.dm_match_topk_queries([fake, fake], [0, 0], [(p.n, p.row_ptr, p.col_idx)], 5)
    assert e.value.code == B.DM_E_INVAL
    with pytest.raises(B.DMError) as e:
        B.dm_match_topk_queries([], [], [(p.n, p.row_ptr, p.col_idx)], 5)
    assert e.value.code == B.DM_E_INVAL


def _motif_edges(motif: int):
    # position pairs of the path and cycle motifs (M_k: k positions in a row; M_{k-O}: closed)
    if motif < 100:
        return [(i, i + 1) for i in range(motif - 1)]
    k = motif - 100
    return [(i, (i + 1) % k) for i in range(k)]


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("motifs", [[2], [3], [4], [4, 2], [104, 2], [104, 106, 2], [112, 4, 2], [8, 4, 2]])
def test_slices_and_back_edges_enforce_exactly_the_pattern_edges(B, motifs, order):
    # Every slice places its motif on pattern edges (so a join never asks for an edge the
    # pattern lacks), and the slices' motif edges together with the back-edges are exactly the
    # pattern's edges (so no pattern edge goes unchecked): the conditions under which Alg. 1
    # returns exactly Emb(G_p, G_d).
    from paper_2508_21287_gb300 import inputs as I
    g = I.heavy_hex(3, 4)
    grid = I.grid(6, 6)
    pats = [I.random_tree(12 + s, s) for s in range(3)] + [I.cycle_with_chords(10 + s, s) for s in range(3)]
    pats += [I.sub_patch(g, 14 + 4 * s, s) for s in range(3)] + [I.sub_patch(grid, 9 + 3 * s, s) for s in range(3)]
    pats += [I.cycle(12), I.cycle(18), I.path(9)]
    for p in pats:
        try:
            d = B.dm_decompose(p.n, p.row_ptr, p.col_idx, motifs, order=order)
        except B.DMError:
            continue  # a motif set that cannot start this pattern (no slice fits) is refused
        edges = set(p.edges())
        enforced = []
        for s in d:
            sl = s["slice"]
            for a, b in _motif_edges(s["motif"]):
                e = tuple(sorted((sl[a], sl[b])))
                assert e in edges, (p.n, motifs, s)
                enforced.append(e)
            enforced += [tuple(sorted(e)) for e in s["backedges"]]
        assert set(enforced) == edges, (p.n, motifs, order)


def _motif_pattern(motif: int):
    from paper_2508_21287_gb300 import inputs as I
    return I.path(motif) if motif < 100 else I.cycle(motif - 100)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("motifs", [[2], [4, 2], [104, 2], [104, 106, 2], [8, 4, 2]])
def test_plan_executed_on_the_host_gives_the_oracle_set(B, motifs, order):
    # The plan's slices run through Alg. 1 in plain Python (motif tables from the oracle, joins on
    # the shared pattern vertices, distinct images, back-edge tests) give exactly the oracle's
    # embedding set: the decomposition is sound and complete, independent of the kernels.
    import numpy as np
    import oracle
    from paper_2508_21287_gb300 import inputs as I
    cases = [(I.grid(5, 5), I.grid(2, 3)), (I.grid(5, 5), I.cycle(6)), (I.grid(5, 5), I.sub_patch(I.grid(6, 6), 8, 2)),
             (I.heavy_hex(2, 3), I.path(7)), (I.heavy_hex(2, 3), I.cycle(12)), (I.grid(4, 5), I.random_tree(8, 3))]
    for data, p in cases:
        d = B.dm_decompose(p.n, p.row_ptr, p.col_idx, motifs, order=order)
        adj = set(data.edges()) | {(b, a) for a, b in data.edges()}
        tables = {}
        R = None  # list of dicts pattern vertex -> data vertex
        for s in d:
            m = s["motif"]
            if m not in tables:
                tables[m] = oracle.enumerate(data, _motif_pattern(m)).rows
            sl = s["slice"]
            out = []
            for t in tables[m]:
                cand = dict(zip(sl, (int(x) for x in t)))
                for row in (R if R is not None else [{}]):
                    if any(row[v] != cand[v] for v in cand if v in row):
                        continue  # join keys disagree
                    new = [cand[v] for v in cand if v not in row]
                    if len(set(new)) != len(new) or set(new) & set(row.values()):
                        continue  # images must stay distinct
                    merged = {**row, **cand}
                    if all((merged[a], merged[b]) in adj for a, b in s["backedges"]):
                        out.append(merged)
            R = out
        got = sorted(tuple(r[v] for v in range(p.n)) for r in R)
        ref = oracle.enumerate(data, p)
        assert got == [tuple(x) for x in np.asarray(ref.rows).tolist()], (p.n, motifs)


@pytest.mark.parametrize("n", [63, 64, 65, 100, 128])
def test_wide_patterns_enforce_exactly_their_edges(B, n):
    # patterns across the 64-vertex word boundary of the planner's vertex sets, up to the
    # 128-vertex limit: the slice and back-edge conditions hold, the plan is deterministic,
    # and one vertex more is refused
    from paper_2508_21287_gb300 import inputs as I
    g = I.heavy_hex(6, 6)
    for p in (I.sub_patch(g, n, 5), I.random_tree(n, n)):
        for order in (0, 1):
            d = B.dm_decompose(p.n, p.row_ptr, p.col_idx, [4, 2], order=order)
            assert d == B.dm_decompose(p.n, p.row_ptr, p.col_idx, [4, 2], order=order)
            edges = set(p.edges())
            enforced, mapped = [], set()
            for s in d:
                sl = s["slice"]
                assert len(set(sl)) == len(sl)
                for a, b in _motif_edges(s["motif"]):
                    e = tuple(sorted((sl[a], sl[b])))
                    assert e in edges
                    enforced.append(e)
                enforced += [tuple(sorted(e)) for e in s["backedges"]]
                mapped |= set(sl)
            assert set(enforced) == edges and mapped == set(range(p.n))
    t = I.random_tree(129, 1)
    with pytest.raises(B.DMError) as e:
        B.dm_decompose(t.n, t.row_ptr, t.col_idx, [4, 2])
    assert e.value.code == B.DM_E_INVAL


def test_query_batch_marshals_once(B):
    import ctypes
    from paper_2508_21287_gb300 import inputs as I
    qs = [I.path(4), I.cycle(6), I.star(3)]
    qb = B.QueryBatch([(q.n, q.row_ptr, q.col_idx) for q in qs], 7)
    assert qb.n == 3 and qb.k == 7 and list(qb.n_p) == [4, 6, 4]
    assert [r.shape for r in qb.rows] == [(7, 4), (7, 6), (7, 4)] and all(x.shape == (7,) for x in qb.scores)
    for i, q in enumerate(qs):  # the pointer arrays point at the marshalled CSR of each query
        assert qb.rps[i][q.n] == q.row_ptr[-1] and qb.cis[i][0] == q.col_idx[0]
    with pytest.raises(ValueError):  # a batch is made for one k
        B.dm_match_topk_queries([ctypes.c_void_p(0x1000)], [0], qb, 5)
