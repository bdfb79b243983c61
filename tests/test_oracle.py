"""Pins for the CPU oracle: things the problem statement and mathematics fix, independent of
the oracle's own code (brute force, closed forms, invariants, a published hash vector).

Problem statement: Sec. 3.1 (injective maps preserving adjacency; non-induced reading, see
the module docstring of ``oracle``). Layout score: Sec. 5.4.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2508_21287_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _graph(name):
    if name.startswith("grid"):
        r, c = name[4:].split("x")
        return I.grid(int(r), int(c))
    if name.startswith("heavyhex"):
        m, n = name[8:].split("x")
        return I.heavy_hex(int(m), int(n))
    if name.startswith("path"):
        return I.path(int(name[4:]))
    if name.startswith("cycle"):
        return I.cycle(int(name[5:]))
    if name.startswith("star"):
        return I.star(int(name[4:]))
    if name.startswith("K"):
        return I.complete(int(name[1:]))
    raise KeyError(name)


def _closed_forms():
    out = []
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = [p.strip() for p in line.split("|")]
            d, p, cnt, deriv = parts[0], parts[1], int(parts[2]), parts[3]
            induced = deriv.rstrip().endswith("; induced")
            out.append((d, p, cnt, induced))
    return out


@pytest.mark.parametrize("d,p,count,induced", _closed_forms())
def test_closed_form_counts(d, p, count, induced):
    r = oracle.enumerate(_graph(d), _graph(p), induced=induced)
    assert r.count == count


def test_grid_degree_closed_forms_any_size():
    # P3 = sum d(d-1), claw = sum d(d-1)(d-2), P4 (triangle-free) = sum over edges of
    # 2 (d(u)-1)(d(v)-1), C4 = 8 (r-1)(c-1), computed here from the degree sequence.
    for r, c in [(2, 3), (3, 5), (4, 4), (5, 7)]:
        g = I.grid(r, c)
        d = g.degree()
        assert oracle.enumerate(g, I.path(3), rows=False).count == int((d * (d - 1)).sum())
        assert oracle.enumerate(g, I.star(3), rows=False).count == int((d * (d - 1) * (d - 2)).sum())
        p4 = sum(2 * (d[u] - 1) * (d[v] - 1) for u, v in g.edges())
        assert oracle.enumerate(g, I.path(4), rows=False).count == p4
        assert oracle.enumerate(g, I.cycle(4), rows=False).count == 8 * (r - 1) * (c - 1)


def test_heavy_hex_cycle12_per_cell():
    for m, n in [(1, 1), (2, 3), (3, 5)]:
        g = I.heavy_hex(m, n)
        assert g.n == 5 * m * n + 4 * m + 4 * n - 1
        assert oracle.enumerate(g, I.cycle(12), rows=False).count == 24 * m * n


def _random_graph(n, p, seed):
    rng = I.SplitMix64(seed)
    edges = [(u, v) for u in range(n) for v in range(u + 1, n) if rng.below(1000) < p * 1000]
    return I.from_edges(n, edges)


def _random_connected_pattern(n, seed):
    rng = I.SplitMix64(seed + 77)
    edges = [(rng.below(i), i) for i in range(1, n)]
    for _ in range(rng.below(3)):
        a, b = rng.below(n), rng.below(n)
        if a != b:
            edges.append((a, b))
    return I.from_edges(n, edges)


@pytest.mark.parametrize("seed", range(12))
def test_backtracking_equals_brute_force(seed):
    d = _random_graph(5 + seed % 5, 0.45, seed)
    p = _random_connected_pattern(2 + seed % 4, seed)
    for induced in (False, True):
        a = oracle.enumerate(d, p, induced=induced)
        b = oracle.brute_force(d, p, induced=induced)
        assert a.count == b.count
        assert np.array_equal(a.rows, b.rows)
        assert a.checksum == b.checksum


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_equals_pure_python(seed):
    d = _random_graph(4 + seed % 3, 0.5, 100 + seed)
    p = _random_connected_pattern(2 + seed % 3, 100 + seed)
    for induced in (False, True):
        a = oracle.brute_force(d, p, induced=induced)
        b = oracle.brute_force_py(d, p, induced=induced)
        assert [tuple(r) for r in a.rows] == b


def test_grid6x6_path5_brute_force():
    g = I.grid(6, 6)
    a = oracle.enumerate(g, I.path(5))
    b = oracle.brute_force(g, I.path(5))
    assert a.count == b.count == 1712
    assert np.array_equal(a.rows, b.rows)


def test_rows_valid_sorted_distinct():
    g = I.heavy_hex(2, 2)
    p = I.path(9)
    r = oracle.enumerate(g, p)
    rows = r.rows
    edges = {(u, int(v)) for u in range(g.n) for v in g.neighbours(u)}
    for row in rows:
        assert len(set(row.tolist())) == p.n
        for u, v in p.edges():
            assert (int(row[u]), int(row[v])) in edges
    keys = [tuple(x) for x in rows.tolist()]
    assert keys == sorted(set(keys))


@pytest.mark.parametrize("pattern", [I.path(6), I.cycle(12), I.star(3), I.random_tree(9, 3)])
def test_automorphism_invariants(pattern):
    g = I.heavy_hex(3, 3)
    aut = oracle.automorphisms(pattern)
    r = oracle.enumerate(g, pattern)
    assert r.count % aut == 0
    assert oracle.images(r.rows).shape[0] * aut == r.count


def test_automorphism_counts_known():
    assert oracle.automorphisms(I.cycle(7)) == 14
    assert oracle.automorphisms(I.path(5)) == 2
    assert oracle.automorphisms(I.star(3)) == 6
    assert oracle.automorphisms(I.complete(4)) == 24


def test_relabelling_maps_the_set():
    g = I.heavy_hex(2, 2)
    rng = I.SplitMix64(5)
    perm = list(range(g.n))
    rng.shuffle(perm)
    h = I.relabel(g, perm)
    p = I.random_tree(7, 11)
    a = oracle.enumerate(g, p).rows
    b = oracle.enumerate(h, p).rows
    mapped = np.asarray(perm, dtype=np.int32)[a]
    mapped = mapped[np.lexsort(mapped.T[::-1])]
    assert np.array_equal(mapped, b)


def test_thread_split_matches_single():
    g = I.heavy_hex(4, 6)
    p = I.path(14)
    a = oracle.enumerate(g, p, threads=1)
    b = oracle.enumerate(g, p, threads=5)
    assert np.array_equal(a.rows, b.rows) and a.checksum == b.checksum


def test_mix64_published_vector():
    want = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(x, 16) for x in f if x.startswith("0x")]
    state = 0
    got = []
    for _ in range(3):
        state = (state + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        got.append(oracle.mix64(state))
    assert got == want
    # the input generators' SplitMix64 must agree with the same vector
    rng = I.SplitMix64(0)
    assert [rng.next_u64() for _ in range(3)] == want
    assert [int(x) for x in I.splitmix64_block(0, 3)] == want


def test_checksum_order_independent_and_matches_enumerator():
    g = I.grid(5, 5)
    r = oracle.enumerate(g, I.path(4))
    rows = r.rows.copy()
    assert oracle.checksum(rows) == r.checksum
    rng = np.random.default_rng(0)
    rng.shuffle(rows)
    assert oracle.checksum(rows) == r.checksum
    assert oracle.checksum(rows[:0]) == 0
    # the hash sees the row width and every position
    assert oracle.row_hash([1, 2]) != oracle.row_hash([2, 1])
    assert oracle.row_hash([1, 2]) != oracle.row_hash([1, 2, 0])


def test_row_hash_binds_every_position():
    # a changed value at any single position, or two swapped positions, changes H(row)
    row = [int(x) for x in np.random.default_rng(3).permutation(1000)[:12]]
    h = oracle.row_hash(row)
    for j in range(len(row)):
        r2 = list(row)
        r2[j] += 1
        assert oracle.row_hash(r2) != h
        for k in range(j + 1, len(row)):
            r3 = list(row)
            r3[j], r3[k] = r3[k], r3[j]
            assert oracle.row_hash(r3) != h
    # the sum over rows is taken mod 2^64: duplicated rows add up, nothing saturates
    rows = np.array([row, row], dtype=np.int32)
    assert oracle.checksum(rows) == (2 * h) % (1 << 64)


def test_fidelity_scores_are_the_log_of_the_product():
    # form 1: exp(-score) is the product of the fidelities 1 - e over the mapped pattern edges
    # and vertices, computed here as a plain product
    g = I.lognormal_weights(I.heavy_hex(2, 3), seed=4, qubits=True)
    p = I.path(6)
    rows = oracle.enumerate(g, p).rows
    s = oracle.scores(g, p, rows, form=1)
    w = {(int(u), int(g.col_idx[k])): float(g.edge_err[k]) for u in range(g.n)
         for k in range(g.row_ptr[u], g.row_ptr[u + 1])}
    for r, sr in zip(rows[:200], s[:200]):
        prod = 1.0
        for a, b in zip(r[:-1], r[1:]):
            prod *= 1.0 - w[(int(a), int(b))]
        for v in r:
            prod *= 1.0 - float(g.qubit_err[v])
        assert np.isclose(np.exp(-sr), prod, rtol=1e-12, atol=0)
    # constant error eps on every edge: m * -log(1 - eps); small errors: close to the sum form
    h = I.grid(4, 4)
    h.edge_err = np.full(len(h.col_idx), 0.01, dtype=np.float32)
    r4 = oracle.enumerate(h, I.cycle(4)).rows
    e32 = float(np.float32(0.01))
    assert np.allclose(oracle.scores(h, I.cycle(4), r4, form=1), -4 * np.log1p(-e32), rtol=1e-14, atol=0)
    s0 = oracle.scores(g, p, rows, form=0)
    assert np.all(s >= s0) and np.all(s <= s0 * 1.02)


def test_scores_unit_weights_equal_edge_count():
    g = I.heavy_hex(2, 3)
    g.edge_err = np.ones(len(g.col_idx), dtype=np.float32)
    p = I.random_tree(8, 4)
    rows = oracle.enumerate(g, p).rows
    s = oracle.scores(g, p, rows)
    assert np.all(s == p.n_edges)
    g.qubit_err = np.ones(g.n, dtype=np.float32)
    s = oracle.scores(g, p, rows)
    assert np.all(s == p.n_edges + p.n)


def test_scores_linear_weights_closed_form():
    # w(a, b) = a + b and w_q(a) = 3a give score(f) = sum_u (deg_p(u) + 3) f(u).
    g = I.grid(4, 5)
    ee = np.empty(len(g.col_idx), dtype=np.float32)
    for u in range(g.n):
        for k in range(g.row_ptr[u], g.row_ptr[u + 1]):
            ee[k] = u + int(g.col_idx[k])
    g.edge_err = ee
    g.qubit_err = 3.0 * np.arange(g.n, dtype=np.float32)
    p = I.cycle_with_chords(6, 1, n_chords=0)
    p2 = I.random_tree(6, 2)
    for pat in (p, p2):
        rows = oracle.enumerate(g, pat).rows
        s = oracle.scores(g, pat, rows)
        deg = pat.degree()
        want = rows.astype(np.float64) @ (deg + 3).astype(np.float64)
        assert np.array_equal(s, want)


def _slot_weights(g, fn):
    """A col_idx-aligned array with fn(u, v) at the slot of u -> v."""
    out = np.empty(len(g.col_idx), dtype=np.float32)
    for u in range(g.n):
        for k in range(g.row_ptr[u], g.row_ptr[u + 1]):
            out[k] = fn(u, int(g.col_idx[k]))
    return out


def _transposed(g, a):
    """The slot array whose u -> v entry is a's v -> u entry."""
    pos = {(u, int(g.col_idx[k])): k for u in range(g.n) for k in range(g.row_ptr[u], g.row_ptr[u + 1])}
    return np.array([a[pos[(int(g.col_idx[k]), u)]] for u in range(g.n)
                     for k in range(g.row_ptr[u], g.row_ptr[u + 1])], dtype=np.float32)


def test_directed_scores_reduce_to_undirected():
    # symmetric device costs and one gate per pattern edge, run from the lower to the higher
    # pattern vertex: the direction-aware score is the undirected score of Sec. 5.4
    g = I.lognormal_weights(I.heavy_hex(2, 3), seed=4, qubits=True)
    for p in (I.path(7), I.sub_patch(g, 9, 2), I.cycle(12)):
        rows = oracle.enumerate(g, p).rows
        w = _slot_weights(p, lambda a, b: 1.0 if a < b else 0.0)
        np.testing.assert_array_equal(oracle.scores_directed(g, g.edge_err, p, w, rows), oracle.scores(g, p, rows))


def test_directed_scores_closed_form():
    # cost(u -> v) = u + 2v on the device and one gate i -> i+1 along a path pattern:
    # score(f) = f(0) + 3 (f(1) + ... + f(n-2)) + 2 f(n-1); with the gates reversed the end
    # coefficients swap
    g = I.grid(4, 5)
    e = _slot_weights(g, lambda u, v: u + 2.0 * v)
    p = I.path(6)
    rows = oracle.enumerate(g, p).rows.astype(np.float64)
    fwd = _slot_weights(p, lambda a, b: 1.0 if b == a + 1 else 0.0)
    want = rows[:, 0] + 3.0 * rows[:, 1:-1].sum(axis=1) + 2.0 * rows[:, -1]
    np.testing.assert_array_equal(oracle.scores_directed(g, e, p, fwd, rows), want)
    bwd = _slot_weights(p, lambda a, b: 1.0 if a == b + 1 else 0.0)
    want = 2.0 * rows[:, 0] + 3.0 * rows[:, 1:-1].sum(axis=1) + rows[:, -1]
    np.testing.assert_array_equal(oracle.scores_directed(g, e, p, bwd, rows), want)


def test_directed_scores_transpose_and_linearity():
    # turning every gate and every device cost around leaves the score unchanged; the score is
    # linear in the gate counts
    g = I.heavy_hex(2, 3)
    e = I.directed_errors(g, seed=9)
    assert not np.array_equal(e, _transposed(g, e))  # really direction dependent
    for s_, p in enumerate((I.path(8), I.random_tree(9, 3), I.sub_patch(g, 10, 1))):
        rows = oracle.enumerate(g, p).rows
        w1, w2 = I.gate_directions(p, 2 * s_), I.gate_directions(p, 2 * s_ + 1)
        a = oracle.scores_directed(g, e, p, w1, rows)
        b = oracle.scores_directed(g, _transposed(g, e), p, _transposed(p, w1), rows)
        np.testing.assert_allclose(a, b, rtol=1e-12)
        c = oracle.scores_directed(g, e, p, w1 + w2, rows)
        np.testing.assert_allclose(c, a + oracle.scores_directed(g, e, p, w2, rows), rtol=1e-12)


def test_topk_matches_full_sort():
    g = I.lognormal_weights(I.heavy_hex(2, 3), seed=3, qubits=True)
    p = I.path(6)
    rows = oracle.enumerate(g, p).rows
    s = oracle.scores(g, p, rows)
    idx = oracle.topk(rows, s, 25)
    order = sorted(range(len(rows)), key=lambda i: (s[i], tuple(rows[i])))
    assert idx.tolist() == order[:25]
    assert oracle.topk(rows, s, 10 ** 6).shape[0] == len(rows)


def test_networkx_monomorphism_counts():
    nx = pytest.importorskip("networkx")
    from networkx.algorithms import isomorphism

    cases = [(I.grid(4, 4), I.path(5)), (I.heavy_hex(2, 2), I.random_tree(6, 1)),
             (I.grid(3, 4), I.cycle(4)), (_random_graph(8, 0.4, 9), _random_connected_pattern(4, 9))]
    for d, p in cases:
        D, P = nx.Graph(), nx.Graph()
        D.add_nodes_from(range(d.n))
        P.add_nodes_from(range(p.n))
        D.add_edges_from(d.edges())
        P.add_edges_from(p.edges())
        gm = isomorphism.GraphMatcher(D, P)
        want = sum(1 for _ in gm.subgraph_monomorphisms_iter())
        assert oracle.enumerate(d, p, rows=False).count == want
        gm = isomorphism.GraphMatcher(D, P)
        want_ind = sum(1 for _ in gm.subgraph_isomorphisms_iter())
        assert oracle.enumerate(d, p, induced=True, rows=False).count == want_ind


def test_disconnected_pattern_rejected():
    p = I.from_edges(4, [(0, 1), (2, 3)])
    with pytest.raises(ValueError):
        oracle.enumerate(I.grid(3, 3), p)


def test_single_vertex_pattern_and_too_large_pattern():
    g = I.grid(3, 3)
    r = oracle.enumerate(g, I.from_edges(1, []))
    assert r.count == 9 and r.rows[:, 0].tolist() == list(range(9))
    assert oracle.enumerate(I.path(3), I.path(5)).count == 0
