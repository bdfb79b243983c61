"""Input generators: sizes, structure and determinism of the synthetic workloads."""
import numpy as np
import pytest

from paper_2508_21287_gb300 import inputs as I


def _check_csr(g):
    assert g.row_ptr[0] == 0 and len(g.row_ptr) == g.n + 1
    assert np.all(np.diff(g.row_ptr) >= 0)
    for u in range(g.n):
        nb = g.neighbours(u)
        assert np.all(np.diff(nb) > 0)          # sorted, no duplicates
        assert u not in nb                       # no self-loop
        for v in nb:
            assert u in g.neighbours(int(v))     # symmetric


@pytest.mark.parametrize("m,n", [(1, 1), (4, 6), (12, 6), (11, 33), (25, 34)])
def test_heavy_hex_sizes(m, n):
    g = I.heavy_hex(m, n)
    assert g.n == 5 * m * n + 4 * m + 4 * n - 1
    assert set(np.unique(g.degree()).tolist()) <= {2, 3}
    assert I.is_connected(g)


def test_heavy_hex_paper_sizes():
    # the paper's heavy-hex data graphs have 1990 and 4485 vertices (Sec. 5.1)
    assert I.heavy_hex(11, 33).n == 1990
    assert I.heavy_hex(25, 34).n == 4485
    assert I.heavy_hex(4, 6).n == 159 and I.heavy_hex(4, 6).n_edges == 182


def test_honeycomb_matches_networkx():
    nx = pytest.importorskip("networkx")
    for m, n in [(1, 1), (2, 3), (3, 2), (4, 6)]:
        h = I.honeycomb(m, n)
        H = nx.Graph()
        H.add_nodes_from(range(h.n))
        H.add_edges_from(h.edges())
        assert nx.is_isomorphic(H, nx.hexagonal_lattice_graph(m, n))


def test_small_graphs_valid():
    for g in [I.grid(6, 6), I.heavy_hex(2, 3), I.random_regular3(64, 1), I.subdivided_grid(3, 4),
              I.random_tree(20, 2), I.cycle_with_chords(15, 3), I.star(3), I.complete(5)]:
        _check_csr(g)


def test_random_regular3():
    g = I.random_regular3(256, 7)
    assert np.all(g.degree() == 3) and I.is_connected(g)
    h = I.random_regular3(256, 7)
    assert np.array_equal(g.col_idx, h.col_idx)


def test_weights_deterministic_and_symmetric():
    g = I.lognormal_weights(I.heavy_hex(4, 6), seed=11, qubits=True)
    h = I.lognormal_weights(I.heavy_hex(4, 6), seed=11, qubits=True)
    assert np.array_equal(g.edge_err, h.edge_err) and np.array_equal(g.qubit_err, h.qubit_err)
    assert g.edge_err.dtype == np.float32 and np.all(g.edge_err > 0)
    for u in range(g.n):
        for k in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col_idx[k])
            kk = g.row_ptr[v] + int(np.searchsorted(g.neighbours(v), u))
            assert g.edge_err[k] == g.edge_err[kk]
    # log-normal(-5, 0.5): the log of the weights has mean ~ -5 and sd ~ 0.5
    big = I.lognormal_weights(I.grid(60, 60), seed=2)
    lw = np.log(big.edge_err.astype(np.float64))
    assert abs(lw.mean() + 5.0) < 0.03 and abs(lw.std() - 0.5) < 0.03


def test_patterns():
    for s in range(30):
        p = I.random_tree(5 + s, s)
        assert p.n_edges == p.n - 1 and I.is_connected(p) and p.degree().max() <= 3
        c = I.cycle_with_chords(10 + s, s)
        assert I.is_connected(c) and c.degree().max() <= 3
        q = I.mixed_pattern(s)
        assert 5 <= q.n <= 40 and I.is_connected(q) and q.degree().max() <= 3
        r = I.c2_pattern(s)
        assert 10 <= r.n <= 30 and I.is_connected(r) and r.degree().max() <= 3


def test_sub_patch_is_an_embedded_induced_subgraph():
    g = I.heavy_hex(4, 6)
    for s in range(5):
        p = I.sub_patch(g, 20, s)
        assert p.n == 20 and I.is_connected(p)
        emb = p.meta["embedding"]
        eset = set(g.edges())
        for u, v in p.edges():
            a, b = emb[u], emb[v]
            assert (min(a, b), max(a, b)) in eset
