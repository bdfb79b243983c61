"""Seeded synthetic inputs for embedding enumeration: data graphs, pattern graphs, weights.

This module only builds inputs. It holds none of the enumeration method's arithmetic, so
that both the CUDA path and the CPU oracle can take their inputs from it.

Graphs are returned as symmetric CSR over int32 vertex ids (``Graph``): sorted neighbour
lists, no self-loops, no duplicate edges. The workloads follow the paper's evaluation
(Sec. 5.1, Sec. 5.2): heavy-hex and square-grid device topologies as data graphs, random
connected subgraphs as patterns, plus random 3-regular graphs and the tree / cycle /
subdivided-grid pattern families used for batching and serving.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), written out here,
so that a seed gives the same graph on every machine and numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64 stream: state advances by the golden gamma, output is the mixed state."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        return _mix64(self.state)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("below() needs n > 0")
        lim = (1 << 64) - ((1 << 64) % n)
        while True:
            x = self.next_u64()
            if x < lim:
                return x % n

    def shuffle(self, xs: list) -> None:
        for i in range(len(xs) - 1, 0, -1):
            j = self.below(i + 1)
            xs[i], xs[j] = xs[j], xs[i]


def splitmix64_block(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 seeded with ``seed``, vectorised (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + i * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


@dataclass
class Graph:
    """Undirected simple graph as symmetric CSR (int32), with optional FP32 weights.

    ``edge_err[k]`` is the weight of the directed slot ``col_idx[k]``; both slots of an
    undirected edge carry the same value. ``qubit_err[v]`` is a per-vertex weight.
    """

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    edge_err: np.ndarray | None = None
    qubit_err: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.row_ptr[-1]) // 2

    def edges(self) -> list[tuple[int, int]]:
        """Undirected edges (u, v) with u < v, sorted."""
        out = []
        for u in range(self.n):
            for k in range(self.row_ptr[u], self.row_ptr[u + 1]):
                v = int(self.col_idx[k])
                if u < v:
                    out.append((u, v))
        return out

    def neighbours(self, u: int) -> np.ndarray:
        return self.col_idx[self.row_ptr[u]:self.row_ptr[u + 1]]

    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def from_edges(n: int, edges, name: str = "", meta: dict | None = None) -> Graph:
    """Symmetric CSR from an undirected edge list; drops self-loops and repeated edges."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        u, v = int(u), int(v)
        if not (0 <= u < n and 0 <= v < n):
            raise ValueError(f"edge ({u},{v}) out of range for n={n}")
        if u == v:
            continue
        adj[u].add(v)
        adj[v].add(u)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for u in range(n):
        row_ptr[u + 1] = row_ptr[u] + len(adj[u])
    col_idx = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for u in range(n):
        col_idx[row_ptr[u]:row_ptr[u + 1]] = sorted(adj[u])
    return Graph(n, row_ptr, col_idx, name=name, meta=dict(meta or {}))


def is_connected(g: Graph) -> bool:
    if g.n == 0:
        return True
    seen = np.zeros(g.n, dtype=bool)
    seen[0] = True
    stack = [0]
    while stack:
        u = stack.pop()
        for v in g.neighbours(u):
            if not seen[v]:
                seen[v] = True
                stack.append(int(v))
    return bool(seen.all())


def relabel(g: Graph, perm) -> Graph:
    """The graph with vertex u renamed perm[u] (weights follow their edges and vertices)."""
    perm = [int(x) for x in perm]
    wmap = {}
    if g.edge_err is not None:
        for u in range(g.n):
            for k in range(g.row_ptr[u], g.row_ptr[u + 1]):
                wmap[(perm[u], perm[int(g.col_idx[k])])] = g.edge_err[k]
    h = from_edges(g.n, [(perm[u], perm[v]) for u, v in g.edges()], name=g.name + "-relabelled")
    if g.edge_err is not None:
        ee = np.empty(len(h.col_idx), dtype=np.float32)
        for u in range(h.n):
            for k in range(h.row_ptr[u], h.row_ptr[u + 1]):
                ee[k] = wmap[(u, int(h.col_idx[k]))]
        h.edge_err = ee
    if g.qubit_err is not None:
        qe = np.empty(g.n, dtype=np.float32)
        qe[np.asarray(perm)] = g.qubit_err
        h.qubit_err = qe
    return h


# ---------------------------------------------------------------------------------------
# Data graphs (Sec. 5.1: heavy-hex and square-grid topologies; random 3-regular for serving)
# ---------------------------------------------------------------------------------------

def grid(rows: int, cols: int) -> Graph:
    """2D square grid, vertex id = r * cols + c, 4-neighbour edges."""
    edges = []
    for r in range(rows):
        for c in range(cols):
            u = r * cols + c
            if c + 1 < cols:
                edges.append((u, u + 1))
            if r + 1 < rows:
                edges.append((u, u + cols))
    return from_edges(rows * cols, edges, name=f"grid{rows}x{cols}", meta={"kind": "grid"})


def honeycomb(m: int, n: int) -> Graph:
    """Honeycomb lattice with m rows and n columns of hexagonal cells (brick-wall layout).

    Lattice sites are (c, r) with c in [0, n], r in [0, 2m+1]. Each column is a vertical
    chain; columns c and c+1 are joined at rows r with (c + r) even. The two corner sites
    left with a single neighbour are dropped, leaving 2(m+1)(n+1) - 2 sites, and m*n cells.
    Ids are assigned in (r, c) row-major order of the kept sites.
    """
    sites = []
    for r in range(2 * m + 2):
        for c in range(n + 1):
            sites.append((c, r))

    def raw_edges():
        for c in range(n + 1):
            for r in range(2 * m + 1):
                yield (c, r), (c, r + 1)
        for c in range(n):
            for r in range(2 * m + 2):
                if (c + r) % 2 == 0:
                    yield (c, r), (c + 1, r)

    deg = {s: 0 for s in sites}
    for a, b in raw_edges():
        deg[a] += 1
        deg[b] += 1
    kept = [s for s in sites if deg[s] >= 2]
    ids = {s: i for i, s in enumerate(kept)}
    edges = [(ids[a], ids[b]) for a, b in raw_edges() if a in ids and b in ids]
    return from_edges(len(kept), edges, name=f"honeycomb{m}x{n}",
                      meta={"kind": "honeycomb", "m": m, "n": n})


def subdivide(g: Graph, name: str = "") -> Graph:
    """Every edge (u, v) replaced by u - x - v with a new vertex x (ids g.n, g.n+1, ...)."""
    edges = []
    x = g.n
    for u, v in g.edges():
        edges.append((u, x))
        edges.append((x, v))
        x += 1
    return from_edges(x, edges, name=name or g.name + "-subdivided")


def heavy_hex(m: int, n: int) -> Graph:
    """Heavy-hex lattice: the m x n honeycomb with every edge subdivided by one vertex.

    V = 5mn + 4m + 4n - 1. Cell count m*n; every cell is a 12-cycle.
    """
    h = subdivide(honeycomb(m, n), name=f"heavyhex{m}x{n}")
    h.meta = {"kind": "heavy_hex", "m": m, "n": n, "cells": m * n}
    return h


def random_regular3(n: int, seed: int) -> Graph:
    """Connected simple 3-regular graph on n (even) vertices from the pairing model.

    Stubs are shuffled with SplitMix64 seeded by ``seed``; a pairing with a loop, a repeated
    edge or more than one component is rejected and the stream continues.
    """
    if n % 2 or n < 4:
        raise ValueError("random_regular3 needs an even n >= 4")
    rng = SplitMix64(seed)
    for _ in range(10000):
        stubs = [v for v in range(n) for _ in range(3)]
        rng.shuffle(stubs)
        seen = set()
        ok = True
        for i in range(0, len(stubs), 2):
            u, v = stubs[i], stubs[i + 1]
            if u == v or (min(u, v), max(u, v)) in seen:
                ok = False
                break
            seen.add((min(u, v), max(u, v)))
        if not ok:
            continue
        g = from_edges(n, sorted(seen), name=f"regular3_{n}_s{seed}", meta={"kind": "regular3"})
        if is_connected(g):
            return g
    raise RuntimeError("random_regular3: no simple connected pairing found")


def lognormal_weights(g: Graph, seed: int, mu: float = -5.0, sigma: float = 0.5,
                      qubits: bool = False) -> Graph:
    """Attach log-normal(mu, sigma) FP32 error weights to every undirected edge.

    One draw per undirected edge (u < v, in sorted edge order) from Box-Muller over
    SplitMix64 uniforms in (0, 1]; both CSR slots of an edge get that value. With
    ``qubits`` a second stream (seed + 1) gives one weight per vertex.
    """
    def draws(s, k):
        x = splitmix64_block(s, 2 * k)
        u = ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u1, u2 = u[0::2], u[1::2]
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        return np.exp(mu + sigma * z).astype(np.float32)

    edges = g.edges()
    w = draws(seed, len(edges))
    wmap = {e: w[i] for i, e in enumerate(edges)}
    ee = np.empty(len(g.col_idx), dtype=np.float32)
    for u in range(g.n):
        for k in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col_idx[k])
            ee[k] = wmap[(min(u, v), max(u, v))]
    g.edge_err = ee
    g.qubit_err = draws(seed + 1, g.n) if qubits else None
    return g


def directed_errors(g: Graph, seed: int, mu: float = -5.0, sigma: float = 0.5,
                    reverse_mu: float = -7.0) -> np.ndarray:
    """Per-direction two-qubit gate costs aligned with ``g.col_idx`` (slot k of row u = a gate
    from u to col_idx[k]), as on hardware whose two-qubit gate runs natively one way per
    coupling: every undirected edge (u < v, sorted order) gets a seeded native direction and a
    log-normal(mu, sigma) error e; the other direction costs e plus two single-qubit gates of
    log-normal(reverse_mu, sigma) error each (the basis change that turns the gate around)."""
    edges = g.edges()
    m = len(edges)
    x = splitmix64_block(seed, 6 * m)
    u = ((x >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    z = np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * math.pi * u[1::2])  # 3m normals
    e = np.exp(mu + sigma * z[:m])
    extra = np.exp(reverse_mu + sigma * z[m:2 * m]) + np.exp(reverse_mu + sigma * z[2 * m:3 * m])
    forward = (x[:m] & np.uint64(1)) == 0  # native direction u -> v (else v -> u)
    cost = {}
    for i, (a, b) in enumerate(edges):
        nat, rev = float(e[i]), float(e[i] + extra[i])
        cost[(a, b)] = nat if forward[i] else rev
        cost[(b, a)] = rev if forward[i] else nat
    out = np.empty(len(g.col_idx), dtype=np.float32)
    for a in range(g.n):
        for k in range(g.row_ptr[a], g.row_ptr[a + 1]):
            out[k] = cost[(a, int(g.col_idx[k]))]
    return out


def gate_directions(p: Graph, seed: int, max_gates: int = 3) -> np.ndarray:
    """Per-direction two-qubit gate counts of a circuit aligned with ``p.col_idx``: every
    pattern edge (u < v) carries 1..max_gates seeded gates, each run from u to v or from v to
    u."""
    rng = SplitMix64(seed)
    cnt = {}
    for a, b in p.edges():
        n = 1 + rng.below(max_gates)
        fwd = sum(1 for _ in range(n) if rng.below(2) == 0)
        cnt[(a, b)], cnt[(b, a)] = fwd, n - fwd
    out = np.empty(len(p.col_idx), dtype=np.float32)
    for a in range(p.n):
        for k in range(p.row_ptr[a], p.row_ptr[a + 1]):
            out[k] = cnt[(a, int(p.col_idx[k]))]
    return out


# ---------------------------------------------------------------------------------------
# Pattern graphs
# ---------------------------------------------------------------------------------------

def path(k: int) -> Graph:
    return from_edges(k, [(i, i + 1) for i in range(k - 1)], name=f"path{k}")


def cycle(k: int) -> Graph:
    return from_edges(k, [(i, (i + 1) % k) for i in range(k)], name=f"cycle{k}")


def star(k: int) -> Graph:
    """Star with one centre (id 0) and k leaves; star(3) is the claw K_{1,3}."""
    return from_edges(k + 1, [(0, i) for i in range(1, k + 1)], name=f"star{k}")


def complete(k: int) -> Graph:
    return from_edges(k, [(i, j) for i in range(k) for j in range(i + 1, k)], name=f"K{k}")


def random_tree(n: int, seed: int, max_deg: int = 3) -> Graph:
    """Random tree on n vertices: vertex i attaches to a uniform earlier vertex of degree < max_deg."""
    rng = SplitMix64(seed)
    deg = [0] * n
    edges = []
    for i in range(1, n):
        cands = [j for j in range(i) if deg[j] < max_deg]
        j = cands[rng.below(len(cands))]
        edges.append((j, i))
        deg[i] += 1
        deg[j] += 1
    return from_edges(n, edges, name=f"tree{n}_s{seed}", meta={"kind": "tree"})


def cycle_with_chords(n: int, seed: int, n_chords: int = 2, max_deg: int = 3) -> Graph:
    """n-cycle plus up to n_chords chords between non-adjacent vertices of degree < max_deg."""
    rng = SplitMix64(seed)
    edges = {(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)}
    deg = [2] * n
    for _ in range(n_chords):
        for _attempt in range(64):
            a, b = rng.below(n), rng.below(n)
            e = (min(a, b), max(a, b))
            if a != b and e not in edges and deg[a] < max_deg and deg[b] < max_deg:
                edges.add(e)
                deg[a] += 1
                deg[b] += 1
                break
    return from_edges(n, sorted(edges), name=f"cyclechords{n}_s{seed}", meta={"kind": "cycle_chords"})


def subdivided_grid(rows: int, cols: int) -> Graph:
    g = subdivide(grid(rows, cols), name=f"subgrid{rows}x{cols}")
    g.meta = {"kind": "subdivided_grid"}
    return g


def sub_patch(g: Graph, n: int, seed: int, scramble: bool = True) -> Graph:
    """Random connected n-vertex induced subgraph of g, grown from a random vertex.

    Each step adds a uniform vertex of the current frontier. The pattern has at least one
    embedding (its own inclusion map). With ``scramble`` the pattern ids are a SplitMix64
    permutation of the growth order.
    """
    if n > g.n:
        raise ValueError("sub_patch larger than the data graph")
    rng = SplitMix64(seed)
    start = rng.below(g.n)
    chosen = [start]
    inside = {start}
    frontier = []
    for v in g.neighbours(start):
        frontier.append(int(v))
    while len(chosen) < n:
        frontier = [v for v in frontier if v not in inside]
        frontier = sorted(set(frontier))
        if not frontier:
            raise ValueError("sub_patch: component smaller than n")
        v = frontier[rng.below(len(frontier))]
        chosen.append(v)
        inside.add(v)
        frontier.extend(int(x) for x in g.neighbours(v))
    order = list(range(n))
    if scramble:
        rng.shuffle(order)
    pid = {chosen[i]: order[i] for i in range(n)}
    edges = [(pid[u], pid[int(v)]) for u in chosen for v in g.neighbours(u) if int(v) in inside]
    p = from_edges(n, edges, name=f"patch{n}_s{seed}", meta={"kind": "sub_patch", "embedding": [
        chosen[order.index(i)] for i in range(n)]})
    return p


# 2 x k grids keep the maximum degree at 3 once subdivided (5k - 2 vertices).
_SUBGRID_SHAPES = [(2, k) for k in range(2, 9)]


def mixed_pattern(seed: int, n_min: int = 5, n_max: int = 40) -> Graph:
    """Pattern of a mixed batch: seed % 3 picks a tree, a cycle or a subdivided grid.

    Trees: max degree 3, n uniform in [n_min, n_max]. Cycles: length uniform in
    [max(12, n_min), n_max] (heavy-hex has girth 12). Subdivided grids: a 2 x k grid with
    every edge subdivided (girth 8, max degree 3), k picked by the seed among the shapes
    whose vertex count is in range.
    """
    rng = SplitMix64(0x5EED0000 + seed)
    kind = seed % 3
    if kind == 0:
        n = n_min + rng.below(n_max - n_min + 1)
        return random_tree(n, seed)
    if kind == 1:
        lo = max(12, n_min)
        n = lo + rng.below(max(1, n_max - lo + 1))
        return cycle(n)
    shapes = [s for s in _SUBGRID_SHAPES
              if n_min <= s[0] * s[1] + s[0] * (s[1] - 1) + s[1] * (s[0] - 1) <= n_max]
    r, c = shapes[rng.below(len(shapes))]
    return subdivided_grid(r, c)


def c2_pattern(seed: int, n_min: int = 10, n_max: int = 30) -> Graph:
    """Layout-query pattern on a ~160-vertex heavy-hex: even seeds give a random tree with
    max degree 3, odd seeds a cycle with chords; size uniform in [n_min, n_max]."""
    rng = SplitMix64(0xC2C2 + seed)
    n = n_min + rng.below(n_max - n_min + 1)
    if seed % 2 == 0:
        return random_tree(n, seed)
    return cycle_with_chords(n, seed, n_chords=1 + rng.below(2))


def random_subtree(g: Graph, n: int, seed: int) -> Graph:
    """Random n-vertex tree that is a subgraph of g: a random spanning tree (Kruskal over
    SplitMix64 edge keys) of the patch ``sub_patch(g, n, seed)``. Always embeddable in g;
    its maximum degree is at most g's."""
    patch = sub_patch(g, n, seed)
    rng = SplitMix64(seed ^ 0x7EEE)
    es = patch.edges()
    keys = [rng.next_u64() for _ in es]
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    tree = []
    for _, (u, v) in sorted(zip(keys, es)):
        a, b = find(u), find(v)
        if a != b:
            parent[a] = b
            tree.append((u, v))
    t = from_edges(n, tree, name=f"subtree{n}_s{seed}", meta={"kind": "subtree"})
    return t


def layout_query(g: Graph, seed: int, n_min: int = 10, n_max: int = 30) -> Graph:
    """A layout query that fits the device graph g: even seeds give a random spanning tree of
    a random device patch, odd seeds the induced patch itself (on heavy-hex it contains the
    12-cycles of the cells with the paths between them as chords). Size uniform in
    [n_min, n_max]."""
    rng = SplitMix64(0x1A70 + seed)
    n = n_min + rng.below(n_max - n_min + 1)
    if seed % 2 == 0:
        return random_subtree(g, n, seed)
    return sub_patch(g, n, seed)
