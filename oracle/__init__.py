"""CPU oracle for Delta-Motif embedding enumeration (arXiv 2508.21287).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg
may import this package; the library's product path never does. It shares no code with
the CUDA library: graphs come in as plain CSR arrays (any object with ``n``, ``row_ptr``,
``col_idx`` and optionally ``edge_err`` / ``qubit_err``).

The heavy lifting is ``oracle.c`` (plain C, compiled with gcc on first use); this module
adds ctypes marshalling, the image (vertex-set) dedup in numpy, and a pure-Python brute
force that serves as a second, independent check on tiny inputs.

What each function follows:
  enumerate / brute_force / brute_force_py - the problem statement of Sec. 3.1: injective
      maps f with every pattern edge mapped to a data edge (non-induced; ``induced`` adds the
      converse condition of the literal "iff").
  scores - Sec. 5.4: the layout score accumulated over the mapped edges (sum of errors,
      the log-domain form of the product of fidelities), FP64.
  scores_directed - the direction-aware post-processing of Sec. 5.4's footnote: every
      pattern slot p -> q weighted by its gate count times the device's cost in the direction
      f(p) -> f(q), FP64.
  topk   - Sec. 5.4 ranking: the k rows with the smallest (score, row).
  images - the distinct vertex sets of the embeddings (deduplication).
  checksum - the library's order-independent checksum (no counterpart in the paper).
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable flags, no -march)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.or_enumerate.restype = ctypes.c_int64
            lib.or_enumerate.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p,
                                         ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(_i32p), _u64p]
            lib.or_brute_force.restype = ctypes.c_int64
            lib.or_brute_force.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p,
                                           ctypes.c_int32, ctypes.POINTER(_i32p), _u64p]
            lib.or_free.argtypes = [ctypes.c_void_p]
            lib.or_mix64.restype = ctypes.c_uint64
            lib.or_mix64.argtypes = [ctypes.c_uint64]
            lib.or_row_hash.restype = ctypes.c_uint64
            lib.or_row_hash.argtypes = [_i32p, ctypes.c_int32]
            lib.or_checksum.restype = ctypes.c_uint64
            lib.or_checksum.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int32]
            lib.or_scores.restype = ctypes.c_int32
            lib.or_scores.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double)]
            lib.or_scores_directed.restype = ctypes.c_int32
            lib.or_scores_directed.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, _i32p, _i32p, ctypes.c_void_p, _i32p,
                                               ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
            lib.or_topk.restype = ctypes.c_int64
            lib.or_topk.argtypes = [_i32p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
            _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


@dataclass
class Result:
    rows: np.ndarray | None   # [count, n_p] int32, sorted lexicographically (None if count-only)
    count: int
    checksum: int


_ERRORS = {-1: "bad argument", -2: "pattern not connected", -3: "out of host memory"}


def _finish(rc, n_p, rows_p, cs, want_rows):
    lib = _load()
    if rc < 0:
        raise ValueError(f"oracle: {_ERRORS.get(rc, rc)}")
    rows = None
    if want_rows:
        rows = np.ctypeslib.as_array(rows_p, shape=(rc * n_p,)).copy().reshape(rc, n_p) if rc else \
            np.zeros((0, n_p), dtype=np.int32)
        lib.or_free(rows_p)
    return Result(rows, int(rc), int(cs.value))


def enumerate(data, pattern, induced: bool = False, threads: int = 1, rows: bool = True) -> Result:
    """All embeddings of ``pattern`` in ``data`` by backtracking (sorted rows, count, checksum)."""
    lib = _load()
    rp_d, ci_d = _i32(data.row_ptr), _i32(data.col_idx)
    rp_p, ci_p = _i32(pattern.row_ptr), _i32(pattern.col_idx)
    rows_p = _i32p()
    cs = ctypes.c_uint64(0)
    rc = lib.or_enumerate(int(data.n), _ptr(rp_d), _ptr(ci_d), int(pattern.n), _ptr(rp_p), _ptr(ci_p),
                          int(bool(induced)), int(threads), ctypes.byref(rows_p) if rows else None,
                          ctypes.byref(cs))
    return _finish(rc, int(pattern.n), rows_p, cs, rows)


def brute_force(data, pattern, induced: bool = False, rows: bool = True) -> Result:
    """All embeddings by trying every injective map (C, tiny inputs only)."""
    lib = _load()
    rp_d, ci_d = _i32(data.row_ptr), _i32(data.col_idx)
    rp_p, ci_p = _i32(pattern.row_ptr), _i32(pattern.col_idx)
    rows_p = _i32p()
    cs = ctypes.c_uint64(0)
    rc = lib.or_brute_force(int(data.n), _ptr(rp_d), _ptr(ci_d), int(pattern.n), _ptr(rp_p), _ptr(ci_p),
                            int(bool(induced)), ctypes.byref(rows_p) if rows else None, ctypes.byref(cs))
    return _finish(rc, int(pattern.n), rows_p, cs, rows)


def _edge_set(g):
    s = set()
    for u in range(int(g.n)):
        for k in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            s.add((u, int(g.col_idx[k])))
    return s


def brute_force_py(data, pattern, induced: bool = False) -> list[tuple[int, ...]]:
    """Pure-Python brute force over itertools.permutations (independent of oracle.c)."""
    de, pe = _edge_set(data), _edge_set(pattern)
    n_p = int(pattern.n)
    out = []
    for f in itertools.permutations(range(int(data.n)), n_p):
        ok = all((f[u], f[v]) in de for (u, v) in pe)
        if ok and induced:
            ok = all((u, v) in pe for u in range(n_p) for v in range(n_p)
                     if u != v and (f[u], f[v]) in de)
        if ok:
            out.append(tuple(f))
    return sorted(out)


def mix64(z: int) -> int:
    return int(_load().or_mix64(ctypes.c_uint64(z & ((1 << 64) - 1))))


def row_hash(row) -> int:
    r = _i32(row)
    return int(_load().or_row_hash(_ptr(r), len(r)))


def checksum(rows: np.ndarray) -> int:
    rows = _i32(rows)
    if rows.ndim != 2:
        raise ValueError("checksum needs a 2-D row array")
    return int(_load().or_checksum(_ptr(rows), rows.shape[0], rows.shape[1]))


def scores(data, pattern, rows: np.ndarray, form: int = 0) -> np.ndarray:
    """FP64 layout score per row over pattern edges (+ vertices): form 0 sums the error rates e,
    form 1 sums -log(1 - e), the negative log of the product of fidelities (Sec. 5.4)."""
    lib = _load()
    if data.edge_err is None:
        raise ValueError("scores need data.edge_err")
    rows = _i32(rows).reshape(-1, int(pattern.n))
    ee = np.ascontiguousarray(data.edge_err, dtype=np.float32)
    qe = None if getattr(data, "qubit_err", None) is None else np.ascontiguousarray(data.qubit_err, np.float32)
    out = np.empty(rows.shape[0], dtype=np.float64)
    rp_d, ci_d = _i32(data.row_ptr), _i32(data.col_idx)
    rp_p, ci_p = _i32(pattern.row_ptr), _i32(pattern.col_idx)
    rc = lib.or_scores(int(data.n), _ptr(rp_d), _ptr(ci_d), ee.ctypes.data,
                       None if qe is None else qe.ctypes.data, int(pattern.n), _ptr(rp_p), _ptr(ci_p),
                       _ptr(rows), rows.shape[0], int(form), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("scores: a row maps a pattern edge onto a non-edge")
    return out


def scores_directed(data, e_dir, pattern, w_dir, rows: np.ndarray) -> np.ndarray:
    """FP64 direction-aware score per row (Sec. 5.4 footnote): sum over pattern slots p -> q
    of w_dir[slot] * e_dir[slot of f(p) -> f(q)], plus data.qubit_err[f(u)] over pattern
    vertices when the data graph has vertex errors. e_dir is aligned with data.col_idx (cost
    of a gate from the row vertex to the column vertex), w_dir with pattern.col_idx."""
    lib = _load()
    rows = _i32(rows).reshape(-1, int(pattern.n))
    ed = np.ascontiguousarray(e_dir, dtype=np.float32)
    wd = np.ascontiguousarray(w_dir, dtype=np.float32)
    if len(ed) != len(data.col_idx) or len(wd) != len(pattern.col_idx):
        raise ValueError("e_dir / w_dir must be aligned with the data / pattern col_idx")
    qe = None if getattr(data, "qubit_err", None) is None else np.ascontiguousarray(data.qubit_err, np.float32)
    out = np.empty(rows.shape[0], dtype=np.float64)
    rp_d, ci_d = _i32(data.row_ptr), _i32(data.col_idx)
    rp_p, ci_p = _i32(pattern.row_ptr), _i32(pattern.col_idx)
    rc = lib.or_scores_directed(int(data.n), _ptr(rp_d), _ptr(ci_d), ed.ctypes.data,
                                None if qe is None else qe.ctypes.data, int(pattern.n), _ptr(rp_p), _ptr(ci_p),
                                wd.ctypes.data, _ptr(rows), rows.shape[0],
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("scores_directed: a row maps a pattern edge onto a non-edge")
    return out


def topk(rows: np.ndarray, score: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k rows with the smallest (score, row) key, in order."""
    rows = _i32(rows)
    sc = np.ascontiguousarray(score, dtype=np.float64)
    out = np.empty(max(1, min(k, rows.shape[0])), dtype=np.int64)
    m = _load().or_topk(_ptr(rows), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), rows.shape[0],
                        rows.shape[1] if rows.ndim == 2 else 1, int(k),
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out[:m]


def images(rows: np.ndarray) -> np.ndarray:
    """Distinct vertex sets covered by the embeddings, each sorted, rows sorted."""
    rows = np.asarray(rows, dtype=np.int32)
    if rows.shape[0] == 0:
        return rows.copy()
    return np.unique(np.sort(rows, axis=1), axis=0)


def automorphisms(pattern) -> int:
    """|Aut(G_p)| as the number of embeddings of the pattern in itself."""
    return enumerate(pattern, pattern, rows=False).count
