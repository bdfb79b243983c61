"""Thin Python binding of include/dm.h (ctypes). Argument marshalling only: every step of the
enumeration runs in libdmotif.so's CUDA kernels. Functions keep the C names; failures raise
DMError with the library's status code.

The library must have been built (``python -m paper_2508_21287_gb300.build`` or
``__graft_entry__.build()``); importing this module without it raises immediately. There is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdmotif.so")

DM_OK = 0
DM_E_INVAL, DM_E_DISCONNECTED, DM_E_NOMEM, DM_E_CAPACITY = -1, -2, -3, -4
DM_E_TIMEOUT, DM_E_CUDA, DM_E_CANCELLED, DM_E_NOTFOUND = -5, -6, -7, -8
DM_ALL, DM_COUNT, DM_DEVICE_ROWS = 0, 1, 0x10
DM_ORDER_PAPER, DM_ORDER_HEURISTIC, DM_ORDER_LEARNED = 0, 1, 2
DM_JOIN_AUTO, DM_JOIN_HASH, DM_JOIN_SORTMERGE = 0, 1, 2
DM_MAX_STEPS = 128


def DM_MOTIF_PATH(k: int) -> int:
    return k


def DM_MOTIF_CYCLE(k: int) -> int:
    return 100 + k


DM_MOTIF_M4_1, DM_MOTIF_M6_2O, DM_MOTIF_M18_O_6 = 201, 202, 203


class DMError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {dm_strerror(code)} ({code})" + (f" [{detail}]" if detail else ""))


class dm_plan_opts(ctypes.Structure):
    _fields_ = [("motifs", ctypes.POINTER(ctypes.c_int32)), ("n_motifs", ctypes.c_int32),
                ("order", ctypes.c_int32), ("join_algo", ctypes.c_int32), ("induced", ctypes.c_int32),
                ("chunk_rows", ctypes.c_int64), ("max_rows", ctypes.c_int64)]


class dm_stats(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("rows", ctypes.c_int64 * DM_MAX_STEPS),
                ("candidates", ctypes.c_int64 * DM_MAX_STEPS), ("chunks", ctypes.c_int64),
                ("max_rows", ctypes.c_int64), ("join_ms", ctypes.c_double),
                ("join_launches", ctypes.c_int64), ("join_bytes", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]


class dm_server_opts(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_int32), ("mem_budget_bytes", ctypes.c_uint64), ("max_rows", ctypes.c_int64),
                ("order", ctypes.c_int32), ("motifs", ctypes.POINTER(ctypes.c_int32)), ("n_motifs", ctypes.c_int32)]


class dm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("pool_used", ctypes.c_uint64), ("pool_total", ctypes.c_uint64),
                ("max_running", ctypes.c_int64), ("overlapped", ctypes.c_int64)]


DM_CHUNK_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_int32)
DM_QUERY_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_int32)

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(the library has no CPU fallback)")
_lib = ctypes.CDLL(LIB_PATH)

_vp, _i32, _i64, _u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_i32p = ctypes.POINTER(ctypes.c_int32)
_fp = ctypes.POINTER(ctypes.c_float)
_u64p = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "dm_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _u64]),
    "dm_destroy": (ctypes.c_int, [_vp]),
    "dm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "dm_set_budget": (ctypes.c_int, [_vp, _u64]),
    "dm_load_data_graph": (ctypes.c_int, [_vp, _i32, _i32p, _i32p, _fp, _fp, _i32p]),
    "dm_load_data_graph_ex": (ctypes.c_int, [_vp, _i32, _i32p, _i32p, _fp, _fp, _i32, _i32p]),
    "dm_motif_table": (ctypes.c_int, [_vp, _i32, _i32, _i32p, _i64, ctypes.POINTER(_i64), _i32p]),
    "dm_plan": (ctypes.c_int, [_vp, _i32, _i32, _i32p, _i32p, ctypes.POINTER(dm_plan_opts), ctypes.POINTER(_vp)]),
    "dm_plan_free": (None, [_vp]),
    "dm_plan_predicted_rows": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), _i32]),
    "dm_match_topk_queries": (ctypes.c_int, [ctypes.POINTER(_vp), _i32p, _i32, _i32, _i32p, ctypes.POINTER(_i32p),
                                             ctypes.POINTER(_i32p), ctypes.POINTER(dm_plan_opts), ctypes.c_int,
                                             DM_QUERY_CB, _vp, _i32, ctypes.POINTER(_i32p), ctypes.POINTER(_fp),
                                             _i32p, _u64p, _u64p, _i32p, ctypes.POINTER(dm_stats)]),
    "dm_plan_batch": (ctypes.c_int, [_vp, _i32, _i32, _i32p, ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                     ctypes.POINTER(dm_plan_opts), ctypes.POINTER(_vp)]),
    "dm_plan_candidates": (_i32, [_vp, _i32, _i32, _i32p, _i32p, ctypes.POINTER(dm_plan_opts), ctypes.POINTER(_vp), _i32]),
    "dm_plan_describe": (_i32, [_vp, _i32p, _i32]),
    "dm_match": (ctypes.c_int, [_vp, _vp, ctypes.c_int, DM_CHUNK_CB, _vp, _u64p, _u64p]),
    "dm_match_batch": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), _i32, ctypes.c_int, _u64p, _u64p]),
    "dm_match_shard": (ctypes.c_int, [_vp, _vp, _i32, _i32, _u64p, _u64p]),
    "dm_score_topk": (ctypes.c_int, [_vp, _vp, _i32, _i32p, _fp, _i32p]),
    "dm_match_topk": (ctypes.c_int, [_vp, _vp, ctypes.c_int, DM_CHUNK_CB, _vp, _i32, _i32p, _fp, _i32p, _u64p, _u64p]),
    "dm_load_directed_errors": (ctypes.c_int, [_vp, _i32, _fp]),
    "dm_score_topk_directed": (ctypes.c_int, [_vp, _vp, _fp, _i32, _i32p, _fp, _i32p]),
    "dm_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(dm_stats)]),
    "dm_enable_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "dm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "dm_last_error": (ctypes.c_char_p, [_vp]),
    "dm_decompose": (_i32, [_i32, _i32p, _i32p, _i32p, _i32, _i32, _i32p, _i32]),
    "dm_sort_rows_static": (ctypes.c_int, [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp]),
    "dm_batch_config": (ctypes.c_int, [_vp, _i32p, ctypes.POINTER(_i64), _i32p, _i32p, ctypes.POINTER(ctypes.c_double),
                                       _i32p, _i32p, ctypes.POINTER(ctypes.c_double)]),
    "dm_set_batch_shape": (ctypes.c_int, [_vp, _i32, _i32]),
    "dm_set_fusion": (ctypes.c_int, [_vp, ctypes.c_int]),
    "dm_batch_latency": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _i32]),
    "dm_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "dm_model_init": (ctypes.c_int, [_vp, _u64]),
    "dm_model_train": (ctypes.c_int, [_vp, _fp, _fp, _i32, _i32, _i32, ctypes.c_float, _u64, _fp]),
    "dm_model_predict": (ctypes.c_int, [_vp, _fp, _i32, _fp]),
    "dm_model_grad": (ctypes.c_int, [_vp, _fp, _fp, _i32, _fp, _fp, _fp]),
    "dm_model_weights": (ctypes.c_int, [_vp, _fp, ctypes.POINTER(_i64)]),
    "dm_model_set_weights": (ctypes.c_int, [_vp, _fp, _i64]),
    "dm_step_log": (ctypes.c_int, [_vp, _fp, _fp, _i64, ctypes.POINTER(_i64), ctypes.c_int]),
    "dm_plan_estimates": (_i32, [_vp, _fp, _fp, _i32]),
    "dm_images": (ctypes.c_int, [_vp, _vp, _i32p, _i64, ctypes.POINTER(_i64)]),
    "dm_plan_cost": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "dm_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(dm_server_opts)]),
    "dm_server_load_graph": (ctypes.c_int, [_vp, _i32, _i32p, _i32p, _fp, _fp, _i32p]),
    "dm_server_set_model": (ctypes.c_int, [_vp, _fp, _i64]),
    "dm_server_submit": (ctypes.c_int, [_vp, _i32, _i32, _i32p, _i32p, _i32, _u64p]),
    "dm_server_wait": (ctypes.c_int, [_vp, _u64, _i32p, _fp, _i32p, _i32p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "dm_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(dm_server_stats)]),
    "dm_server_destroy": (ctypes.c_int, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def dm_strerror(code: int) -> str:
    return _lib.dm_strerror(int(code)).decode()


def dm_last_error(ctx) -> str:
    return _lib.dm_last_error(ctx).decode()


def _check(rc: int, what: str, ctx=None):
    if rc != DM_OK:
        raise DMError(rc, what, dm_last_error(ctx) if ctx else "")


def _arr_i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


def dm_create(device: int = 0, mem_budget_bytes: int = 0):
    h = _vp()
    _check(_lib.dm_create(ctypes.byref(h), int(device), int(mem_budget_bytes)), "dm_create")
    return h


def dm_destroy(ctx) -> None:
    _check(_lib.dm_destroy(ctx), "dm_destroy")


def dm_set_stream(ctx, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None for the context's own."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(_lib.dm_set_stream(ctx, _vp(raw) if raw else None), "dm_set_stream", ctx)


def dm_set_budget(ctx, mem_budget_bytes: int) -> None:
    _check(_lib.dm_set_budget(ctx, int(mem_budget_bytes)), "dm_set_budget", ctx)


def dm_load_data_graph(ctx, n_vertices: int, row_ptr, col_idx, edge_err=None, qubit_err=None) -> int:
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    ee = None if edge_err is None else np.ascontiguousarray(edge_err, dtype=np.float32)
    qe = None if qubit_err is None else np.ascontiguousarray(qubit_err, dtype=np.float32)
    out = _i32()
    rc = _lib.dm_load_data_graph(ctx, int(n_vertices), _p32(rp), _p32(ci),
                                 None if ee is None else ee.ctypes.data_as(_fp),
                                 None if qe is None else qe.ctypes.data_as(_fp), ctypes.byref(out))
    _check(rc, "dm_load_data_graph", ctx)
    return out.value


DM_SCORE_ERROR_SUM, DM_SCORE_LOG_FIDELITY = 0, 1


def dm_load_data_graph_ex(ctx, n_vertices: int, row_ptr, col_idx, edge_err=None, qubit_err=None,
                          score_form: int = DM_SCORE_ERROR_SUM) -> int:
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    ee = None if edge_err is None else np.ascontiguousarray(edge_err, dtype=np.float32)
    qe = None if qubit_err is None else np.ascontiguousarray(qubit_err, dtype=np.float32)
    out = _i32()
    rc = _lib.dm_load_data_graph_ex(ctx, int(n_vertices), _p32(rp), _p32(ci),
                                    None if ee is None else ee.ctypes.data_as(_fp),
                                    None if qe is None else qe.ctypes.data_as(_fp), int(score_form),
                                    ctypes.byref(out))
    _check(rc, "dm_load_data_graph_ex", ctx)
    return out.value


def dm_motif_table(ctx, graph: int, motif_id: int) -> np.ndarray:
    n, k = _i64(), _i32()
    _check(_lib.dm_motif_table(ctx, int(graph), int(motif_id), None, 0, ctypes.byref(n), ctypes.byref(k)),
           "dm_motif_table", ctx)
    rows = np.empty((n.value, k.value), dtype=np.int32)
    if n.value:
        _check(_lib.dm_motif_table(ctx, int(graph), int(motif_id), _p32(rows), n.value, ctypes.byref(n),
                                   ctypes.byref(k)), "dm_motif_table", ctx)
    return rows


def dm_plan(ctx, graph: int, n_p: int, row_ptr, col_idx, motifs=None, order: int = DM_ORDER_PAPER,
            join_algo: int = DM_JOIN_AUTO, chunk_rows: int = 0, max_rows: int = 0, induced: bool = False):
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    opts = dm_plan_opts()
    keep = None
    if motifs:
        keep = _arr_i32(list(motifs))
        opts.motifs = _p32(keep)
        opts.n_motifs = len(keep)
    opts.order, opts.join_algo = int(order), int(join_algo)
    opts.chunk_rows, opts.max_rows = int(chunk_rows), int(max_rows)
    opts.induced = int(bool(induced))
    h = _vp()
    _check(_lib.dm_plan(ctx, int(graph), int(n_p), _p32(rp), _p32(ci), ctypes.byref(opts), ctypes.byref(h)),
           "dm_plan", ctx)
    return h


def dm_plan_batch(ctx, graph: int, patterns, motifs=None, order: int = DM_ORDER_PAPER,
                  join_algo: int = DM_JOIN_AUTO, chunk_rows: int = 0, max_rows: int = 0,
                  induced: bool = False) -> list:
    """dm_plan for a list of (n_p, row_ptr, col_idx) patterns with shared options."""
    n = len(patterns)
    arrs = [(_arr_i32(rp), _arr_i32(ci)) for _, rp, ci in patterns]
    n_p = _arr_i32([int(p[0]) for p in patterns] or [0])
    rps = (_i32p * max(1, n))(*[_p32(a[0]) for a in arrs])
    cis = (_i32p * max(1, n))(*[_p32(a[1]) for a in arrs])
    opts = dm_plan_opts()
    keep = None
    if motifs:
        keep = _arr_i32(list(motifs))
        opts.motifs = _p32(keep)
        opts.n_motifs = len(keep)
    opts.order, opts.join_algo = int(order), int(join_algo)
    opts.chunk_rows, opts.max_rows = int(chunk_rows), int(max_rows)
    opts.induced = int(bool(induced))
    out = (_vp * max(1, n))()
    _check(_lib.dm_plan_batch(ctx, int(graph), n, _p32(n_p), rps, cis, ctypes.byref(opts), out),
           "dm_plan_batch", ctx)
    return [_vp(out[i]) for i in range(n)]


def dm_plan_free(plan) -> None:
    _lib.dm_plan_free(plan)


def dm_plan_candidates(ctx, graph: int, n_p: int, row_ptr, col_idx, motifs=None, max_rows: int = 0) -> list:
    """The candidate plans DM_ORDER_LEARNED chooses from, as plan handles (free each)."""
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    opts = dm_plan_opts()
    opts.max_rows = int(max_rows)
    keep = None
    if motifs:
        keep = _arr_i32(list(motifs))
        opts.motifs = _p32(keep)
        opts.n_motifs = len(keep)
    n = _lib.dm_plan_candidates(ctx, int(graph), int(n_p), _p32(rp), _p32(ci), ctypes.byref(opts), None, 0)
    _check(min(n, 0), "dm_plan_candidates", ctx)
    arr = (_vp * max(1, n))()
    got = _lib.dm_plan_candidates(ctx, int(graph), int(n_p), _p32(rp), _p32(ci), ctypes.byref(opts), arr, n)
    _check(min(got, 0), "dm_plan_candidates", ctx)
    return [_vp(arr[i]) for i in range(got)]


def _parse_description(words: list[int]) -> list[dict]:
    steps, i = [], 1
    for _ in range(words[0]):
        motif, k = words[i], words[i + 1]
        sl = words[i + 2:i + 2 + k]
        i += 2 + k
        n_keys, n_be = words[i], words[i + 1]
        i += 2
        be = [(words[i + 2 * j], words[i + 2 * j + 1]) for j in range(n_be)]
        i += 2 * n_be
        steps.append({"motif": motif, "slice": sl, "n_keys": n_keys, "backedges": be})
    return steps


def dm_plan_describe(plan) -> list[dict]:
    n = _lib.dm_plan_describe(plan, None, 0)
    if n < 0:
        raise DMError(n, "dm_plan_describe")
    buf = np.zeros(n, dtype=np.int32)
    _lib.dm_plan_describe(plan, _p32(buf), n)
    return _parse_description(buf.tolist())


def dm_decompose(n_p: int, row_ptr, col_idx, motifs, order: int = DM_ORDER_PAPER) -> list[dict]:
    """Host-only decomposition (no data graph): the plan's slice list, as dm_plan_describe."""
    rp, ci, ms = _arr_i32(row_ptr), _arr_i32(col_idx), _arr_i32(list(motifs))
    n = _lib.dm_decompose(int(n_p), _p32(rp), _p32(ci), _p32(ms), len(ms), int(order), None, 0)
    if n < 0:
        raise DMError(n, "dm_decompose")
    buf = np.zeros(n, dtype=np.int32)
    _lib.dm_decompose(int(n_p), _p32(rp), _p32(ci), _p32(ms), len(ms), int(order), _p32(buf), n)
    return _parse_description(buf.tolist())


def _make_cb(cb, mode, err):
    def _tramp(user, rows, scores, nrows, ncols):
        try:
            if mode & DM_DEVICE_ROWS:
                r = cb(ctypes.cast(rows, ctypes.c_void_p).value, ctypes.cast(scores, ctypes.c_void_p).value,
                       nrows, ncols)
            else:
                a = np.ctypeslib.as_array(rows, shape=(nrows * ncols,)).reshape(nrows, ncols).copy()
                s = np.ctypeslib.as_array(scores, shape=(nrows,)).copy() if scores else None
                r = cb(a, s)
            return int(bool(r))
        except BaseException as e:  # noqa: BLE001 - re-raised after the C call returns
            err.append(e)
            return 1
    return DM_CHUNK_CB(_tramp) if cb is not None else DM_CHUNK_CB()


def dm_match_topk(ctx, plan, mode: int, cb, k: int, n_p: int):
    """All rows through cb (as dm_match) plus the top-k; returns (rows, scores, count, checksum)."""
    err = []
    c_cb = _make_cb(cb, mode, err)
    rows = np.zeros((k, n_p), dtype=np.int32)
    scores = np.zeros(k, dtype=np.float32)
    n = _i32()
    cnt, cs = _u64(), _u64()
    rc = _lib.dm_match_topk(ctx, plan, int(mode), c_cb, None, int(k), _p32(rows), scores.ctypes.data_as(_fp),
                            ctypes.byref(n), ctypes.byref(cnt), ctypes.byref(cs))
    if err:
        raise err[0]
    _check(rc, "dm_match_topk", ctx)
    return rows[:n.value], scores[:n.value], cnt.value, cs.value


class QueryBatch:
    """Queries marshalled once for dm_match_topk_queries, with their output buffers: a caller
    that answers the same queries repeatedly passes this instead of the pattern list."""

    def __init__(self, patterns, k: int):
        self.k = int(k)
        self.n = n = len(patterns)
        self._arrs = [(_arr_i32(rp), _arr_i32(ci)) for _, rp, ci in patterns]
        self.n_p = _arr_i32([int(p[0]) for p in patterns] or [0])
        self.rps = (_i32p * max(1, n))(*[_p32(a[0]) for a in self._arrs])
        self.cis = (_i32p * max(1, n))(*[_p32(a[1]) for a in self._arrs])
        self.rows = [np.zeros((self.k, int(p[0])), dtype=np.int32) for p in patterns]
        self.scores = [np.zeros(self.k, dtype=np.float32) for _ in patterns]
        self.rows_p = (_i32p * max(1, n))(*[_p32(r) for r in self.rows])
        self.scores_p = (_fp * max(1, n))(*[x.ctypes.data_as(_fp) for x in self.scores])
        self.out_n = np.zeros(max(1, n), dtype=np.int32)
        self.counts = np.zeros(max(1, n), dtype=np.uint64)
        self.sums = np.zeros(max(1, n), dtype=np.uint64)
        self.status = np.zeros(max(1, n), dtype=np.int32)


def dm_match_topk_queries(ctxs, gids, patterns, k: int, mode: int = DM_ALL, cb=None, motifs=None,
                          order: int = DM_ORDER_PAPER):
    """Many (n_p, row_ptr, col_idx) queries (or a QueryBatch) over several contexts at once,
    one host thread per context. cb(query, rows, scores) receives host copies, or cb(query,
    rows_ptr, scores_ptr, m, n) device pointers with DM_DEVICE_ROWS, from the worker threads.
    Returns a list of (rows, scores, count, checksum, status) per query (rows and scores are
    views of the batch's buffers) and the summed statistics."""
    qb = patterns if isinstance(patterns, QueryBatch) else QueryBatch(patterns, k)
    if qb.k != int(k):
        raise ValueError("QueryBatch was made for another k")
    n = qb.n
    ctx_arr = (_vp * len(ctxs))(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    gid_arr = _arr_i32(list(gids))
    opts = dm_plan_opts()
    keep = None
    if motifs:
        keep = _arr_i32(list(motifs))
        opts.motifs = _p32(keep)
        opts.n_motifs = len(keep)
    opts.order = int(order)
    err = []

    def _tramp(user, q, r, sc, nrows, ncols):
        try:
            if mode & DM_DEVICE_ROWS:
                res = cb(q, ctypes.cast(r, ctypes.c_void_p).value, ctypes.cast(sc, ctypes.c_void_p).value, nrows, ncols)
            else:
                a = np.ctypeslib.as_array(r, shape=(nrows * ncols,)).reshape(nrows, ncols).copy()
                s_ = np.ctypeslib.as_array(sc, shape=(nrows,)).copy() if sc else None
                res = cb(q, a, s_)
            return int(bool(res))
        except BaseException as e:  # noqa: BLE001 - re-raised after the C call returns
            err.append(e)
            return 1
    c_cb = DM_QUERY_CB(_tramp) if cb is not None else DM_QUERY_CB()
    st = dm_stats()
    rc = _lib.dm_match_topk_queries(ctx_arr, _p32(gid_arr), len(ctxs), n, _p32(qb.n_p), qb.rps, qb.cis,
                                    ctypes.byref(opts), int(mode), c_cb, None, int(k), qb.rows_p, qb.scores_p,
                                    _p32(qb.out_n), qb.counts.ctypes.data_as(_u64p), qb.sums.ctypes.data_as(_u64p),
                                    _p32(qb.status), ctypes.byref(st))
    if err:
        raise err[0]
    _check(rc, "dm_match_topk_queries")
    on, cn, sm, stt = qb.out_n.tolist(), qb.counts.tolist(), qb.sums.tolist(), qb.status.tolist()
    res = [(qb.rows[i][:on[i]], qb.scores[i][:on[i]], cn[i], sm[i], stt[i]) for i in range(n)]
    stats = {"chunks": st.chunks, "max_rows": st.max_rows, "join_ms": st.join_ms, "join_launches": st.join_launches,
             "join_bytes": st.join_bytes, "total_ms": st.total_ms, "kernel_launches": st.kernel_launches}
    return res, stats


def dm_match(ctx, plan, mode: int = DM_ALL, cb=None):
    """Run the plan. cb(rows ndarray [m, n] int32, scores ndarray [m] or None) receives host
    copies (DM_ALL); with DM_DEVICE_ROWS in mode it receives (rows_ptr, scores_ptr, m, n) raw
    device pointers instead. Returns (count, checksum)."""
    err = []
    c_cb = _make_cb(cb, mode, err)
    cnt, cs = _u64(), _u64()
    rc = _lib.dm_match(ctx, plan, int(mode), c_cb, None, ctypes.byref(cnt), ctypes.byref(cs))
    if err:
        raise err[0]
    _check(rc, "dm_match", ctx)
    return cnt.value, cs.value


def dm_match_shard(ctx, plan, shard: int, n_shards: int):
    """Count and checksum of one shard of R_0 (see include/dm.h); returns (count, checksum)."""
    cnt, cs = _u64(), _u64()
    _check(_lib.dm_match_shard(ctx, plan, int(shard), int(n_shards), ctypes.byref(cnt), ctypes.byref(cs)),
           "dm_match_shard", ctx)
    return cnt.value, cs.value


def dm_match_batch(ctx, plans, mode: int = DM_COUNT):
    arr = (_vp * len(plans))(*[p.value if isinstance(p, _vp) else p for p in plans])
    counts = np.zeros(len(plans), dtype=np.uint64)
    sums = np.zeros(len(plans), dtype=np.uint64)
    rc = _lib.dm_match_batch(ctx, arr, len(plans), int(mode), counts.ctypes.data_as(_u64p),
                             sums.ctypes.data_as(_u64p))
    _check(rc, "dm_match_batch", ctx)
    return counts, sums


def dm_batch_config(ctx) -> dict:
    tr, ch, gr, nh, hv = _i32(), _i64(), _i32(), _i32(), ctypes.c_double()
    th, cps, lf = _i32(), _i32(), ctypes.c_double()
    _check(_lib.dm_batch_config(ctx, ctypes.byref(tr), ctypes.byref(ch), ctypes.byref(gr), ctypes.byref(nh),
                                ctypes.byref(hv), ctypes.byref(th), ctypes.byref(cps), ctypes.byref(lf)),
           "dm_batch_config", ctx)
    return {"tile_rows": tr.value, "root_chunk": ch.value, "grid": gr.value, "stepwise_plans": nh.value,
            "heavy_rows": hv.value if hv.value < 1e300 else None, "threads_per_cta": th.value,
            "ctas_per_sm": cps.value, "hash_load_factor": lf.value}


def dm_set_batch_shape(ctx, threads_per_cta: int = 256, ctas_per_sm: int = 0) -> None:
    """Block shape of dm_match_batch without autotuning: 128 or 256 threads a CTA (CTA walks),
    or 32 (one walk per warp, two warps a CTA); ctas_per_sm 0 = as many as fit."""
    _check(_lib.dm_set_batch_shape(ctx, int(threads_per_cta), int(ctas_per_sm)), "dm_set_batch_shape", ctx)


def dm_set_fusion(ctx, on: bool = True) -> None:
    _check(_lib.dm_set_fusion(ctx, int(bool(on))), "dm_set_fusion", ctx)


def dm_batch_latency(ctx, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.float64)
    _check(_lib.dm_batch_latency(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n)),
           "dm_batch_latency", ctx)
    return out


def dm_set_tuning(ctx, autotune: bool = True, hash_load_factor: float = 0.5, heavy_rows: float = 0.0) -> None:
    _check(_lib.dm_set_tuning(ctx, int(bool(autotune)), float(hash_load_factor), float(heavy_rows)),
           "dm_set_tuning", ctx)


DM_MODEL_FEATURES = 32


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _pf(a: np.ndarray):
    return a.ctypes.data_as(_fp)


def dm_model_init(ctx, seed: int = 1) -> None:
    _check(_lib.dm_model_init(ctx, int(seed)), "dm_model_init", ctx)


def dm_model_train(ctx, feats, targets, epochs: int = 30, batch: int = 256, lr: float = 1e-3, seed: int = 1):
    x, t = _f32(feats).reshape(-1, DM_MODEL_FEATURES), _f32(targets)
    loss = np.zeros(epochs, dtype=np.float32)
    _check(_lib.dm_model_train(ctx, _pf(x), _pf(t), len(t), int(epochs), int(batch), float(lr), int(seed), _pf(loss)),
           "dm_model_train", ctx)
    return loss


def dm_model_predict(ctx, feats) -> np.ndarray:
    x = _f32(feats).reshape(-1, DM_MODEL_FEATURES)
    out = np.zeros(len(x), dtype=np.float32)
    _check(_lib.dm_model_predict(ctx, _pf(x), len(x), _pf(out)), "dm_model_predict", ctx)
    return out


def dm_model_grad(ctx, feats, targets=None):
    x = _f32(feats).reshape(-1, DM_MODEL_FEATURES)
    t = None if targets is None else _f32(targets)
    pred = np.zeros(len(x), dtype=np.float32)
    n = _i64()
    _lib.dm_model_weights(ctx, None, ctypes.byref(n))
    grads = np.zeros(n.value - 2 * DM_MODEL_FEATURES, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(_lib.dm_model_grad(ctx, _pf(x), None if t is None else _pf(t), len(x), _pf(pred),
                              _pf(grads) if t is not None else None, _pf(loss)), "dm_model_grad", ctx)
    return pred, (grads if t is not None else None), float(loss[0])


def dm_model_weights(ctx) -> np.ndarray:
    n = _i64()
    _check(_lib.dm_model_weights(ctx, None, ctypes.byref(n)), "dm_model_weights", ctx)
    w = np.zeros(n.value, dtype=np.float32)
    _check(_lib.dm_model_weights(ctx, _pf(w), ctypes.byref(n)), "dm_model_weights", ctx)
    return w


def dm_model_set_weights(ctx, w) -> None:
    w = _f32(w)
    _check(_lib.dm_model_set_weights(ctx, _pf(w), len(w)), "dm_model_set_weights", ctx)


def dm_step_log(ctx, clear: bool = False):
    n = _i64()
    _check(_lib.dm_step_log(ctx, None, None, 0, ctypes.byref(n), 0), "dm_step_log", ctx)
    f = np.zeros((n.value, DM_MODEL_FEATURES), dtype=np.float32)
    t = np.zeros(n.value, dtype=np.float32)
    _check(_lib.dm_step_log(ctx, _pf(f), _pf(t), n.value, ctypes.byref(n), int(bool(clear))), "dm_step_log", ctx)
    return f, t


def dm_images(ctx, plan, n_p: int) -> np.ndarray:
    n = _i64()
    _check(_lib.dm_images(ctx, plan, None, 0, ctypes.byref(n)), "dm_images", ctx)
    out = np.zeros((n.value, n_p), dtype=np.int32)
    if n.value:
        _check(_lib.dm_images(ctx, plan, _p32(out), n.value, ctypes.byref(n)), "dm_images", ctx)
    return out


def dm_plan_cost(plan):
    c, m = ctypes.c_double(), ctypes.c_double()
    _check(_lib.dm_plan_cost(plan, ctypes.byref(c), ctypes.byref(m)), "dm_plan_cost")
    return c.value, m.value


def dm_plan_predicted_rows(plan) -> np.ndarray:
    n = _lib.dm_plan_predicted_rows(plan, None, 0)
    _check(min(n, 0), "dm_plan_predicted_rows")
    out = np.zeros(max(1, n), dtype=np.float64)
    _lib.dm_plan_predicted_rows(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
    return out[:n]


def dm_plan_estimates(plan):
    n = _lib.dm_plan_estimates(plan, None, None, 0)
    f = np.zeros((n, DM_MODEL_FEATURES), dtype=np.float32)
    h = np.zeros(n, dtype=np.float32)
    _lib.dm_plan_estimates(plan, _pf(f), _pf(h), n)
    return f, h


def dm_server_create(device: int = 0, n_slots: int = 4, mem_budget_bytes: int = 0, max_rows: int = 0,
                     order: int = DM_ORDER_PAPER, motifs=None):
    o = dm_server_opts()
    o.n_slots, o.mem_budget_bytes, o.max_rows, o.order = int(n_slots), int(mem_budget_bytes), int(max_rows), int(order)
    keep = None
    if motifs:
        keep = _arr_i32(list(motifs))
        o.motifs, o.n_motifs = _p32(keep), len(keep)
    h = _vp()
    _check(_lib.dm_server_create(ctypes.byref(h), int(device), ctypes.byref(o)), "dm_server_create")
    return h


def dm_server_load_graph(srv, n_vertices: int, row_ptr, col_idx, edge_err=None, qubit_err=None) -> int:
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    ee = None if edge_err is None else _f32(edge_err)
    qe = None if qubit_err is None else _f32(qubit_err)
    out = _i32()
    _check(_lib.dm_server_load_graph(srv, int(n_vertices), _p32(rp), _p32(ci), None if ee is None else _pf(ee),
                                     None if qe is None else _pf(qe), ctypes.byref(out)), "dm_server_load_graph")
    return out.value


def dm_server_set_model(srv, w) -> None:
    w = _f32(w)
    _check(_lib.dm_server_set_model(srv, _pf(w), len(w)), "dm_server_set_model")


def dm_server_submit(srv, graph: int, n_p: int, row_ptr, col_idx, k: int) -> int:
    rp, ci = _arr_i32(row_ptr), _arr_i32(col_idx)
    rid = _u64()
    _check(_lib.dm_server_submit(srv, int(graph), int(n_p), _p32(rp), _p32(ci), int(k), ctypes.byref(rid)),
           "dm_server_submit")
    return rid.value


def dm_server_wait(srv, rid: int, k: int, n_p: int) -> dict:
    rows = np.zeros((k, n_p), dtype=np.int32)
    scores = np.zeros(k, dtype=np.float32)
    n, st = _i32(), _i32()
    lat, q = ctypes.c_double(), ctypes.c_double()
    _check(_lib.dm_server_wait(srv, int(rid), _p32(rows), _pf(scores), ctypes.byref(n), ctypes.byref(st),
                               ctypes.byref(lat), ctypes.byref(q)), "dm_server_wait")
    return {"rows": rows[:n.value], "scores": scores[:n.value], "status": st.value, "latency_ms": lat.value,
            "queue_ms": q.value}


def dm_server_stats_get(srv) -> dict:
    s = dm_server_stats()
    _check(_lib.dm_server_stats_get(srv, ctypes.byref(s)), "dm_server_stats_get")
    return {f: getattr(s, f) for f, _ in dm_server_stats._fields_}


def dm_server_destroy(srv) -> None:
    _check(_lib.dm_server_destroy(srv), "dm_server_destroy")


def dm_score_topk(ctx, plan, k: int, n_p: int):
    rows = np.zeros((k, n_p), dtype=np.int32)
    scores = np.zeros(k, dtype=np.float32)
    n = _i32()
    _check(_lib.dm_score_topk(ctx, plan, int(k), _p32(rows), scores.ctypes.data_as(_fp), ctypes.byref(n)),
           "dm_score_topk", ctx)
    return rows[:n.value], scores[:n.value]


def dm_load_directed_errors(ctx, graph: int, e_dir) -> None:
    e = _f32(e_dir)
    _check(_lib.dm_load_directed_errors(ctx, int(graph), _pf(e)), "dm_load_directed_errors", ctx)


def dm_score_topk_directed(ctx, plan, w_dir, k: int, n_p: int):
    """k best layouts by the direction-aware score; returns (rows [m, n_p], scores [m])."""
    w = _f32(w_dir)
    rows = np.zeros((k, n_p), dtype=np.int32)
    scores = np.zeros(k, dtype=np.float32)
    n = _i32()
    _check(_lib.dm_score_topk_directed(ctx, plan, _pf(w), int(k), _p32(rows), _pf(scores), ctypes.byref(n)),
           "dm_score_topk_directed", ctx)
    return rows[:n.value], scores[:n.value]


def dm_get_stats(ctx) -> dict:
    s = dm_stats()
    _check(_lib.dm_get_stats(ctx, ctypes.byref(s)), "dm_get_stats", ctx)
    n = s.n_steps
    return {"n_steps": n, "rows": list(s.rows[:n]), "candidates": list(s.candidates[:n]),
            "chunks": s.chunks, "max_rows": s.max_rows, "join_ms": s.join_ms,
            "join_launches": s.join_launches, "join_bytes": s.join_bytes, "total_ms": s.total_ms,
            "kernel_launches": s.kernel_launches}


DM_SORT_STATIC_MAX_ROWS = 1 << 20


def dm_sort_rows_static(rows_in_ptr: int, scores_in_ptr, n: int, w: int, bits: int, rows_out_ptr: int,
                        scores_out_ptr, stream=None) -> None:
    """Sort n x w device rows into rows_out without allocating (raw device pointers, e.g.
    torch's data_ptr()); work is enqueued on `stream` and not waited for. For callers that
    cannot allocate device memory at that point (see include/dm.h)."""
    raw = getattr(stream, "cuda_stream", stream)
    rc = _lib.dm_sort_rows_static(_vp(rows_in_ptr), _vp(scores_in_ptr) if scores_in_ptr else None, int(n), int(w),
                                  int(bits), _vp(rows_out_ptr), _vp(scores_out_ptr) if scores_out_ptr else None,
                                  _vp(raw) if raw else None)
    _check(rc, "dm_sort_rows_static")


def dm_enable_timing(ctx, on: bool = True) -> None:
    _check(_lib.dm_enable_timing(ctx, int(bool(on))), "dm_enable_timing", ctx)


# ------------------------------------------------------------------- convenience ----------
class Context:
    """Owns a dm_ctx; graphs are objects with n, row_ptr, col_idx[, edge_err, qubit_err]."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.h = dm_create(device, mem_budget_bytes)

    def close(self):
        if self.h:
            dm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load(self, g, weights: bool = True, score_form: int = DM_SCORE_ERROR_SUM) -> int:
        return dm_load_data_graph_ex(self.h, g.n, g.row_ptr, g.col_idx,
                                     getattr(g, "edge_err", None) if weights else None,
                                     getattr(g, "qubit_err", None) if weights else None, score_form)

    def plan(self, graph: int, pattern, **kw):
        return Plan(self, dm_plan(self.h, graph, pattern.n, pattern.row_ptr, pattern.col_idx, **kw), pattern.n)

    def motif_table(self, graph: int, motif_id: int) -> np.ndarray:
        return dm_motif_table(self.h, graph, motif_id)

    def stats(self) -> dict:
        return dm_get_stats(self.h)


class Plan:
    def __init__(self, ctx: Context, h, n_p: int):
        self.ctx, self.h, self.n_p = ctx, h, n_p

    def __del__(self):
        if getattr(self, "h", None):
            dm_plan_free(self.h)
            self.h = None

    def describe(self) -> list[dict]:
        return dm_plan_describe(self.h)

    def all(self):
        """All embeddings: (rows [count, n_p] int32 in canonical order, scores or None, count, checksum)."""
        rows, scores = [], []

        def cb(r, s):
            rows.append(r)
            if s is not None:
                scores.append(s)
            return 0

        cnt, cs = dm_match(self.ctx.h, self.h, DM_ALL, cb)
        R = np.concatenate(rows) if rows else np.zeros((0, self.n_p), dtype=np.int32)
        S = np.concatenate(scores) if scores else None
        return R, S, cnt, cs

    def count(self):
        return dm_match(self.ctx.h, self.h, DM_COUNT, None)

    def topk(self, k: int):
        return dm_score_topk(self.ctx.h, self.h, k, self.n_p)
