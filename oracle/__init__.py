"""CPU oracle for repeated k-NN over moving objects -- TEST INFRASTRUCTURE.

Plain, slow, obviously correct restatements of what the per-tick hot path
computes, written from the paper (Def. 1 and Section 2.2 for the k-NN result
and update semantics, Section 4.1.1 for Morton codes and the PR-quadtree).
Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may use this package.  It shares no code with the CUDA library.

The arithmetic lives in C (``knn_oracle.c``, ``quadtree_oracle.c``) compiled
with ``-ffp-contract=off``; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import build as _build

_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_apply_updates.restype = ctypes.c_int64
        L.oracle_apply_updates.argtypes = [ctypes.c_int64, _f32p, _f32p, ctypes.c_int64,
                                           _i32p, _f32p, _f32p]
        L.oracle_sqdist.restype = ctypes.c_float
        L.oracle_sqdist.argtypes = [ctypes.c_float] * 4
        L.oracle_knn.restype = ctypes.c_int64
        L.oracle_knn.argtypes = [ctypes.c_int64, _f32p, _f32p, ctypes.c_int64, _i32p, _f32p,
                                 _f32p, ctypes.c_int32, _i32p, _f32p, ctypes.c_int]
        L.oracle_morton_key.restype = ctypes.c_uint32
        L.oracle_morton_key.argtypes = [ctypes.c_float] * 5 + [ctypes.c_int]
        L.oracle_pr_quadtree.restype = ctypes.c_int64
        L.oracle_pr_quadtree.argtypes = [ctypes.c_int64, _f32p, _f32p, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_int,
                                         ctypes.c_int32, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int64, _i32p, _u32p, _i32p, _i32p, _i32p]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray], typ):
    if a is None:
        return None
    return a.ctypes.data_as(typ)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def apply_updates(x: np.ndarray, y: np.ndarray, upd_id, upd_x, upd_y):
    """Section 2.2: apply one tick's updates in array order (last one wins).

    Returns new (x, y) arrays and the number of skipped (invalid) entries."""
    x = _f32(x).copy()
    y = _f32(y).copy()
    uid, ux, uy = _i32(upd_id), _f32(upd_x), _f32(upd_y)
    bad = lib().oracle_apply_updates(x.shape[0], _p(x, _f32p), _p(y, _f32p), uid.shape[0],
                                     _p(uid, _i32p), _p(ux, _f32p), _p(uy, _f32p))
    return x, y, int(bad)


def sqdist(qx: float, qy: float, px: float, py: float) -> float:
    return float(lib().oracle_sqdist(qx, qy, px, py))


def knn(x, y, q_id, k: int, q_x=None, q_y=None, n_threads: int = 0):
    """Def. 1 with (distance, id) tie-breaking; returns (ids[nq,k] int32, d2[nq,k] float32,
    number of invalid queries)."""
    x, y, qid = _f32(x), _f32(y), _i32(q_id)
    qx = None if q_x is None else _f32(q_x)
    qy = None if q_y is None else _f32(q_y)
    nq = qid.shape[0]
    ids = np.empty((nq, k), np.int32)
    d2 = np.empty((nq, k), np.float32)
    bad = lib().oracle_knn(x.shape[0], _p(x, _f32p), _p(y, _f32p), nq, _p(qid, _i32p),
                           _p(qx, _f32p), _p(qy, _f32p), k, _p(ids, _i32p), _p(d2, _f32p),
                           int(n_threads))
    if bad < 0:
        raise ValueError("oracle_knn: invalid arguments")
    return ids, d2, int(bad)


def morton_key(x: float, y: float, L: int, x0: float = 0.0, y0: float = 0.0,
               scale: Optional[float] = None) -> int:
    if scale is None:
        scale = float(np.float32(2.0 ** L))
    return int(lib().oracle_morton_key(x, y, x0, y0, scale, L))


def pr_quadtree(x, y, L: int, th: int, min_level: int = 0, emit_empty: bool = False,
                x0: float = 0.0, y0: float = 0.0, scale: Optional[float] = None):
    """Section 4.1.1 PR-quadtree leaves in Morton (z'') order.

    Returns dict with level, z, start, count arrays and the sorted object order."""
    x, y = _f32(x), _f32(y)
    n = x.shape[0]
    if scale is None:
        scale = float(np.float32(2.0 ** L))
    cap = max(16, 4 * n + 4 * (4 ** min(min_level, 10)) + 16)
    lv = np.empty(cap, np.int32)
    z = np.empty(cap, np.uint32)
    st = np.empty(cap, np.int32)
    ct = np.empty(cap, np.int32)
    order = np.empty(max(n, 1), np.int32)
    m = lib().oracle_pr_quadtree(n, _p(x, _f32p), _p(y, _f32p), x0, y0, scale, L, th,
                                 min_level, 1 if emit_empty else 0, cap, _p(lv, _i32p),
                                 _p(z, _u32p), _p(st, _i32p), _p(ct, _i32p),
                                 _p(order, _i32p))
    if m < 0:
        raise RuntimeError(f"pr_quadtree: capacity {cap} too small, need {-m}")
    return {"level": lv[:m].copy(), "z": z[:m].copy(), "start": st[:m].copy(),
            "count": ct[:m].copy(), "order": order[:n].copy()}


def run_ticks(x0, y0, ticks, n_threads: int = 0, sample=None):
    """Replay a sequence of ticks (objects with .upd_id/.upd_x/.upd_y/.q_id/.q_x/.q_y/.k)
    and return the per-tick (ids, d2).  ``sample`` (an index array) restricts each
    tick's queries to those rows."""
    x, y = _f32(x0).copy(), _f32(y0).copy()
    out = []
    for t in ticks:
        x, y, _ = apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
        qid = t.q_id if sample is None else t.q_id[sample]
        qx = None if t.q_x is None else (t.q_x if sample is None else t.q_x[sample])
        qy = None if t.q_y is None else (t.q_y if sample is None else t.q_y[sample])
        ids, d2, _ = knn(x, y, qid, t.k, qx, qy, n_threads)
        out.append((ids, d2))
    return out


def available() -> bool:
    try:
        lib()
        return True
    except Exception:  # noqa: BLE001
        return False


__all__ = ["apply_updates", "sqdist", "knn", "morton_key", "pr_quadtree", "run_ticks",
           "available", "lib"]

