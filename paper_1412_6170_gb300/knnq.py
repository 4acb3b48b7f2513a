"""ctypes binding of the C ABI in ``include/knn.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and takes plain
integers for pointers (``tensor.data_ptr()``) and streams
(``torch.cuda.current_stream().cuda_stream``).  The ``World`` class at the end
is a thin convenience wrapper for torch tensors; all work happens in the CUDA
library.  There is no CPU fallback: importing this module fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
# KNNQ_DEBUG=1 loads the build with device bounds checks (build.build_debug())
LIB_PATH = os.path.join(HERE, "_build_debug" if os.environ.get("KNNQ_DEBUG") == "1" else "_build",
                        "libknnq.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "knn.h")

KNN_OK = 0
KNN_ERR_INVALID = -1
KNN_ERR_OOM = -2
KNN_ERR_CUDA = -3
KNN_ERR_TIMEOUT = -4
KNN_ERR_ADMISSION = -5
KNN_ERR_DEVICE_INPUT = -6

ERR_BAD_UPDATE_ID = 1
ERR_NONFINITE_UPDATE = 2
ERR_BAD_QUERY = 4
ERR_TIMEOUT = 8
ERR_DEBUG_BOUNDS = 16


class KnnError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"knn status {status}: {message}")
        self.status = status
        self.message = message


class knn_world_desc(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("y0", ctypes.c_float), ("side", ctypes.c_float),
                ("leaf_capacity", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("max_queries", ctypes.c_int64)]


class knn_tuning(ctypes.Structure):
    _fields_ = [("leaf_capacity", ctypes.c_int32), ("grid_level", ctypes.c_int32),
                ("packet_level", ctypes.c_int32), ("expansion", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class knn_server_desc(ctypes.Structure):
    _fields_ = [("n_slots", _i32), ("reserved", _i32), ("hbm_budget_bytes", _i64)]


class knn_server_counters(ctypes.Structure):
    _fields_ = [("worlds", _i32), ("resident_worlds", _i32), ("scratch_bytes", _i64),
                ("largest_world_scratch", _i64), ("admitted", _i64), ("completed", _i64),
                ("evictions", _i64), ("pending", _i64)]


class knn_tick_args(ctypes.Structure):
    _fields_ = [("upd_id_dev", _vp), ("upd_x_dev", _vp), ("upd_y_dev", _vp), ("n_upd", _i64),
                ("q_id_dev", _vp), ("q_x_dev", _vp), ("q_y_dev", _vp), ("n_q", _i64),
                ("k", _i32), ("out_ids_dev", _vp), ("out_d2_dev", _vp), ("q_k_dev", _vp)]

_SIGNATURES = {
    "knn_world_create": ([ctypes.POINTER(knn_world_desc), _vp, _vp, _i64, _vp,
                          ctypes.POINTER(_vp)], ctypes.c_int),
    "knn_tick_ex": ([_vp, ctypes.POINTER(knn_tick_args), _vp], ctypes.c_int),
    "knn_tick": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp],
                 ctypes.c_int),
    "knn_tick_host": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp],
                      ctypes.c_int),
    "knn_tick_status": ([_vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "knn_world_destroy": ([_vp], ctypes.c_int),
    "knn_last_error": ([], ctypes.c_char_p),
    "knn_world_set_tuning": ([_vp, ctypes.POINTER(knn_tuning)], ctypes.c_int),
    "knn_world_get_tuning": ([_vp, _i64, _i32, ctypes.POINTER(knn_tuning)], ctypes.c_int),
    "knn_world_leaves": ([_vp, _vp, _vp, _vp, _vp, _vp, _i64, ctypes.POINTER(_i64), _vp],
                         ctypes.c_int),
    "knn_world_positions": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "knn_world_launches": ([_vp, ctypes.POINTER(_i64)], ctypes.c_int),
    "knn_world_set_profiling": ([_vp, _i32], ctypes.c_int),
    "knn_world_set_graphs": ([_vp, _i32], ctypes.c_int),
    "knn_world_set_host_io": ([_vp, _i32], ctypes.c_int),
    "knn_world_test_wait_timeout": ([_vp, _vp], ctypes.c_int),
    "knn_tick_host_submit": ([_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i64, _i32, _vp, _vp,
                              _vp, ctypes.POINTER(_i64)], ctypes.c_int),
    "knn_tick_host_wait": ([_vp, _i64], ctypes.c_int),
    "knn_brute_force": ([_vp, _vp, _i64, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp], ctypes.c_int),
    "knn_world_set_index_reuse": ([_vp, _i32, ctypes.c_float], ctypes.c_int),
    "knn_world_index_info": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)], ctypes.c_int),
    "knn_world_expand_info": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
    "knn_debug_build": ([], ctypes.c_int),
    "knn_world_test_bounds_check": ([_vp, _vp], ctypes.c_int),
    "knn_world_record_tick": ([_vp, ctypes.POINTER(knn_tick_args)], ctypes.c_int),
    "knn_world_stage_times": ([_vp, ctypes.POINTER(ctypes.c_float), _i32], ctypes.c_int),
    "knn_stage_name": ([_i32], ctypes.c_char_p),
    "knn_batch_tick": ([_i32, ctypes.POINTER(_vp), ctypes.POINTER(knn_tick_args), _vp],
                       ctypes.c_int),
    "knn_world_autotune": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _i32,
                            ctypes.POINTER(knn_tuning), _vp], ctypes.c_int),
    "knn_batch_autotune": ([_i32, ctypes.POINTER(_vp), ctypes.POINTER(knn_tick_args), _i32,
                            ctypes.POINTER(knn_tuning), _vp], ctypes.c_int),
    "knn_server_create": ([ctypes.POINTER(knn_server_desc), ctypes.POINTER(_vp)], ctypes.c_int),
    "knn_server_add_world": ([_vp, ctypes.POINTER(knn_world_desc), _vp, _vp, _i64,
                              ctypes.POINTER(_i32)], ctypes.c_int),
    "knn_server_submit": ([_vp, _i32, ctypes.POINTER(knn_tick_args), ctypes.POINTER(_i64)],
                          ctypes.c_int),
    "knn_server_poll": ([_vp, _i64, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)],
                        ctypes.c_int),
    "knn_server_wait": ([_vp, _i64, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "knn_server_stats": ([_vp, ctypes.POINTER(knn_server_counters)], ctypes.c_int),
    "knn_server_world_status": ([_vp, _i32, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "knn_server_destroy": ([_vp], ctypes.c_int),
    "knn_query_static": ([ctypes.POINTER(knn_world_desc), _vp, _vp, _i64, _vp, _vp, _vp, _i64,
                          _i32, _vp, _vp, _vp], ctypes.c_int),
}

_lib = None


def lib():
    """Load ``libknnq.so``; raises when it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_functions(path: str = HEADER) -> list:
    """Names of every function the C header declares."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(knn_[a-z_0-9]+)\s*\(", src)))


def knn_last_error() -> str:
    return lib().knn_last_error().decode()


def _check(st: int) -> None:
    if st != KNN_OK:
        raise KnnError(st, knn_last_error())


def knn_world_create(desc: knn_world_desc, x_dev: int, y_dev: int, n: int,
                     stream: int = 0) -> int:
    h = _vp()
    _check(lib().knn_world_create(ctypes.byref(desc), x_dev, y_dev, n, stream, ctypes.byref(h)))
    return h.value


def knn_tick(w: int, upd_id, upd_x, upd_y, n_upd: int, q_id, q_x, q_y, n_q: int, k: int,
             out_ids, out_d2, stream: int = 0) -> None:
    _check(lib().knn_tick(w, upd_id, upd_x, upd_y, n_upd, q_id, q_x, q_y, n_q, k, out_ids,
                          out_d2, stream))


def knn_tick_host(w: int, upd_id, upd_x, upd_y, n_upd: int, q_id, q_x, q_y, n_q: int, k: int,
                  out_ids, out_d2, stream: int = 0) -> None:
    _check(lib().knn_tick_host(w, upd_id, upd_x, upd_y, n_upd, q_id, q_x, q_y, n_q, k,
                               out_ids, out_d2, stream))


def knn_tick_host_submit(w: int, upd_id, upd_x, upd_y, n_upd: int, q_id, q_x, q_y, n_q: int,
                         k: int, out_ids, out_d2, stream: int = 0) -> int:
    t = _i64(0)
    _check(lib().knn_tick_host_submit(w, upd_id, upd_x, upd_y, n_upd, q_id, q_x, q_y, n_q, k,
                                      out_ids, out_d2, stream, ctypes.byref(t)))
    return t.value


def knn_tick_host_wait(w: int, ticket: int) -> None:
    _check(lib().knn_tick_host_wait(w, ticket))


def knn_tick_status(w: int) -> tuple:
    bits = ctypes.c_uint32(0)
    st = lib().knn_tick_status(w, ctypes.byref(bits))
    return st, bits.value


def knn_world_destroy(w: int) -> None:
    _check(lib().knn_world_destroy(w))


def knn_world_set_tuning(w: int, leaf_capacity=0, grid_level=0, packet_level=0,
                         expansion=0) -> None:
    t = knn_tuning(leaf_capacity, grid_level, packet_level, expansion)
    _check(lib().knn_world_set_tuning(w, ctypes.byref(t)))


def knn_world_get_tuning(w: int, n_q: int, k: int) -> dict:
    t = knn_tuning()
    _check(lib().knn_world_get_tuning(w, n_q, k, ctypes.byref(t)))
    return {"leaf_capacity": t.leaf_capacity, "grid_level": t.grid_level,
            "packet_level": t.packet_level, "expansion": t.expansion}


def knn_world_leaves(w: int, level, z, start, count, sorted_ids, cap: int,
                     stream: int = 0) -> int:
    m = _i64(0)
    _check(lib().knn_world_leaves(w, level, z, start, count, sorted_ids, cap, ctypes.byref(m),
                                  stream))
    return m.value


def knn_world_positions(w: int, x_dev: int, y_dev: int, stream: int = 0) -> None:
    _check(lib().knn_world_positions(w, x_dev, y_dev, stream))


def knn_world_launches(w: int) -> int:
    c = _i64(0)
    _check(lib().knn_world_launches(w, ctypes.byref(c)))
    return c.value


def knn_world_set_profiling(w: int, enable: bool) -> None:
    _check(lib().knn_world_set_profiling(w, 1 if enable else 0))


def knn_world_set_graphs(w: int, enable: bool) -> None:
    _check(lib().knn_world_set_graphs(w, 1 if enable else 0))


def knn_world_set_host_io(w: int, mode: int) -> None:
    _check(lib().knn_world_set_host_io(w, mode))


def knn_world_test_wait_timeout(w: int, stream: int = 0) -> None:
    _check(lib().knn_world_test_wait_timeout(w, stream))


def knn_brute_force(x_dev, y_dev, n: int, q_id_dev, q_x_dev, q_y_dev, n_q: int, k: int,
                    out_ids_dev, out_d2_dev, stream: int = 0) -> None:
    _check(lib().knn_brute_force(x_dev, y_dev, n, q_id_dev, q_x_dev, q_y_dev, n_q, k,
                                 out_ids_dev, out_d2_dev, stream))


def brute_force(x, y, k: int, q_id, q_x=None, q_y=None, stream=None):
    """knn_brute_force on torch tensors; returns (ids, d2) of shape (n_q, k)."""
    import torch
    n_q = int(q_id.shape[0])
    ids = torch.empty((n_q, k), dtype=torch.int32, device=q_id.device)
    d2 = torch.empty((n_q, k), dtype=torch.float32, device=q_id.device)
    knn_brute_force(_ptr(x), _ptr(y), int(x.shape[0]), _ptr(q_id), _ptr(q_x), _ptr(q_y), n_q, k,
                    _ptr(ids), _ptr(d2), _stream(stream))
    return ids, d2


def knn_world_set_index_reuse(w: int, max_age: int, factor: float = 0.0) -> None:
    _check(lib().knn_world_set_index_reuse(w, max_age, factor))


def knn_world_index_info(w: int) -> dict:
    age, rebuilt = _i32(), _i32()
    _check(lib().knn_world_index_info(w, ctypes.byref(age), ctypes.byref(rebuilt)))
    return {"age": age.value, "rebuilt": rebuilt.value}


def knn_world_expand_info(w: int) -> dict:
    gathered, back = _i64(0), _i64(0)
    _check(lib().knn_world_expand_info(w, ctypes.byref(gathered), ctypes.byref(back)))
    return {"gathered": int(gathered.value), "handed_back": int(back.value)}


def knn_debug_build() -> bool:
    """True when the loaded library was built with device bounds checks."""
    return lib().knn_debug_build() == KNN_OK


def knn_world_test_bounds_check(w: int, stream: int = 0) -> None:
    _check(lib().knn_world_test_bounds_check(w, stream))


def knn_world_record_tick(w: int, args: knn_tick_args) -> None:
    _check(lib().knn_world_record_tick(w, ctypes.byref(args)))


def knn_world_stage_times(w: int, n: int = 16) -> list:
    buf = (ctypes.c_float * n)()
    _check(lib().knn_world_stage_times(w, buf, n))
    return list(buf)


def knn_stage_name(i: int) -> Optional[str]:
    s = lib().knn_stage_name(i)
    return None if s is None else s.decode()


def stage_names() -> list:
    out, i = [], 0
    while True:
        s = knn_stage_name(i)
        if s is None:
            return out
        out.append(s)
        i += 1


def knn_batch_tick(worlds, args, stream: int = 0) -> None:
    """One tick of every world in ``worlds`` (handles) with ``args`` (knn_tick_args),
    recorded into and launched as one CUDA graph."""
    n = len(worlds)
    wa = (_vp * n)(*worlds)
    aa = (knn_tick_args * n)(*args)
    _check(lib().knn_batch_tick(n, wa, aa, stream))


def knn_world_autotune(w: int, q_id, q_x, q_y, n_q: int, k: int, out_ids, out_d2,
                       trials: int = 2, stream: int = 0) -> dict:
    t = knn_tuning()
    _check(lib().knn_world_autotune(w, q_id, q_x, q_y, n_q, k, out_ids, out_d2, trials,
                                    ctypes.byref(t), stream))
    return {"leaf_capacity": t.leaf_capacity, "grid_level": t.grid_level,
            "packet_level": t.packet_level, "expansion": t.expansion}


def knn_batch_autotune(worlds, args, trials: int = 2, stream: int = 0) -> list:
    """Settings for the batch's worlds chosen by timing whole batch ticks; returns
    one tuning dict per world (the settings stay in the worlds)."""
    n = len(worlds)
    wa = (_vp * n)(*worlds)
    aa = (knn_tick_args * n)(*args)
    ts = (knn_tuning * n)()
    _check(lib().knn_batch_autotune(n, wa, aa, trials, ts, stream))
    return [{"leaf_capacity": t.leaf_capacity, "grid_level": t.grid_level,
             "packet_level": t.packet_level, "expansion": t.expansion} for t in ts]


def tick_args(k: int, q_id=None, upd_id=None, upd_x=None, upd_y=None, q_x=None, q_y=None,
              out_ids=None, out_d2=None, q_k=None) -> knn_tick_args:
    """knn_tick_args from torch tensors (or None); q_k: per-query list sizes."""
    return knn_tick_args(_ptr(upd_id), _ptr(upd_x), _ptr(upd_y),
                         0 if upd_id is None else int(upd_id.shape[0]), _ptr(q_id), _ptr(q_x),
                         _ptr(q_y), 0 if q_id is None else int(q_id.shape[0]), k,
                         _ptr(out_ids), _ptr(out_d2), _ptr(q_k))


def knn_tick_ex(w: int, args: knn_tick_args, stream: int = 0) -> None:
    _check(lib().knn_tick_ex(w, ctypes.byref(args), stream))


def knn_server_create(n_slots: int = 4, hbm_budget_bytes: int = 0) -> int:
    h = _vp()
    d = knn_server_desc(n_slots, 0, hbm_budget_bytes)
    _check(lib().knn_server_create(ctypes.byref(d), ctypes.byref(h)))
    return h.value


def knn_server_add_world(s: int, desc: knn_world_desc, x_dev: int, y_dev: int, n: int) -> int:
    idx = _i32(0)
    _check(lib().knn_server_add_world(s, ctypes.byref(desc), x_dev, y_dev, n, ctypes.byref(idx)))
    return idx.value


def knn_server_submit(s: int, world_index: int, args: knn_tick_args) -> int:
    rid = _i64(0)
    _check(lib().knn_server_submit(s, world_index, ctypes.byref(args), ctypes.byref(rid)))
    return rid.value


def knn_server_poll(s: int, request_id: int) -> tuple:
    st = _i32(0)
    lat = ctypes.c_double(0.0)
    _check(lib().knn_server_poll(s, request_id, ctypes.byref(st), ctypes.byref(lat)))
    return st.value, lat.value


def knn_server_wait(s: int, request_id: int) -> float:
    lat = ctypes.c_double(0.0)
    _check(lib().knn_server_wait(s, request_id, ctypes.byref(lat)))
    return lat.value


def knn_server_stats(s: int) -> dict:
    c = knn_server_counters()
    _check(lib().knn_server_stats(s, ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in knn_server_counters._fields_}


def knn_server_world_status(s: int, world_index: int) -> tuple:
    bits = ctypes.c_uint32(0)
    st = lib().knn_server_world_status(s, world_index, ctypes.byref(bits))
    return st, bits.value


def knn_server_destroy(s: int) -> None:
    _check(lib().knn_server_destroy(s))


def knn_query_static(desc: knn_world_desc, x_dev, y_dev, n: int, q_id, q_x, q_y, n_q: int,
                     k: int, out_ids, out_d2, stream: int = 0) -> None:
    """One-shot k-NN that allocates nothing (scratch in a static device array;
    n, n_q <= 65536).  For callers that must not call cudaMalloc."""
    _check(lib().knn_query_static(ctypes.byref(desc), x_dev, y_dev, n, q_id, q_x, q_y, n_q, k,
                                  out_ids, out_d2, stream))


# ---------------------------------------------------------------------------
# torch convenience wrapper (device memory and streams only)

def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class World:
    """A world of moving objects resident on the current GPU."""

    def __init__(self, x, y, k_max: int = 64, max_queries: Optional[int] = None,
                 domain=(0.0, 0.0, 1.0), leaf_capacity: int = 0, max_depth: int = 0,
                 stream=None):
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and y.dtype == torch.float32
        x = x.contiguous()
        y = y.contiguous()
        self.n = int(x.shape[0])
        self.k_max = k_max
        self.max_queries = self.n if max_queries is None else int(max_queries)
        desc = knn_world_desc(domain[0], domain[1], domain[2], leaf_capacity, max_depth, k_max,
                              self.max_queries)
        self.handle = knn_world_create(desc, x.data_ptr(), y.data_ptr(), self.n,
                                       _stream(stream))
        self.device = x.device

    def close(self):
        if getattr(self, "handle", None):
            knn_world_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def tick(self, k: int, q_id=None, upd_id=None, upd_x=None, upd_y=None, q_x=None, q_y=None,
             out_ids=None, out_d2=None, stream=None, q_k=None):
        """One tick; q_k (optional int32 tensor of n_q list sizes in [0, k]) asks
        query i for its q_k[i] nearest objects (the rest of its row is padding)."""
        import torch
        n_upd = 0 if upd_id is None else int(upd_id.shape[0])
        n_q = 0 if q_id is None else int(q_id.shape[0])
        if n_q and out_ids is None:
            out_ids = torch.empty((n_q, k), dtype=torch.int32, device=self.device)
            out_d2 = torch.empty((n_q, k), dtype=torch.float32, device=self.device)
        if q_k is None:
            knn_tick(self.handle, _ptr(upd_id), _ptr(upd_x), _ptr(upd_y), n_upd, _ptr(q_id),
                     _ptr(q_x), _ptr(q_y), n_q, k, _ptr(out_ids), _ptr(out_d2),
                     _stream(stream))
        else:
            knn_tick_ex(self.handle, tick_args(k, q_id, upd_id, upd_x, upd_y, q_x, q_y, out_ids,
                                               out_d2, q_k), _stream(stream))
        return out_ids, out_d2

    def status(self):
        return knn_tick_status(self.handle)

    def set_tuning(self, leaf_capacity=0, grid_level=0, packet_level=0, expansion=0):
        knn_world_set_tuning(self.handle, leaf_capacity, grid_level, packet_level, expansion)

    def get_tuning(self, n_q: int, k: int) -> dict:
        return knn_world_get_tuning(self.handle, n_q, k)

    def leaves(self, stream=None):
        import torch
        m = knn_world_leaves(self.handle, None, None, None, None, None, 0, _stream(stream))
        dev = self.device
        level = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        z = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        start = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        count = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        order = torch.empty(self.n, dtype=torch.int32, device=dev)
        knn_world_leaves(self.handle, level.data_ptr(), z.data_ptr(), start.data_ptr(),
                         count.data_ptr(), order.data_ptr(), m, _stream(stream))
        return {"level": level[:m], "z": z[:m], "start": start[:m], "count": count[:m],
                "order": order}

    def positions(self, stream=None):
        import torch
        x = torch.empty(self.n, dtype=torch.float32, device=self.device)
        y = torch.empty(self.n, dtype=torch.float32, device=self.device)
        knn_world_positions(self.handle, x.data_ptr(), y.data_ptr(), _stream(stream))
        return x, y

    def autotune(self, k: int, q_id, q_x=None, q_y=None, trials: int = 2, stream=None) -> dict:
        import torch
        n_q = int(q_id.shape[0])
        oi = torch.empty((max(n_q, 1), k), dtype=torch.int32, device=self.device)
        od = torch.empty((max(n_q, 1), k), dtype=torch.float32, device=self.device)
        return knn_world_autotune(self.handle, _ptr(q_id), _ptr(q_x), _ptr(q_y), n_q, k,
                                  oi.data_ptr(), od.data_ptr(), trials, _stream(stream))

    def launches(self) -> int:
        return knn_world_launches(self.handle)

    def set_profiling(self, enable: bool = True):
        knn_world_set_profiling(self.handle, enable)

    def set_graphs(self, enable: bool = True):
        knn_world_set_graphs(self.handle, enable)

    def test_wait_timeout(self, stream=None):
        """Run one bounded device wait that runs out (see knn_world_test_wait_timeout)."""
        knn_world_test_wait_timeout(self.handle, _stream(stream))

    def set_host_io(self, write_rows: bool = True, read_inputs: bool = False):
        """How tick_host uses pinned host arrays in place (see knn_world_set_host_io)."""
        knn_world_set_host_io(self.handle, (1 if write_rows else 0) | (2 if read_inputs else 0))

    def set_index_reuse(self, max_age: int, factor: float = 0.0):
        knn_world_set_index_reuse(self.handle, max_age, factor)

    def index_info(self) -> dict:
        return knn_world_index_info(self.handle)

    def expand_info(self) -> dict:
        return knn_world_expand_info(self.handle)

    def record_tick(self, k: int, q_id=None, upd_id=None, upd_x=None, upd_y=None, q_x=None,
                    q_y=None, out_ids=None, out_d2=None):
        """Record (without running) the graph that tick() with these tensors replays."""
        knn_world_record_tick(self.handle, tick_args(k, q_id, upd_id, upd_x, upd_y, q_x, q_y,
                                                     out_ids, out_d2))

    def stage_times(self) -> dict:
        names = stage_names()
        ms = knn_world_stage_times(self.handle, len(names))
        return dict(zip(names, ms))
