"""The C-ABI library loads and exports every symbol the header declares, and
host-side argument validation works without touching a GPU (CPU only)."""
import ctypes

import pytest

from paper_1412_6170_gb300 import build as cuda_build
from paper_1412_6170_gb300 import knnq


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return knnq.lib()


def test_header_symbols_exported(lib):
    names = knnq.header_functions()
    assert "knn_tick" in names and "knn_world_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert all(hasattr(knnq, n) for n in names)


def test_stage_names(lib):
    names = knnq.stage_names()
    assert names[-2:] == ["expand", "pass-on"] and len(names) == 7


def desc(**kw):
    d = dict(x0=0.0, y0=0.0, side=1.0, leaf_capacity=0, max_depth=0, k_max=16, max_queries=10)
    d.update(kw)
    return knnq.knn_world_desc(**d)


@pytest.mark.parametrize("kw,n", [({"side": 0.0}, 10), ({"side": float("nan")}, 10),
                                  ({"k_max": 0}, 10), ({"k_max": 513}, 10),
                                  ({"max_depth": 17}, 10), ({"leaf_capacity": 5000}, 10),
                                  ({"max_queries": -1}, 10), ({}, 0), ({}, 2 ** 30 + 1)])
def test_create_rejects_bad_description(lib, kw, n):
    h = ctypes.c_void_p()
    st = lib.knn_world_create(ctypes.byref(desc(**kw)), 1, 1, n, None, ctypes.byref(h))
    assert st == knnq.KNN_ERR_INVALID
    assert h.value is None
    assert knnq.knn_last_error()


def test_create_rejects_null_positions(lib):
    h = ctypes.c_void_p()
    st = lib.knn_world_create(ctypes.byref(desc()), None, None, 10, None, ctypes.byref(h))
    assert st == knnq.KNN_ERR_INVALID


def test_null_world_calls_are_rejected(lib):
    assert lib.knn_tick(None, None, None, None, 0, None, None, None, 0, 1, None, None,
                        None) == knnq.KNN_ERR_INVALID
    assert lib.knn_world_destroy(None) == knnq.KNN_ERR_INVALID
    assert knnq.knn_tick_status(None)[0] == knnq.KNN_ERR_INVALID
    with pytest.raises(knnq.KnnError) as e:
        knnq.knn_world_set_tuning(None, 1, 1, 1)
    assert e.value.status == knnq.KNN_ERR_INVALID
    assert lib.knn_world_set_host_io(None, 1) == knnq.KNN_ERR_INVALID
    assert lib.knn_world_set_graphs(None, 1) == knnq.KNN_ERR_INVALID
    assert lib.knn_tick_host_wait(None, 0) == knnq.KNN_ERR_INVALID
    t = ctypes.c_int64(0)
    assert lib.knn_tick_host_submit(None, None, None, None, 0, None, None, None, 0, 1, None, None,
                                    None, ctypes.byref(t)) == knnq.KNN_ERR_INVALID
    assert lib.knn_world_test_wait_timeout(None, None) == knnq.KNN_ERR_INVALID
