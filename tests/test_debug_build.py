"""The debug build (-DKNN_DEBUG: device bounds checks that record a failure and
skip the access instead of trapping) compiles for sm_103a and exports every
entry point of include/knn.h (CPU: nvcc cross-compiles, nothing runs)."""
import ctypes

from paper_1412_6170_gb300 import build, knnq


def test_debug_library_builds_and_exports_every_symbol():
    path = build.build_debug()
    lib = ctypes.CDLL(path)
    missing = [f for f in knnq.header_functions() if not hasattr(lib, f)]
    assert not missing, missing
    assert lib.knn_debug_build() == knnq.KNN_OK
