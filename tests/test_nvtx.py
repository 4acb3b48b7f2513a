"""NVTX ranges of the library reach a profiler (CPU): a minimal injection
library (tests/nvtx_record.c, loaded by NVTX through NVTX_INJECTION64_PATH)
records the ranges of a process that makes one library call."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_nvtx_ranges_reach_a_profiler(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    sys.path.insert(0, ROOT)
    from paper_1412_6170_gb300 import build
    build.build()
    include = os.path.join(os.path.dirname(os.path.dirname(build.nvcc())), "include")
    so = tmp_path / "libnvtx_record.so"
    subprocess.run([gcc, "-shared", "-fPIC", "-O1", "-I", include,
                    os.path.join(ROOT, "tests", "nvtx_record.c"), "-o", str(so)], check=True)
    log = tmp_path / "nvtx.log"
    # a call that fails its argument check (no device work): its range is
    # pushed first and popped on return
    code = ("from paper_1412_6170_gb300 import knnq\n"
            "st = knnq.lib().knn_query_static(None, None, None, 0, None, None, None, 0, 1,"
            " None, None, None)\n"
            "assert st == knnq.KNN_ERR_INVALID, st\n")
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), KNNQ_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, check=True)
    lines = log.read_text().splitlines()
    assert "push knnq query_static" in lines, lines
    assert lines.count("pop") == sum(1 for x in lines if x.startswith("push")), lines
