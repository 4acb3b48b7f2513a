"""The debug build on the GPU: ticks through the build with device bounds
checks give the oracle's rows and raise no bounds bit; a check that fails on
purpose (an index one past the objects, the access skipped) is reported by
knn_tick_status as error bit 16 and the world stays usable.  Runs in a child
process, which loads the debug library (KNNQ_DEBUG=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle
from paper_1412_6170_gb300 import build, knnq, synth
build.build_debug()
assert knnq.knn_debug_build()
dev = torch.device("cuda:0")
for k, expansion in ((16, 0), (8, 1), (40, 0)):
    w = synth.skewed_moving(n=30000, k=k, ticks=1, seed=61, query_frac=0.5)
    t = w.ticks[0]
    world = knnq.World(torch.from_numpy(w.x0).to(dev), torch.from_numpy(w.y0).to(dev), k_max=64,
                       max_queries=t.q_id.shape[0])
    world.set_tuning(expansion=expansion)
    ids, d2 = world.tick(k, torch.from_numpy(t.q_id).to(dev), torch.from_numpy(t.upd_id).to(dev),
                         torch.from_numpy(t.upd_x).to(dev), torch.from_numpy(t.upd_y).to(dev))
    torch.cuda.synchronize()
    rows = np.arange(0, t.q_id.shape[0], 7)
    rid, rd2, _ = oracle.knn(t.upd_x, t.upd_y, t.q_id[rows], k)
    assert np.array_equal(ids.cpu().numpy()[rows], rid), k
    assert np.array_equal(d2.cpu().numpy()[rows].view(np.uint32), rd2.view(np.uint32)), k
    st, bits = world.status()
    assert st == knnq.KNN_OK and bits == 0, (k, st, bits)
    # one failing check on purpose: reported, and the next tick is clean
    knnq.knn_world_test_bounds_check(world.handle, torch.cuda.current_stream().cuda_stream)
    st, bits = world.status()
    assert st == knnq.KNN_ERR_CUDA and bits & knnq.ERR_DEBUG_BOUNDS, (st, bits)
    ids2, d22 = world.tick(k, torch.from_numpy(t.q_id).to(dev))
    torch.cuda.synchronize()
    assert np.array_equal(ids2.cpu().numpy(), ids.cpu().numpy())
    assert world.status() == (knnq.KNN_OK, 0)
    world.close()
print("debug ok")
'''


def test_debug_build_ticks_match_oracle_and_report_a_failed_check():
    env = dict(os.environ, KNNQ_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "debug ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
