"""The device-built PR-quadtree leaves (Section 4.1.1) equal the oracle's
level-by-level construction exactly: same sorted object order, same leaves
(level, code, start, count) in Morton order (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import synth
from tests.gpu_util import gpu_tick, make_world

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    ("uniform", 50000, 32, 8, 16),
    ("uniform", 30011, 1, 1, 16),
    ("uniform", 1000, 5000 // 2, 1, 16),
    ("clustered", 100000, 16, 6, 16),
    ("clustered", 100000, 300, 3, 12),
    ("clustered", 20000, 4096, 1, 16),
    ("coincident", 4000, 8, 2, 16),
    ("uniform", 1_000_000, 32, 8, 16),
]


@pytest.mark.parametrize("dist,n,th,G,L", CASES)
def test_leaves_match_oracle(dist, n, th, G, L):
    if dist == "uniform":
        x, y = synth.uniform_positions(n, 1)
    elif dist == "clustered":
        x, y = synth.clustered_positions(n, 2)
    else:
        x = np.full(n, 0.375, np.float32)
        y = np.full(n, 0.625, np.float32)
        x[: n // 2] = 0.125
    world = make_world(x, y, k_max=8, max_depth=L)
    try:
        world.set_tuning(leaf_capacity=th, grid_level=G, packet_level=min(G, 4))
        t = synth.Tick(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                       np.arange(min(n, 100), dtype=np.int32), 4)
        gpu_tick(world, t)
        got = {k: v.cpu().numpy() for k, v in world.leaves().items()}
    finally:
        world.close()
    got["z"] = got["z"].view(np.uint32)   # codes travel as int32 bit patterns
    want = oracle.pr_quadtree(x, y, L, th, min_level=G)
    assert np.array_equal(got["order"], want["order"])
    for key in ("level", "z", "start", "count"):
        assert np.array_equal(got[key].astype(np.int64), want[key].astype(np.int64)), key


@pytest.mark.parametrize("n,L", [(100_000, 12), (1 << 20, 12), ((1 << 20) + 1, 16)])
def test_automatic_depth(n, L):
    # a world created without max_depth takes l_max = 12 up to 2^20 objects and
    # 16 above; its leaves are the oracle's at that depth
    x, y = synth.clustered_positions(n, 6)
    world = make_world(x, y, k_max=8)
    try:
        world.set_tuning(leaf_capacity=16, grid_level=7, packet_level=4)
        t = synth.Tick(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                       np.arange(100, dtype=np.int32), 4)
        gpu_tick(world, t)
        got = {k: v.cpu().numpy() for k, v in world.leaves().items()}
    finally:
        world.close()
    got["z"] = got["z"].view(np.uint32)
    want = oracle.pr_quadtree(x, y, L, 16, min_level=7)
    assert np.array_equal(got["order"], want["order"])
    for key in ("level", "z", "start", "count"):
        assert np.array_equal(got[key].astype(np.int64), want[key].astype(np.int64)), key


@pytest.mark.parametrize("dist,n,th,G", [("clustered", 100000, 16, 8), ("half", 30000, 8, 6)])
def test_reuse_leaves_cover_every_cell(dist, n, th, G):
    # with index reuse on, the leaves are the oracle's plus one empty leaf at
    # level G for every level-G cell without objects, all in Morton order
    L = 16
    if dist == "clustered":
        x, y = synth.clustered_positions(n, 3)
    else:
        x, y = synth.uniform_positions(n, 4)
        x = (x * 0.5).astype(np.float32)
    world = make_world(x, y, k_max=8, max_depth=L)
    try:
        world.set_tuning(leaf_capacity=th, grid_level=G, packet_level=min(G, 4))
        world.set_index_reuse(4)
        t = synth.Tick(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                       np.arange(100, dtype=np.int32), 4)
        gpu_tick(world, t)
        got = {k: v.cpu().numpy() for k, v in world.leaves().items()}
    finally:
        world.close()
    got["z"] = got["z"].view(np.uint32)
    want = oracle.pr_quadtree(x, y, L, th, min_level=G)
    lv, z = want["level"].astype(np.int64), want["z"].astype(np.int64)
    start, count = want["start"].astype(np.int64), want["count"].astype(np.int64)
    cell = z >> (2 * (lv - G))
    empty = np.setdiff1d(np.arange(4 ** G), cell)
    zpp = np.concatenate([z << (2 * (L - lv)), empty << (2 * (L - G))])
    order = np.argsort(zpp, kind="stable")
    e_level = np.concatenate([lv, np.full(empty.size, G)])[order]
    e_z = np.concatenate([z, empty])[order]
    e_count = np.concatenate([count, np.zeros(empty.size, np.int64)])[order]
    # an empty leaf starts where the next non-empty one does (n after the last)
    e_start = np.concatenate([start, np.full(empty.size, -1)])[order]
    nxt = n
    for i in range(e_start.size - 1, -1, -1):
        if e_start[i] < 0:
            e_start[i] = nxt
        else:
            nxt = e_start[i]
    assert empty.size > 0
    assert np.array_equal(got["order"], want["order"])
    for key, val in (("level", e_level), ("z", e_z), ("start", e_start), ("count", e_count)):
        assert np.array_equal(got[key].astype(np.int64), val), key
