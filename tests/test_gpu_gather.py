"""The gathered form of the expansion (each packet fixes its search box from
the local density, gathers the box's useful leaves and objects in one pass and
tests them in one loop) against the CPU oracle and against the packet walk
(GPU).  Bit-exact throughout: ids equal, squared distances equal as binary32
bit patterns.  Besides the rows, these tests check that the gathered form
really finishes the packets (knn_world_expand_info), since rows stay exact
even when every packet is handed back to the packet walk."""
import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import knnq, synth
from tests.gpu_util import (assert_rows_equal, gpu_tick, make_world, oracle_rows, sample_rows,
                            to_dev, torch_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def ticks_vs_oracle(w, tuning=None, sample=None, k_max=64, what=""):
    """Every tick of ``w`` with the gathered form (unless ``tuning`` says otherwise)
    against the oracle; returns the expand_info of each tick."""
    world = make_world(w.x0, w.y0, k_max=k_max,
                       max_queries=max(t.q_id.shape[0] for t in w.ticks))
    infos = []
    try:
        world.set_tuning(**(tuning or dict(expansion=4)))
        x, y = w.x0.copy(), w.y0.copy()
        for ti, t in enumerate(w.ticks):
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            ids, d2 = gpu_tick(world, t)
            infos.append(world.expand_info())
            rows = np.arange(t.q_id.shape[0]) if sample is None else \
                sample_rows(t.q_id.shape[0], sample, seed=ti)
            rid, rd2 = oracle_rows(x, y, t, rows)
            assert_rows_equal(ids, d2, rid, rd2, rows, what=f"{what} tick {ti}")
        st, bits = world.status()
        assert st == knnq.KNN_OK, (st, bits)
    finally:
        world.close()
    return infos


def test_gather_serves_the_uniform_workload():
    # 200k uniform objects, all querying, k = 16: the gathered form finishes
    # nearly every packet
    w = synth.plain_uniform_moving(n=200_000, k=16, ticks=2, seed=31)
    infos = ticks_vs_oracle(w, sample=12000, k_max=16, what="200k uniform k=16")
    packets = 200_000 // 32
    for info in infos:
        assert info["gathered"] >= packets - packets // 100, info
        assert info["handed_back"] <= packets // 100, info


@pytest.mark.parametrize("k", [1, 4, 8, 16, 32, 48, 64])
def test_gather_clustered_subset_full(k):
    # dense hotspots with deep leaves and a sparse background; every row
    # against the oracle
    w = synth.skewed_moving(n=50_000, k=k, ticks=2, seed=32, query_frac=0.4)
    infos = ticks_vs_oracle(w, what=f"50k clustered k={k}")
    assert all(i["gathered"] > 20 * i["handed_back"] for i in infos), infos


@pytest.mark.parametrize("k", [5, 16])
def test_gather_and_walk_give_identical_rows(k):
    # the same ticks with the gathered form (expansion 4) and with the packet
    # walk only (expansion 1): identical rows, tick by tick
    w = synth.skewed_moving(n=30_000, k=k, ticks=2, seed=33, query_frac=0.7)
    nq = max(t.q_id.shape[0] for t in w.ticks)
    rows = {}
    for expansion in (4, 1):
        world = make_world(w.x0, w.y0, k_max=32, max_queries=nq)
        try:
            world.set_tuning(expansion=expansion)
            rows[expansion] = [gpu_tick(world, t) for t in w.ticks]
            info = world.expand_info()
            if expansion == 1:
                assert info == {"gathered": 0, "handed_back": 0}, info
        finally:
            world.close()
    for (a_ids, a_d2), (b_ids, b_d2) in zip(rows[4], rows[1]):
        assert_rows_equal(a_ids, a_d2, b_ids, b_d2, what=f"gathered vs walk k={k}")


def test_gather_dense_hotspot():
    # one very tight hotspot: its level-G cells hold hundreds of small leaves,
    # so the gathered leaves are culled by their boxes
    n = 40_000
    r = np.random.default_rng(34)
    x = np.clip(r.normal(0.3, 0.002, n), 0, 1 - 2 ** -24).astype(np.float32)
    y = np.clip(r.normal(0.6, 0.002, n), 0, 1 - 2 ** -24).astype(np.float32)
    bg = r.random(n) < 0.2
    x[bg] = r.random(bg.sum()).astype(np.float32)
    y[bg] = r.random(bg.sum()).astype(np.float32)
    ids = np.arange(n, dtype=np.int32)
    uid = np.zeros(0, np.int32)
    uf = np.zeros(0, np.float32)
    w = synth.Workload("hotspot", n, 8, x, y, [synth.Tick(uid, uf, uf, ids, 8)])
    infos = ticks_vs_oracle(w, what="tight hotspot k=8")
    assert infos[0]["gathered"] > 10 * infos[0]["handed_back"], infos


def test_gather_small_and_degenerate_worlds():
    # fewer objects than k, a single object, all coincident, lattice ties: the
    # gathered form finishes or hands back, the rows stay exact either way
    cases = []
    for n, k in ((1, 4), (3, 8), (17, 16), (33, 32)):
        x, y = synth.uniform_positions(n, 35 + n)
        cases.append((x, y, k))
    cases.append((np.full(50, 0.25, np.float32), np.full(50, 0.75, np.float32), 8))
    g = np.arange(32, dtype=np.float32) / 64
    lx, ly = np.meshgrid(g, g)
    cases.append((lx.ravel().astype(np.float32), ly.ravel().astype(np.float32), 12))
    for x, y, k in cases:
        n = len(x)
        ids = np.arange(n, dtype=np.int32)
        uid = np.zeros(0, np.int32)
        uf = np.zeros(0, np.float32)
        w = synth.Workload("small", n, k, x, y, [synth.Tick(uid, uf, uf, ids, k)])
        ticks_vs_oracle(w, k_max=32, tuning=dict(expansion=4), what=f"n={n} k={k}")


def test_gather_explicit_centres_outside_domain_and_per_query_k():
    torch, dev = torch_dev()
    w = synth.skewed_moving(n=20_000, k=16, ticks=1, seed=36, query_frac=0.5)
    t = w.ticks[0]
    nq = t.q_id.shape[0]
    r = np.random.default_rng(37)
    qx = np.clip(r.normal(0.5, 0.4, nq), -0.5, 1.5).astype(np.float32)
    qy = np.clip(r.normal(0.5, 0.4, nq), -0.5, 1.5).astype(np.float32)
    qid = np.where(r.random(nq) < 0.3, -1, t.q_id).astype(np.int32)
    w.ticks[0] = synth.Tick(t.upd_id, t.upd_x, t.upd_y, qid, 16, qx, qy)
    ticks_vs_oracle(w, k_max=16, what="explicit centres")
    # per-query list sizes: query i gets its q_k[i] nearest, then padding
    x, y, _ = oracle.apply_updates(w.x0, w.y0, t.upd_id, t.upd_x, t.upd_y)
    world = make_world(w.x0, w.y0, k_max=16, max_queries=nq)
    try:
        world.set_tuning(expansion=4)
        qk = r.integers(0, 17, nq).astype(np.int32)
        ids, d2 = world.tick(16, to_dev(t.q_id), to_dev(t.upd_id), to_dev(t.upd_x),
                             to_dev(t.upd_y), q_k=to_dev(qk))
        torch.cuda.synchronize()
        ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
        rid, rd2, _ = oracle.knn(x, y, t.q_id, 16)
        keep = np.arange(16)[None, :] < qk[:, None]
        rid = np.where(keep, rid, -1).astype(np.int32)
        rd2 = np.where(keep, rd2, np.float32(np.inf)).astype(np.float32)
        assert_rows_equal(ids, d2, rid, rd2, what="per-query k, gathered")
        assert world.expand_info()["gathered"] > 0
    finally:
        world.close()
