"""The tiled form of the expansion (one block per level-Gp cell of the sorted
queries stages the objects around it once; each lane scans its own search
box with 32-bit selection keys) against the CPU oracle (GPU).  Bit-exact
throughout: ids equal, squared distances equal as binary32 bit patterns.
Besides the rows, these tests check how many packets the tiled form passed on
to the gathered form (knn_world_expand_info counts them as "gathered"), since
rows stay exact even when every packet is passed on."""
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


def ticks_vs_oracle(w, tuning=None, sample=None, k_max=32, what=""):
    """Every tick of ``w`` with the tiled form (unless ``tuning`` says otherwise)
    against the oracle; returns the expand_info of each tick."""
    world = make_world(w.x0, w.y0, k_max=k_max,
                       max_queries=max(t.q_id.shape[0] for t in w.ticks))
    infos = []
    try:
        world.set_tuning(**(tuning or dict(expansion=5)))
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


def passed_on(info):
    return info["gathered"] + info["handed_back"]


def test_tile_is_the_automatic_form_up_to_k_32():
    torch, dev = torch_dev()
    x, y = synth.uniform_positions(20_000, seed=40)
    world = make_world(x, y, k_max=64)
    try:
        for k, form in ((1, 5), (8, 5), (9, 5), (16, 5), (32, 5), (33, 2)):
            assert world.get_tuning(20_000, k)["expansion"] == form, k
    finally:
        world.close()


def test_tile_serves_the_uniform_workload():
    # 200k uniform objects, all querying, k = 16: the tiled form finishes
    # nearly every packet itself
    w = synth.plain_uniform_moving(n=200_000, k=16, ticks=2, seed=41)
    infos = ticks_vs_oracle(w, sample=12000, k_max=16, what="200k uniform k=16")
    packets = 200_000 // 32
    for info in infos:
        assert passed_on(info) <= packets // 50, info


@pytest.mark.parametrize("k", [1, 4, 8, 9, 12, 16, 20, 31, 32])
def test_tile_uniform_every_row(k):
    w = synth.plain_uniform_moving(n=30_000, k=k, ticks=2, seed=42 + k)
    infos = ticks_vs_oracle(w, what=f"30k uniform k={k}")
    assert all(passed_on(i) <= 30_000 // 32 // 10 for i in infos), infos


@pytest.mark.parametrize("k", [12, 16, 32])
def test_tile_clustered_every_row(k):
    # dense hotspots (tiles too full to stage go on to the gathered form) and
    # a sparse background; a fraction of the objects querying
    w = synth.skewed_moving(n=60_000, k=k, ticks=2, seed=43, query_frac=0.4)
    ticks_vs_oracle(w, what=f"60k clustered k={k}")


def test_tile_all_querying_clustered_every_row():
    w = synth.skewed_moving(n=40_000, k=16, ticks=2, seed=44, query_frac=1.0)
    ticks_vs_oracle(w, what="40k clustered all querying k=16")


def test_tile_ties_go_on_and_stay_exact():
    # a lattice: many equal distances (equal codes), plus exact duplicates of
    # positions; the packets with ties go on to the gathered form
    g = np.arange(120, dtype=np.float32) / np.float32(120)
    gx, gy = np.meshgrid(g, g)
    x = gx.ravel().astype(np.float32)
    y = gy.ravel().astype(np.float32)
    x[::7] = x[3]
    y[::7] = y[3]
    w = synth.Workload("lattice", x.size, 16, x, y,
                       [synth.Tick(*synth._empty_updates(), np.arange(x.size, dtype=np.int32), 16)])
    infos = ticks_vs_oracle(w, k_max=16, what="lattice with duplicates k=16")
    assert passed_on(infos[0]) > 0, infos


def test_tile_repeated_and_subset_queries():
    # queries at issuers in any order, some issuers several times
    n = 25_000
    x, y = synth.uniform_positions(n, seed=45)
    r = np.random.default_rng(46)
    q = r.integers(0, n, 30_000).astype(np.int32)
    w = synth.Workload("repeated issuers", n, 16, x, y, [synth.Tick(*synth._empty_updates(), q, 16)])
    ticks_vs_oracle(w, k_max=16, what="repeated issuers k=16")


def test_tile_per_query_k_rows_are_prefixes():
    torch, dev = torch_dev()
    n = 30_000
    x, y = synth.uniform_positions(n, seed=47)
    q = np.arange(n, dtype=np.int32)
    r = np.random.default_rng(48)
    qk = r.integers(0, 17, n).astype(np.int32)
    world = make_world(x, y, k_max=16, max_queries=n)
    try:
        world.set_tuning(expansion=5)
        ids, d2 = world.tick(16, to_dev(q), q_k=to_dev(qk))
        torch.cuda.synchronize()
        ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
    finally:
        world.close()
    rid, rd2, _ = oracle.knn(x, y, q, 16)
    keep = np.arange(16)[None, :] < qk[:, None]
    rid = np.where(keep, rid, -1).astype(np.int32)
    rd2 = np.where(keep, rd2, np.float32(np.inf)).astype(np.float32)
    assert_rows_equal(ids, d2, rid, rd2, what="per-query k, tiled")


def test_tile_matches_gathered_and_walk_on_moving_ticks():
    # the same ticks with the tiled, gathered and walk forms: identical rows
    w = synth.plain_uniform_moving(n=50_000, k=16, ticks=3, seed=49)
    rows = {}
    for expansion in (5, 4, 1):
        world = make_world(w.x0, w.y0, k_max=16, max_queries=50_000)
        try:
            world.set_tuning(expansion=expansion)
            rows[expansion] = [gpu_tick(world, t) for t in w.ticks]
        finally:
            world.close()
    for ti in range(len(w.ticks)):
        for e in (4, 1):
            assert np.array_equal(rows[5][ti][0], rows[e][ti][0]), (ti, e)
            assert np.array_equal(rows[5][ti][1].view(np.uint32),
                                  rows[e][ti][1].view(np.uint32)), (ti, e)


def test_tile_headline_size_sampled_rows():
    # 1M uniform objects, all querying, k = 16 (the headline workload) in the
    # launch configuration the benchmark times: sampled rows against the oracle
    w = synth.plain_uniform_moving(n=1_000_000, k=16, ticks=2, seed=50)
    infos = ticks_vs_oracle(w, sample=6000, k_max=16, tuning=dict(expansion=0),
                            what="1M uniform k=16")
    for info in infos:
        assert passed_on(info) <= 1_000_000 // 32 // 50, info


def test_tile_batch_every_row_and_tiles_used():
    # knn_batch_tick over worlds of several sizes and list sizes, uniform and
    # clustered, one with explicit centres (no tiles): every row against the
    # oracle, twice (the second call replays the recorded batch); the uniform
    # worlds' tiles finish nearly all their packets (the batched tile grid ran)
    torch, dev = torch_dev()
    specs = [(3_000, 4, "u"), (20_000, 8, "u"), (60_000, 16, "u"), (45_000, 32, "u"),
             (30_000, 16, "c"), (25_000, 12, "u"), (15_000, 16, "x")]
    worlds, bufs, pos = [], [], []
    try:
        for si, (n, k, kind) in enumerate(specs):
            if kind == "c":
                x, y = synth.clustered_positions(n, seed=60 + si)
            else:
                x, y = synth.uniform_positions(n, seed=60 + si)
            worlds.append(knnq.World(to_dev(x), to_dev(y), k_max=32, max_queries=n))
            q = np.arange(n, dtype=np.int32)
            b = {"q": to_dev(q),
                 "oi": torch.empty((n, k), dtype=torch.int32, device=dev),
                 "od": torch.empty((n, k), dtype=torch.float32, device=dev)}
            if kind == "x":  # explicit centres, shifted off the issuers
                b["qx"] = to_dev((x + np.float32(1e-4)).astype(np.float32))
                b["qy"] = to_dev(y)
            bufs.append(b)
            pos.append((x, y, k, kind))
        args = [knnq.tick_args(p[2], b["q"], q_x=b.get("qx"), q_y=b.get("qy"), out_ids=b["oi"],
                               out_d2=b["od"]) for b, p in zip(bufs, pos)]
        s = torch.cuda.current_stream().cuda_stream
        for call in range(2):
            for b in bufs:
                b["oi"].fill_(-7)
            knnq.knn_batch_tick([w.handle for w in worlds], args, s)
            torch.cuda.synchronize()
            for i, ((x, y, k, kind), b, w) in enumerate(zip(pos, bufs, worlds)):
                q = b["q"].cpu().numpy()
                if kind == "x":
                    qx, qy = b["qx"].cpu().numpy(), b["qy"].cpu().numpy()
                    rid, rd2, _ = oracle.knn(x, y, q, k, qx, qy)
                else:
                    rid, rd2, _ = oracle.knn(x, y, q, k)
                assert_rows_equal(b["oi"].cpu().numpy(), b["od"].cpu().numpy(), rid, rd2,
                                  what=f"world {i} ({kind}, k={k}) call {call}")
                if kind == "u":
                    assert passed_on(w.expand_info()) <= q.shape[0] // 32 // 10, (i, w.expand_info())
                assert w.status()[0] == knnq.KNN_OK
    finally:
        for w in worlds:
            w.close()
