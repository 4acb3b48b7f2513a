"""Serving loop (GPU): every request's rows are the same whether it runs alone
or mixed with other worlds' requests on several streams under a device-memory
budget that forces scratch evictions, equal to plain knn_tick rows, and equal
to the CPU oracle (sampled rows of every request)."""
import numpy as np
import pytest

from paper_1412_6170_gb300 import knnq, synth
from tests.gpu_util import assert_rows_equal, oracle_rows, sample_rows, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_requests(ws, ticks):
    """One request per (world, tick), interleaved in a seeded random arrival order
    that keeps each world's ticks in order."""
    r = np.random.default_rng(1)
    order = []
    nxt = [0] * len(ws)
    while any(n < ticks for n in nxt):
        i = int(r.integers(0, len(ws)))
        if nxt[i] < ticks:
            order.append((i, nxt[i]))
            nxt[i] += 1
    return order


def check_against_oracle(ws, order, res, count=200):
    """Every request of a world tick sets all positions, so a request's rows depend
    only on its own tick: sampled rows of each against the oracle."""
    for j, ((i, ti), (ids, d2)) in enumerate(zip(order, res)):
        t = ws[i].ticks[ti]
        rows = sample_rows(t.q_id.shape[0], count, seed=j)
        rid, rd2 = oracle_rows(t.upd_x, t.upd_y, t, rows, k=ws[i].k)
        assert_rows_equal(ids, d2, rid, rd2, rows, what=f"request {j} (world {i}, tick {ti})")


def run_server(ws, order, n_slots, budget, torch, dev, k_max=32):
    srv = knnq.knn_server_create(n_slots, budget)
    keep = []
    try:
        idx = []
        for w in ws:
            x, y = to_dev(w.x0), to_dev(w.y0)
            keep += [x, y]
            d = knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, k_max, w.n)
            idx.append(knnq.knn_server_add_world(srv, d, x.data_ptr(), y.data_ptr(), w.n))
        outs, rids = [], []
        for i, ti in order:
            t = ws[i].ticks[ti]
            tens = [to_dev(t.q_id), to_dev(t.upd_id), to_dev(t.upd_x), to_dev(t.upd_y)]
            oi = torch.empty((t.q_id.shape[0], ws[i].k), dtype=torch.int32, device=dev)
            od = torch.empty((t.q_id.shape[0], ws[i].k), dtype=torch.float32, device=dev)
            keep += tens + [oi, od]
            a = knnq.tick_args(ws[i].k, *tens, out_ids=oi, out_d2=od)
            rids.append(knnq.knn_server_submit(srv, idx[i], a))
            outs.append((oi, od))
        lat = [knnq.knn_server_wait(srv, rid) for rid in rids]
        stats = knnq.knn_server_stats(srv)
        for j in idx:
            assert knnq.knn_server_world_status(srv, j)[0] == knnq.KNN_OK
        res = [(oi.cpu().numpy(), od.cpu().numpy()) for oi, od in outs]
    finally:
        knnq.knn_server_destroy(srv)
    return res, lat, stats


def test_alone_and_mixed_give_identical_rows():
    torch, dev = torch_dev()
    ws = synth.many_worlds(n_worlds=7, seed=11, n_lo=2000, n_hi=60000, ks=(4, 16, 32),
                           ticks=3, query_frac=(0.2, 1.0))
    order = make_requests(ws, 3)
    alone, lat_a, st_a = run_server(ws, order, n_slots=1, budget=0, torch=torch, dev=dev)
    # a budget of 1.5 times the largest world's scratch: admission must evict and re-admit
    assert st_a["scratch_bytes"] > 2 * st_a["largest_world_scratch"]
    budget = int(1.5 * st_a["largest_world_scratch"])
    mixed, lat_m, st = run_server(ws, order, n_slots=4, budget=budget, torch=torch, dev=dev)
    assert st["completed"] == len(order) and st["evictions"] > 0
    assert all(v > 0 for v in lat_a + lat_m)
    for (ai, ad), (mi, md) in zip(alone, mixed):
        assert np.array_equal(ai, mi)
        assert np.array_equal(ad.view(np.uint32), md.view(np.uint32))
    # and both equal plain ticks, world by world
    plain = {}
    for i, w in enumerate(ws):
        world = knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n)
        try:
            for ti, t in enumerate(w.ticks):
                ids, d2 = world.tick(w.k, to_dev(t.q_id), to_dev(t.upd_id), to_dev(t.upd_x),
                                     to_dev(t.upd_y))
                torch.cuda.synchronize()
                plain[(i, ti)] = (ids.cpu().numpy(), d2.cpu().numpy())
        finally:
            world.close()
    for (i, ti), (mi, md) in zip(order, mixed):
        pi, pd = plain[(i, ti)]
        assert np.array_equal(pi, mi) and np.array_equal(pd.view(np.uint32), md.view(np.uint32))
    # and the oracle, request by request
    check_against_oracle(ws, order, mixed)


def test_serving_mix_like_the_serving_workload_matches_oracle():
    # clustered worlds of uneven size, k up to 64, 10-100 % of the objects
    # querying, a budget of a third of the worlds' total scratch: admission
    # evicts and re-admits, and every request's sampled rows equal the oracle
    torch, dev = torch_dev()
    ws = [synth.serving_world(i, seed=3, n_worlds=10, n_lo=5000, n_hi=120000) for i in range(10)]
    order = make_requests(ws, 1) * 2  # every world twice (the same tick again)
    order = [order[j] for j in np.random.default_rng(5).permutation(len(order))]
    _, _, st_a = run_server(ws, order[:len(ws)], n_slots=2, budget=0, torch=torch, dev=dev,
                            k_max=64)
    budget = max(int(1.5 * st_a["largest_world_scratch"]), st_a["scratch_bytes"] // 3)
    res, lat, st = run_server(ws, order, n_slots=4, budget=budget, torch=torch, dev=dev,
                              k_max=64)
    assert st["completed"] == len(order) and st["evictions"] > 0
    assert all(v > 0 for v in lat)
    check_against_oracle(ws, order, res)


def test_world_that_can_never_fit_is_refused():
    torch, dev = torch_dev()
    srv = knnq.knn_server_create(2, 1 << 20)
    try:
        x = to_dev(np.random.default_rng(0).random(100000).astype(np.float32))
        d = knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, 16, 100000)
        with pytest.raises(knnq.KnnError) as e:
            knnq.knn_server_add_world(srv, d, x.data_ptr(), x.data_ptr(), 100000)
        assert e.value.status == knnq.KNN_ERR_ADMISSION
    finally:
        knnq.knn_server_destroy(srv)
