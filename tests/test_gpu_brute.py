"""The GPU brute-force baseline (every query against every object) gives the
same rows as the oracle and as the indexed path (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import knnq, synth
from tests.gpu_util import assert_rows_equal, gpu_tick, make_world, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def brute(x, y, k, q_id, q_x=None, q_y=None):
    torch, _ = torch_dev()
    ids, d2 = knnq.brute_force(to_dev(np.asarray(x, np.float32)), to_dev(np.asarray(y, np.float32)),
                               k, to_dev(np.asarray(q_id, np.int32)),
                               None if q_x is None else to_dev(np.asarray(q_x, np.float32)),
                               None if q_y is None else to_dev(np.asarray(q_y, np.float32)))
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d2.cpu().numpy()


def test_brute_10k_uniform_k8_full():
    w = synth.plain_uniform_one_tick()
    t = w.ticks[0]
    x, y, _ = oracle.apply_updates(w.x0, w.y0, t.upd_id, t.upd_x, t.upd_y)
    ids, d2 = brute(x, y, t.k, t.q_id)
    rid, rd2, _ = oracle.knn(x, y, t.q_id, t.k)
    assert_rows_equal(ids, d2, rid, rd2, what="brute 10k")


@pytest.mark.parametrize("k", [1, 16, 33, 64])
def test_brute_ragged_full(k):
    x, y = synth.clustered_positions(3001, 7)
    q = synth.random_subset(3001, 1500, seed=8, tick=0)
    ids, d2 = brute(x, y, k, q)
    rid, rd2, _ = oracle.knn(x, y, q, k)
    assert_rows_equal(ids, d2, rid, rd2, what=f"brute ragged k={k}")


def test_brute_explicit_anonymous_and_invalid_queries():
    r = np.random.default_rng(9)
    n = 2000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    q_id = np.array([5, -1, 17, n + 3, -7, 100], np.int32)
    q_x = np.array([0.5, 0.25, np.nan, 0.1, 0.2, 1.5], np.float32)
    q_y = np.array([0.5, 0.75, 0.3, 0.1, 0.2, -0.5], np.float32)
    ids, d2 = brute(x, y, 6, q_id, q_x, q_y)
    ok = np.array([0, 1, 5])            # valid rows (query 5 lies outside the domain)
    rid, rd2, _ = oracle.knn(x, y, q_id[ok], 6, q_x[ok], q_y[ok])
    assert_rows_equal(ids[ok], d2[ok], rid, rd2, what="brute explicit")
    bad = np.array([2, 3, 4])           # non-finite centre, issuer out of range
    assert np.all(ids[bad] == -1) and np.all(np.isinf(d2[bad]))


def test_brute_fewer_objects_than_k_and_empty_set():
    ids, d2 = brute([0.1, 0.2, 0.3], [0.1, 0.2, 0.3], 5, [0, 2])
    rid, rd2, _ = oracle.knn(np.array([0.1, 0.2, 0.3], np.float32),
                             np.array([0.1, 0.2, 0.3], np.float32), np.array([0, 2], np.int32), 5)
    assert_rows_equal(ids, d2, rid, rd2, what="brute n < k")
    torch, _ = torch_dev()
    q = to_dev(np.array([-1], np.int32))
    e = to_dev(np.zeros(1, np.float32))
    ids, d2 = knnq.brute_force(e[:0], e[:0], 4, q, e, e)
    assert np.all(ids.cpu().numpy() == -1) and np.all(np.isinf(d2.cpu().numpy()))


def test_brute_matches_indexed_ticks():
    w = synth.skewed_moving(n=40000, k=16, ticks=2, seed=10)
    world = make_world(w.x0, w.y0, k_max=16, max_queries=max(t.q_id.shape[0] for t in w.ticks))
    try:
        x, y = w.x0.copy(), w.y0.copy()
        for t in w.ticks:
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            ids, d2 = gpu_tick(world, t)
            bids, bd2 = brute(x, y, t.k, t.q_id)
            assert np.array_equal(ids, bids)
            assert np.array_equal(d2.view(np.uint32), bd2.view(np.uint32))
    finally:
        world.close()


def test_brute_rejects_bad_arguments():
    torch, _ = torch_dev()
    q = to_dev(np.zeros(1, np.int32))
    x = to_dev(np.zeros(4, np.float32))
    with pytest.raises(knnq.KnnError):
        knnq.brute_force(x, x, 65, q)
    with pytest.raises(knnq.KnnError):
        knnq.brute_force(x, x, 0, q)
