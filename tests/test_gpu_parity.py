"""Parity of the CUDA path with the CPU oracle (GPU).  Every comparison is
bit-exact: ids equal and squared distances equal as binary32 bit patterns."""
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


def run_and_compare(w, k_max=64, tuning=None, sample=None, world_kw=None, what=""):
    """Replay all ticks of workload ``w`` on the GPU and compare every tick with
    the oracle (all rows, or ``sample`` rows per tick)."""
    world = make_world(w.x0, w.y0, k_max=k_max,
                       max_queries=max(t.q_id.shape[0] for t in w.ticks), **(world_kw or {}))
    try:
        if tuning:
            world.set_tuning(**tuning)
        x, y = w.x0.copy(), w.y0.copy()
        for ti, t in enumerate(w.ticks):
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            ids, d2 = gpu_tick(world, t)
            rows = np.arange(t.q_id.shape[0]) if sample is None else \
                sample_rows(t.q_id.shape[0], sample, seed=ti)
            rid, rd2 = oracle_rows(x, y, t, rows)
            assert_rows_equal(ids, d2, rid, rd2, rows, what=f"{what} tick {ti}")
        st, bits = world.status()
        assert st == knnq.KNN_OK, (st, bits)
    finally:
        world.close()


# -------------------------------------------------------------------------
# The five workload shapes


def test_uniform_10k_k8_one_tick_full():
    run_and_compare(synth.plain_uniform_one_tick(), what="10k uniform k=8")


@pytest.mark.parametrize("k", [1, 5, 16, 33, 64])
def test_uniform_ragged_several_ticks_full(k):
    # 30011 objects: many sort tiles and leaf tiles, ragged tails everywhere
    w = synth.plain_uniform_moving(n=30011, k=k, ticks=2, seed=5)
    run_and_compare(w, what=f"30011 uniform k={k}")


@pytest.mark.parametrize("k", [4, 32])
def test_clustered_subset_queries_full(k):
    w = synth.skewed_moving(n=60000, k=k, ticks=2, seed=9)
    run_and_compare(w, what=f"60k clustered k={k}")


# -------------------------------------------------------------------------
# Large k: one warp per query, the list in shared memory (k > 64)


@pytest.mark.parametrize("k", [65, 100, 256, 512])
def test_large_k_uniform_ragged_full(k):
    w = synth.plain_uniform_moving(n=30011, k=k, ticks=2, seed=21)
    run_and_compare(w, k_max=512, what=f"30011 uniform k={k}")


@pytest.mark.parametrize("k", [128, 500])
def test_large_k_clustered_subset_sampled(k):
    w = synth.skewed_moving(n=120000, k=k, ticks=2, seed=22)
    run_and_compare(w, k_max=512, sample=3000, what=f"120k clustered k={k}")


@pytest.mark.parametrize("expansion", [1, 2, 3, 4])
@pytest.mark.parametrize("k", [1, 16, 64])
def test_expansion_kernels_agree(k, expansion):
    w = synth.skewed_moving(n=40000, k=k, ticks=2, seed=23, query_frac=0.5)
    run_and_compare(w, tuning=dict(expansion=expansion), what=f"k={k} expansion {expansion}")


def test_large_k_1m_uniform_sampled():
    w = synth.plain_uniform_moving(n=1_000_000, k=512, ticks=1, seed=24)
    w.ticks[0] = synth.Tick(w.ticks[0].upd_id, w.ticks[0].upd_x, w.ticks[0].upd_y,
                            synth.random_subset(1_000_000, 50_000, seed=25, tick=0), 512)
    run_and_compare(w, k_max=512, sample=1500, what="1M uniform k=512")


def test_uniform_1m_k16_full_size_sampled():
    w = synth.plain_uniform_moving(n=1_000_000, k=16, ticks=2, seed=0)
    run_and_compare(w, k_max=16, sample=20000, what="1M uniform k=16")


@pytest.mark.slow
def test_uniform_1m_k16_one_tick_every_row():
    # the benchmark workload's first tick, every one of its 1M rows against the
    # oracle (about a minute and a half of brute force on 16 host cores)
    w = synth.plain_uniform_moving(n=1_000_000, k=16, ticks=1, seed=0)
    run_and_compare(w, k_max=16, what="1M uniform k=16, every row")


def test_clustered_4m_k32_full_size_sampled():
    w = synth.skewed_moving(n=4_000_000, k=32, ticks=2, seed=0)
    run_and_compare(w, k_max=32, sample=8000, what="4M clustered k=32")


# -------------------------------------------------------------------------
# Index parameters never change a result


@pytest.mark.parametrize("tuning", [dict(leaf_capacity=1), dict(leaf_capacity=3, grid_level=2),
                                    dict(leaf_capacity=200, grid_level=4, packet_level=1),
                                    dict(leaf_capacity=4096, grid_level=1, packet_level=0),
                                    dict(leaf_capacity=16, grid_level=9, packet_level=9),
                                    dict(expansion=2), dict(expansion=2, leaf_capacity=3),
                                    dict(expansion=1, leaf_capacity=300, grid_level=3)])
def test_tuning_invariance(tuning):
    w = synth.skewed_moving(n=20000, k=16, ticks=1, seed=11, query_frac=0.5)
    run_and_compare(w, tuning=tuning, what=f"tuning {tuning}")


@pytest.mark.parametrize("k", [4, 8, 32])
def test_crowded_cells_explicit_centres(k):
    # a coarse cell map over small leaves: most cells hold many leaves, so the
    # walk narrows them to the key range of the packet box; explicit centres
    # (some outside the domain) and issuers at their positions
    w = synth.skewed_moving(n=30000, k=k, ticks=2, seed=13, query_frac=0.4)
    r = np.random.default_rng(14)
    t0 = w.ticks[0]
    nq = t0.q_id.shape[0]
    qx = np.clip(r.normal(0.5, 0.3, nq), -0.2, 1.2).astype(np.float32)
    qy = np.clip(r.normal(0.5, 0.3, nq), -0.2, 1.2).astype(np.float32)
    w.ticks[0] = synth.Tick(t0.upd_id, t0.upd_x, t0.upd_y, t0.q_id, k, qx, qy)
    run_and_compare(w, k_max=k, tuning=dict(leaf_capacity=4, grid_level=3, packet_level=3),
                    what=f"crowded cells k={k}")


def test_max_depth_invariance():
    w = synth.skewed_moving(n=20000, k=8, ticks=1, seed=12)
    for depth in (1, 3, 9):
        run_and_compare(w, world_kw=dict(max_depth=depth), what=f"max_depth {depth}")


# -------------------------------------------------------------------------
# Degenerate and edge cases


def tick(q_id, k, upd=None, q_x=None, q_y=None):
    uid, ux, uy = upd if upd is not None else (np.zeros(0, np.int32), np.zeros(0, np.float32),
                                               np.zeros(0, np.float32))
    return synth.Tick(np.asarray(uid, np.int32), np.asarray(ux, np.float32),
                      np.asarray(uy, np.float32), np.asarray(q_id, np.int32), k,
                      None if q_x is None else np.asarray(q_x, np.float32),
                      None if q_y is None else np.asarray(q_y, np.float32))


def compare_ticks(x0, y0, ticks, k_max=64, tuning=None, expect_status=knnq.KNN_OK):
    x0, y0 = np.asarray(x0, np.float32), np.asarray(y0, np.float32)
    world = make_world(x0, y0, k_max=k_max, max_queries=max(1, max(t.q_id.shape[0] for t in ticks)))
    try:
        if tuning:
            world.set_tuning(**tuning)
        x, y = np.asarray(x0, np.float32), np.asarray(y0, np.float32)
        for t in ticks:
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            ids, d2 = gpu_tick(world, t)
            if t.q_id.shape[0]:
                rid, rd2, _ = oracle.knn(x, y, t.q_id, t.k, t.q_x, t.q_y)
                assert_rows_equal(ids, d2, rid, rd2)
        st, bits = world.status()
        assert st == expect_status, (st, bits)
        return bits
    finally:
        world.close()


def test_single_object_pads():
    compare_ticks([0.5], [0.5], [tick([0], 3)])


@pytest.mark.parametrize("n,k", [(2, 1), (2, 5), (5, 4), (5, 5), (7, 64), (7, 65), (300, 512),
                                 (513, 512)])
def test_fewer_objects_than_k(n, k):
    r = np.random.default_rng(n * 100 + k)
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    compare_ticks(x, y, [tick(np.arange(n), k)], k_max=max(64, k))


def test_all_coincident_objects():
    n = 5000
    x = np.full(n, 0.25, np.float32)
    compare_ticks(x, x.copy(), [tick(np.arange(n), 16), tick(np.arange(0, n, 7), 64)])


def test_duplicates_and_lattice_ties():
    g = 70
    ii, jj = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    x = np.concatenate([ii.ravel() / 128.0, ii.ravel()[:500] / 128.0]).astype(np.float32)
    y = np.concatenate([jj.ravel() / 128.0, jj.ravel()[:500] / 128.0]).astype(np.float32)
    n = x.shape[0]
    for k in (4, 5, 12, 13, 40):
        compare_ticks(x, y, [tick(np.arange(n), k)], tuning=dict(leaf_capacity=2))


def test_duplicate_update_ids_last_wins():
    r = np.random.default_rng(3)
    n = 3000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    uid = np.concatenate([np.arange(n), r.integers(0, n, 4000)]).astype(np.int32)
    ux, uy = r.random(uid.shape[0]).astype(np.float32), r.random(uid.shape[0]).astype(np.float32)
    compare_ticks(x, y, [tick(np.arange(n), 8, (uid, ux, uy)),
                         tick(np.arange(n)[::-1], 8, (uid[::-1], ux, uy))])


def test_invalid_updates_skipped_and_reported():
    r = np.random.default_rng(4)
    n = 2000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    uid = np.array([5, -1, n, 7, 7, 9], np.int32)
    ux = np.array([0.5, 0.1, 0.1, 0.2, np.nan, np.inf], np.float32)
    uy = np.array([0.5, 0.1, 0.1, 0.2, 0.3, 0.1], np.float32)
    bits = compare_ticks(x, y, [tick(np.arange(n), 8, (uid, ux, uy))],
                         expect_status=knnq.KNN_ERR_DEVICE_INPUT)
    assert bits & knnq.ERR_BAD_UPDATE_ID and bits & knnq.ERR_NONFINITE_UPDATE


def test_invalid_queries_padded_and_reported():
    r = np.random.default_rng(5)
    n = 2000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    bits = compare_ticks(x, y, [tick([0, -1, n, 3, -7, 3], 4)],
                         expect_status=knnq.KNN_ERR_DEVICE_INPUT)
    assert bits & knnq.ERR_BAD_QUERY
    q = [0, -1, 5, n, -1]
    qx = [0.3, 0.2, np.nan, 0.5, 0.9]
    bits = compare_ticks(x, y, [tick(q, 4, None, qx, qx)], expect_status=knnq.KNN_ERR_DEVICE_INPUT)
    assert bits & knnq.ERR_BAD_QUERY


@pytest.mark.parametrize("expansion", [0, 2, 3])
def test_explicit_and_anonymous_centres_outside_domain(expansion):
    r = np.random.default_rng(6)
    n = 20000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    x[:300] = (r.random(300) * 6 - 3).astype(np.float32)   # objects outside [0,1)
    y[:300] = (r.random(300) * 6 - 3).astype(np.float32)
    nq = 5000
    qid = np.where(r.random(nq) < 0.5, -1, r.integers(0, n, nq)).astype(np.int32)
    qx = (r.random(nq) * 1.4 - 0.2).astype(np.float32)
    qy = (r.random(nq) * 1.4 - 0.2).astype(np.float32)
    qx[:50] = 7.5
    compare_ticks(x, y, [tick(qid, 16, None, qx, qy), tick(qid[::2], 3, None, qx[::2], qy[::2])],
                  tuning=dict(expansion=expansion) if expansion else None)


def test_repeated_query_ids_and_empty_tick():
    r = np.random.default_rng(7)
    n = 5000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    q = r.integers(0, n, 3000).astype(np.int32)
    q[:100] = 17
    compare_ticks(x, y, [tick(q, 10), tick(np.zeros(0, np.int32), 4), tick(q[:1], 1)])


@pytest.mark.parametrize("nq", [1200, 2600, 5000])
def test_repeated_query_ids_both_counting_sorts(nq):
    # fewer queries than half the objects are counted by place, more by issuer
    # id; both with issuers that query several times and issuers that query once
    r = np.random.default_rng(17)
    n = 5000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    q = r.integers(0, n, nq).astype(np.int32)
    q[:40] = 23
    q[40:43] = 4999
    compare_ticks(x, y, [tick(q, 9), tick(r.permutation(n)[:nq].astype(np.int32), 6)])


def test_updates_aligned_and_offset_arrays():
    # the same updates (repeated ids, ids out of range, non-finite positions, a
    # length that is not a multiple of 4) through 16-byte aligned caller arrays
    # and through arrays one element off
    torch, dev = torch_dev()
    r = np.random.default_rng(23)
    n = 5000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    m = 4003
    uid = r.integers(-3, n + 3, m).astype(np.int32)
    uid[100:140] = 77
    ux = r.random(m).astype(np.float32)
    uy = r.random(m).astype(np.float32)
    ux[5] = np.nan
    uy[9] = np.inf
    q = np.arange(n, dtype=np.int32)
    xe, ye, _ = oracle.apply_updates(x, y, uid, ux, uy)
    rid, rd2, _ = oracle.knn(xe, ye, q, 8)
    for off in (0, 1):
        bufs = []
        for a in (uid, ux, uy):
            t = torch.zeros(m + off, dtype=torch.from_numpy(a).dtype, device=dev)
            t[off:] = torch.from_numpy(a).to(dev)
            bufs.append(t[off:])
        world = make_world(x, y, k_max=8, max_queries=n)
        try:
            ids, d2 = world.tick(8, to_dev(q), *bufs)
            torch.cuda.synchronize()
            assert_rows_equal(ids.cpu().numpy(), d2.cpu().numpy(), rid, rd2, what=f"offset {off}")
            st, bits = world.status()
            assert st == knnq.KNN_ERR_DEVICE_INPUT, (st, bits)
            assert bits & knnq.ERR_BAD_UPDATE_ID and bits & knnq.ERR_NONFINITE_UPDATE
        finally:
            world.close()


def test_one_query_per_object_and_near_misses():
    # as many queries as objects, counted by issuer id: a permutation of the
    # objects (each queries once: the query offsets are the identity and their
    # scan is skipped), then the cases that look alike but are not -- one
    # issuer twice and another never, one invalid issuer -- which take the scan
    r = np.random.default_rng(19)
    n = 20000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    perm = r.permutation(n).astype(np.int32)
    dup = perm.copy()
    dup[100] = dup[200]
    moved = (r.random(n) < 0.5).astype(bool)
    uid = np.flatnonzero(moved).astype(np.int32)
    upd = (uid, np.clip(x[uid] + 1e-3, 0, 1), np.clip(y[uid] - 1e-3, 0, 1))
    compare_ticks(x, y, [tick(perm, 16), tick(dup, 16, upd), tick(perm, 8), tick(perm[::-1], 16)])
    bad = perm.copy()
    bad[5] = -7
    compare_ticks(x, y, [tick(perm, 16), tick(bad, 16), tick(perm, 16)],
                  expect_status=knnq.KNN_ERR_DEVICE_INPUT)


def test_domain_offset_and_scale():
    r = np.random.default_rng(8)
    n = 20000
    x = (1000.0 + 50.0 * r.random(n)).astype(np.float32)
    y = (-20.0 + 50.0 * r.random(n)).astype(np.float32)
    torch, dev = torch_dev()
    from paper_1412_6170_gb300 import knnq as K
    world = K.World(to_dev(x), to_dev(y), k_max=16, domain=(1000.0, -20.0, 50.0))
    try:
        ids, d2 = world.tick(16, to_dev(np.arange(n, dtype=np.int32)))
        torch.cuda.synchronize()
        rid, rd2, _ = oracle.knn(x, y, np.arange(n, dtype=np.int32), 16)
        assert_rows_equal(ids.cpu().numpy(), d2.cpu().numpy(), rid, rd2)
    finally:
        world.close()


# -------------------------------------------------------------------------
# API paths


def test_host_buffer_tick_matches_device_tick():
    import ctypes
    w = synth.plain_uniform_moving(n=50000, k=16, ticks=1, seed=2)
    t = w.ticks[0]
    a = make_world(w.x0, w.y0, k_max=16)
    b = make_world(w.x0, w.y0, k_max=16)
    try:
        ids, d2 = gpu_tick(a, t)
        nq = t.q_id.shape[0]
        hid = np.empty((nq, 16), np.int32)
        hd2 = np.empty((nq, 16), np.float32)
        p = lambda arr: arr.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        knnq.knn_tick_host(b.handle, p(t.upd_id), p(t.upd_x), p(t.upd_y), t.upd_id.shape[0],
                           p(t.q_id), None, None, nq, 16, p(hid), p(hd2), 0)
        assert np.array_equal(ids, hid) and np.array_equal(d2.view(np.uint32), hd2.view(np.uint32))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("k,explicit", [(16, False), (5, True)])
def test_pinned_host_tick_matches_device_tick(mode, k, explicit):
    # pinned arrays written (bit 0) and read (bit 1) in place by the kernels,
    # over several ticks, give the rows of the device-array tick
    w = synth.plain_uniform_moving(n=60000, k=k, ticks=3, seed=5)
    a = make_world(w.x0, w.y0, k_max=k)
    b = make_world(w.x0, w.y0, k_max=k)
    b.set_host_io(write_rows=bool(mode & 1), read_inputs=bool(mode & 2))
    torch, dev = torch_dev()
    try:
        for i, t in enumerate(w.ticks):
            nq = t.q_id.shape[0]
            if explicit:
                qx = (w.x0[t.q_id] + np.float32(0.001 * (i + 1))).astype(np.float32)
                qy = w.y0[t.q_id].copy()
                pin = [torch.from_numpy(v).pin_memory()
                       for v in (t.upd_id, t.upd_x, t.upd_y, t.q_id, qx, qy)]
                ids, d2 = a.tick(k, *(v.to(dev) for v in (pin[3], pin[0], pin[1], pin[2])),
                                 q_x=pin[4].to(dev), q_y=pin[5].to(dev))
            else:
                pin = [torch.from_numpy(v).pin_memory()
                       for v in (t.upd_id, t.upd_x, t.upd_y, t.q_id)]
                ids, d2 = a.tick(k, *(v.to(dev) for v in (pin[3], pin[0], pin[1], pin[2])))
            torch.cuda.synchronize()
            hid = torch.full((nq, k), 7, dtype=torch.int32).pin_memory()
            hd2 = torch.full((nq, k), 7.0, dtype=torch.float32).pin_memory()
            knnq.knn_tick_host(b.handle, pin[0].data_ptr(), pin[1].data_ptr(), pin[2].data_ptr(),
                               t.upd_id.shape[0], pin[3].data_ptr(),
                               pin[4].data_ptr() if explicit else None,
                               pin[5].data_ptr() if explicit else None, nq, k,
                               hid.data_ptr(), hd2.data_ptr(), 0)
            assert np.array_equal(ids.cpu().numpy(), hid.numpy())
            assert np.array_equal(d2.cpu().numpy().view(np.uint32), hd2.numpy().view(np.uint32))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_pipelined_host_ticks_match_device_ticks(pinned):
    # two ticks in flight (two sets of output arrays), waited for one tick late
    import ctypes
    k = 16
    w = synth.plain_uniform_moving(n=70000, k=k, ticks=5, seed=6)
    a = make_world(w.x0, w.y0, k_max=k)
    b = make_world(w.x0, w.y0, k_max=k)
    torch, dev = torch_dev()
    try:
        want = [gpu_tick(a, t) for t in w.ticks]
        nq = w.ticks[0].q_id.shape[0]
        if pinned:
            ins = [[torch.from_numpy(v).pin_memory() for v in (t.upd_id, t.upd_x, t.upd_y, t.q_id)]
                   for t in w.ticks]
            outs = [(torch.empty((nq, k), dtype=torch.int32).pin_memory(),
                     torch.empty((nq, k), dtype=torch.float32).pin_memory()) for _ in range(2)]
            ptr = lambda v: v.data_ptr()  # noqa: E731
            view = lambda v: v.numpy()  # noqa: E731
        else:
            ins = [[np.ascontiguousarray(v) for v in (t.upd_id, t.upd_x, t.upd_y, t.q_id)]
                   for t in w.ticks]
            outs = [(np.empty((nq, k), np.int32), np.empty((nq, k), np.float32))
                    for _ in range(2)]
            ptr = lambda v: v.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
            view = lambda v: v  # noqa: E731
        s = torch.cuda.Stream()
        tickets = []
        for i, t in enumerate(w.ticks):
            u, ux, uy, q = ins[i]
            oi, od = outs[i % 2]
            tickets.append(knnq.knn_tick_host_submit(
                b.handle, ptr(u), ptr(ux), ptr(uy), t.upd_id.shape[0], ptr(q), None, None, nq,
                k, ptr(oi), ptr(od), s.cuda_stream))
            if i >= 1:
                knnq.knn_tick_host_wait(b.handle, tickets[i - 1])
                pi, pd = outs[(i - 1) % 2]
                assert np.array_equal(view(pi), want[i - 1][0]), i - 1
                assert np.array_equal(view(pd).view(np.uint32), want[i - 1][1].view(np.uint32))
        knnq.knn_tick_host_wait(b.handle, tickets[-1])
        li, ld = outs[(len(w.ticks) - 1) % 2]
        assert np.array_equal(view(li), want[-1][0])
        assert np.array_equal(view(ld).view(np.uint32), want[-1][1].view(np.uint32))
        with pytest.raises(knnq.KnnError):
            knnq.knn_tick_host_wait(b.handle, tickets[-1] + 1)
        assert b.status()[0] == knnq.KNN_OK
    finally:
        a.close()
        b.close()


def test_bounded_wait_runs_out_and_world_stays_usable():
    # failure detection without a fault: a look-back wait that nothing
    # satisfies gives up after its poll limit, the status reports the timeout,
    # and the next tick is exact again
    import time
    torch, _ = torch_dev()
    w = synth.plain_uniform_moving(n=20000, k=8, ticks=2, seed=15)
    world = make_world(w.x0, w.y0, k_max=8)
    try:
        x, y, _ = oracle.apply_updates(w.x0, w.y0, w.ticks[0].upd_id, w.ticks[0].upd_x,
                                       w.ticks[0].upd_y)
        gpu_tick(world, w.ticks[0])
        assert world.status()[0] == knnq.KNN_OK
        t0 = time.perf_counter()
        world.test_wait_timeout()
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < 10.0
        st, bits = world.status()
        assert st == knnq.KNN_ERR_TIMEOUT and bits & 8
        assert world.status()[0] == knnq.KNN_OK  # reported once, then cleared
        t = w.ticks[1]
        x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
        ids, d2 = gpu_tick(world, t)
        rid, rd2, _ = oracle.knn(x, y, t.q_id, t.k)
        assert_rows_equal(ids, d2, rid, rd2, what="tick after a timed-out wait")
        assert world.status()[0] == knnq.KNN_OK
    finally:
        world.close()


def test_checkpoint_resume_bit_identical():
    w = synth.plain_uniform_moving(n=40000, k=8, ticks=6, seed=4)
    a = make_world(w.x0, w.y0, k_max=8)
    try:
        for t in w.ticks[:3]:
            gpu_tick(a, t)
        px, py = a.positions()
        from paper_1412_6170_gb300 import knnq as K
        b = K.World(px, py, k_max=8)
        try:
            for t in w.ticks[3:]:
                ra = gpu_tick(a, t)
                rb = gpu_tick(b, t)
                assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        finally:
            b.close()
    finally:
        a.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_stage_profiling_reports_every_stage(graphs):
    w = synth.plain_uniform_moving(n=100000, k=16, ticks=2, seed=1)
    world = make_world(w.x0, w.y0, k_max=16)
    try:
        world.set_graphs(graphs)
        world.set_profiling(True)
        for t in w.ticks:
            gpu_tick(world, t)
            st = world.stage_times()
            assert list(st) == knnq.stage_names()
            assert all(v >= 0 for v in st.values()) and st["expand"] > 0
    finally:
        world.close()


def test_tick_graph_replay_matches_direct_launches():
    # three input sets cycled: from the fourth tick on, knn_tick replays the
    # graphs it recorded; a second world launches every kernel directly
    torch, _ = torch_dev()
    w = synth.plain_uniform_moving(n=30011, k=16, ticks=3, seed=12)
    dev_ticks = [[to_dev(a) for a in (t.q_id, t.upd_id, t.upd_x, t.upd_y)] for t in w.ticks]
    n_q = w.ticks[0].q_id.shape[0]
    outs = [[(torch.empty((n_q, 16), dtype=torch.int32, device="cuda"),
              torch.empty((n_q, 16), dtype=torch.float32, device="cuda")) for _ in range(3)]
            for _ in range(2)]  # same output buffers for the same input set
    a = make_world(w.x0, w.y0, k_max=16)
    b = make_world(w.x0, w.y0, k_max=16)
    try:
        b.set_graphs(False)
        # sets 0 and 1 recorded up front (nothing runs); set 2 is recorded by its first tick
        for j in range(2):
            a.record_tick(16, *dev_ticks[j], out_ids=outs[0][j][0], out_d2=outs[0][j][1])
        assert a.launches() == 0
        x, y = w.x0.copy(), w.y0.copy()
        for i in range(8):
            t = w.ticks[i % 3]
            if i == 5:  # profiling marks change the recording; the results do not
                a.set_profiling(True)
            oa, ob = outs[0][i % 3], outs[1][i % 3]
            ids_a, d2_a = a.tick(16, *dev_ticks[i % 3], out_ids=oa[0], out_d2=oa[1])
            ids_b, d2_b = b.tick(16, *dev_ticks[i % 3], out_ids=ob[0], out_d2=ob[1])
            torch.cuda.synchronize()
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            rows = sample_rows(t.q_id.shape[0], 2000, seed=i)
            rid, rd2 = oracle_rows(x, y, t, rows)
            ia, da = ids_a.cpu().numpy(), d2_a.cpu().numpy()
            assert_rows_equal(ia, da, rid, rd2, rows, what=f"graph tick {i}")
            assert np.array_equal(ia, ids_b.cpu().numpy())
            assert np.array_equal(da.view(np.uint32), d2_b.cpu().numpy().view(np.uint32))
        assert a.launches() == b.launches()
        st = a.stage_times()
        assert st["expand"] > 0 and all(v >= 0 for v in st.values())
        for world in (a, b):
            s, bits = world.status()
            assert s == knnq.KNN_OK, (s, bits)
    finally:
        a.close()
        b.close()


# -------------------------------------------------------------------------
# Index reuse: the leaves kept across ticks give the same rows


@pytest.mark.parametrize("max_age,factor", [(3, 0.0), (100, 1.25)])
def test_index_reuse_uniform_matches_oracle(max_age, factor):
    w = synth.plain_uniform_moving(n=30011, k=16, ticks=6, seed=31)
    world = make_world(w.x0, w.y0, k_max=16, max_queries=30011)
    try:
        world.set_index_reuse(max_age, factor)
        x, y = w.x0.copy(), w.y0.copy()
        ages = []
        for ti, t in enumerate(w.ticks):
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            ids, d2 = gpu_tick(world, t)
            rid, rd2 = oracle_rows(x, y, t, np.arange(t.q_id.shape[0]))
            assert_rows_equal(ids, d2, rid, rd2, what=f"reuse tick {ti}")
            ages.append(world.index_info()["age"])
        assert ages[0] == 0 and max(ages) >= 1, ages  # built once, then reused
        if factor == 0.0:
            assert max(ages) <= max_age, ages
        st, bits = world.status()
        assert st == knnq.KNN_OK, (st, bits)
    finally:
        world.close()


def test_index_reuse_clustered_subset_queries_and_explicit_centres():
    w = synth.skewed_moving(n=60000, k=8, ticks=5, seed=32)
    world = make_world(w.x0, w.y0, k_max=8, max_queries=max(t.q_id.shape[0] for t in w.ticks))
    try:
        world.set_index_reuse(50)
        x, y = w.x0.copy(), w.y0.copy()
        r = np.random.default_rng(33)
        for ti, t in enumerate(w.ticks):
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            if ti % 2:  # explicit centres near the issuers
                qx = np.clip(x[t.q_id] + r.normal(0, 0.01, t.q_id.shape[0]), 0, 1).astype(np.float32)
                qy = np.clip(y[t.q_id] + r.normal(0, 0.01, t.q_id.shape[0]), 0, 1).astype(np.float32)
                t = synth.Tick(t.upd_id, t.upd_x, t.upd_y, t.q_id, t.k, qx, qy)
            ids, d2 = gpu_tick(world, t)
            rows = sample_rows(t.q_id.shape[0], 3000, seed=ti)
            rid, rd2 = oracle_rows(x, y, t, rows)
            assert_rows_equal(ids, d2, rid, rd2, rows, what=f"clustered reuse tick {ti}")
        assert world.index_info()["age"] >= 1
    finally:
        world.close()


def test_index_reuse_across_empty_cells_and_cost_rebuild():
    # every object in the left half; half of them jump into the right half,
    # whose level-G cells only have empty leaves; then every object jumps into
    # one small square, which piles them into a few leaves: the next tick's
    # cost test rebuilds.  Every tick stays exact.
    n = 20000
    r = np.random.default_rng(34)
    x0 = (r.random(n) * 0.5).astype(np.float32)
    y0 = r.random(n).astype(np.float32)
    ids = np.arange(n, dtype=np.int32)
    none = (np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32))
    world = make_world(x0, y0, k_max=8, max_queries=n)
    try:
        world.set_index_reuse(1000, 2.0)
        x, y = x0.copy(), y0.copy()
        infos = []
        for ti in range(5):
            if ti == 2:
                moved = ids[: n // 2]
                upd = (moved, (x[moved] + 0.5).astype(np.float32), y[moved].copy())
            elif ti == 3:
                upd = (ids, (0.3 + 0.01 * r.random(n)).astype(np.float32),
                       (0.6 + 0.01 * r.random(n)).astype(np.float32))
            else:
                upd = none
            t = synth.Tick(upd[0], upd[1], upd[2], ids, 8)
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            got_ids, got_d2 = gpu_tick(world, t)
            rows = sample_rows(n, 3000, seed=ti)
            rid, rd2 = oracle_rows(x, y, t, rows)
            assert_rows_equal(got_ids, got_d2, rid, rd2, rows, what=f"jump tick {ti}")
            infos.append(world.index_info())
        assert [i["age"] for i in infos[:4]] == [0, 1, 2, 3], infos
        assert infos[4]["rebuilt"] == 1, infos
        st, bits = world.status()
        assert st == knnq.KNN_OK, (st, bits)
    finally:
        world.close()


# -------------------------------------------------------------------------
# Per-query list sizes (q = (x, y, k))


@pytest.mark.parametrize("k,expansion", [(16, 0), (16, 2), (16, 3), (33, 0), (100, 0), (5, 1)])
def test_per_query_k_rows_are_prefixes(k, expansion):
    torch, _ = torch_dev()
    w = synth.skewed_moving(n=30000, k=k, ticks=2, seed=41, query_frac=0.6)
    world = make_world(w.x0, w.y0, k_max=128, max_queries=max(t.q_id.shape[0] for t in w.ticks))
    r = np.random.default_rng(42)
    try:
        if expansion:
            world.set_tuning(expansion=expansion)
        x, y = w.x0.copy(), w.y0.copy()
        for ti, t in enumerate(w.ticks):
            x, y, _ = oracle.apply_updates(x, y, t.upd_id, t.upd_x, t.upd_y)
            qk = r.integers(0, k + 1, t.q_id.shape[0]).astype(np.int32)
            ids, d2 = world.tick(k, to_dev(t.q_id), to_dev(t.upd_id), to_dev(t.upd_x),
                                 to_dev(t.upd_y), q_k=to_dev(qk))
            torch.cuda.synchronize()
            ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
            rows = sample_rows(t.q_id.shape[0], 3000, seed=ti)
            rid, rd2 = oracle_rows(x, y, t, rows, k=k)
            cols = np.arange(k)[None, :]
            keep = cols < qk[rows][:, None]  # the first q_k entries; padding after them
            rid = np.where(keep, rid, -1).astype(np.int32)
            rd2 = np.where(keep, rd2, np.float32(np.inf)).astype(np.float32)
            assert_rows_equal(ids, d2, rid, rd2, rows, what=f"per-query k tick {ti}")
        st, bits = world.status()
        assert st == knnq.KNN_OK, (st, bits)
    finally:
        world.close()


def test_per_query_k_out_of_range_pads_and_reports():
    torch, _ = torch_dev()
    r = np.random.default_rng(43)
    n = 5000
    x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    world = make_world(x, y, k_max=8, max_queries=4)
    try:
        q = np.array([1, 2, 3, 4], np.int32)
        qk = np.array([3, -1, 9, 8], np.int32)
        ids, d2 = world.tick(8, to_dev(q), q_k=to_dev(qk))
        torch.cuda.synchronize()
        ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
        rid, rd2, _ = oracle.knn(x, y, q, 8)
        assert np.array_equal(ids[0, :3], rid[0, :3]) and np.all(ids[0, 3:] == -1)
        assert np.array_equal(ids[3], rid[3])
        assert np.all(ids[1:3] == -1) and np.all(np.isinf(d2[1:3]))
        st, bits = world.status()
        assert st != knnq.KNN_OK and bits & 4, (st, bits)
    finally:
        world.close()
