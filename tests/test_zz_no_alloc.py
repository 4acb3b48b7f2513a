"""knn_query_static, the allocation-free one-shot call (GPU).

This entry point is for callers that must not allocate device memory:
latency-critical loops where cudaMalloc/cudaFree would synchronize the device,
services whose device memory belongs to another allocator or a fixed budget,
and code that must not fail mid-request because an allocation did.  Its
scratch is a static device array, so the tests check that calls in a row
(each one finding the previous one's leftovers in that array, at other sizes)
give exactly the rows of the regular path, knn_world_create + knn_tick without
updates, and of the CPU oracle.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import knnq, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()


def regular_path(x, y, q_id, k, q_x=None, q_y=None, leaf_capacity=0):
    """Rows from the existing entry points (a world plus one tick, no updates)."""
    import torch
    world = knnq.World(dev(x), dev(y), k_max=64, max_queries=len(q_id),
                       leaf_capacity=leaf_capacity)
    try:
        ids, d2 = world.tick(k, dev(q_id), q_x=dev(q_x), q_y=dev(q_y))
        torch.cuda.synchronize()
        return ids.cpu().numpy(), d2.cpu().numpy()
    finally:
        world.close()


def static_path(x, y, q_id, k, q_x=None, q_y=None, leaf_capacity=0):
    import torch
    n, nq = len(x), len(q_id)
    xd, yd, qd, qxd, qyd = dev(x), dev(y), dev(q_id), dev(q_x), dev(q_y)
    out_ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    out_d2 = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    desc = knnq.knn_world_desc(0.0, 0.0, 1.0, leaf_capacity, 0, 64, nq)
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    knnq.knn_query_static(desc, p(xd), p(yd), n, p(qd), p(qxd), p(qyd), nq, k, p(out_ids),
                          p(out_d2), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out_ids.cpu().numpy(), out_d2.cpu().numpy()


def same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32),
                                                         b[1].view(np.uint32))


def test_static_matches_regular_path_twice_in_a_row():
    # call 1: 60000 clustered objects, every object queries at its position, k = 16
    x1, y1 = synth.clustered_positions(60000, 21)
    q1 = np.arange(60000, dtype=np.int32)
    first = static_path(x1, y1, q1, 16)
    assert same(first, regular_path(x1, y1, q1, 16))
    # call 2: other sizes and explicit anonymous centres; the scratch still holds
    # call 1's index, which must not leak into this answer
    x2, y2 = synth.uniform_positions(30011, 22)
    r = np.random.default_rng(23)
    q2 = np.where(r.random(4099) < 0.5, -1, r.integers(0, 30011, 4099)).astype(np.int32)
    qx = r.random(4099).astype(np.float32)
    qy = r.random(4099).astype(np.float32)
    second = static_path(x2, y2, q2, 5, qx, qy, leaf_capacity=12)
    assert same(second, regular_path(x2, y2, q2, 5, qx, qy, leaf_capacity=12))
    # and call 1 again gives call 1's rows
    assert same(static_path(x1, y1, q1, 16), first)


def oracle_path(x, y, q_id, k, q_x=None, q_y=None):
    ids, d2, _ = oracle.knn(x, y, q_id, k, q_x, q_y)
    return ids, d2


def test_static_matches_oracle_directly():
    # the rows of the allocation-free call against the CPU oracle itself (Def. 1
    # brute force), not only against the regular path: issuer queries at k = 8
    # and anonymous explicit centres at k = 3
    x, y = synth.uniform_positions(12007, 31)
    q = np.arange(0, 12007, 2, dtype=np.int32)
    assert same(static_path(x, y, q, 8), oracle_path(x, y, q, 8))
    r = np.random.default_rng(32)
    qa = np.full(2000, -1, dtype=np.int32)
    qx = r.random(2000).astype(np.float32)
    qy = r.random(2000).astype(np.float32)
    assert same(static_path(x, y, qa, 3, qx, qy), oracle_path(x, y, qa, 3, qx, qy))


def test_static_many_calls_alternating_sizes():
    # every call finds the previous call's arrays at other places of the shared
    # scratch: large and small (n, n_q) alternate so that a call's scan status
    # words fall where the last call kept ids and offsets; every call must
    # still match the regular path bit for bit
    worlds = []
    for i, n in enumerate((65536, 3001, 50000, 777, 65000, 12345)):
        x, y = (synth.clustered_positions(n, 40 + i) if i % 2 == 0
                else synth.uniform_positions(n, 40 + i))
        worlds.append((x, y))
    ks = (16, 4, 8, 1, 32, 5)
    expected = {}
    for call in range(24):
        j = call % len(worlds)
        x, y = worlds[j]
        n = len(x)
        nq = n if call % 4 < 2 else max(1, n // 3)
        q = np.arange(n, dtype=np.int32)[:nq] if nq == n else \
            np.random.default_rng(100 + j).choice(n, nq, replace=False).astype(np.int32)
        got = static_path(x, y, q, ks[j])
        key = (j, nq)
        if key not in expected:
            expected[key] = regular_path(x, y, q, ks[j])
        assert same(got, expected[key]), f"call {call}: world {j}, n_q {nq}, k {ks[j]}"


def test_static_accepts_positions_not_16_byte_aligned():
    # caller arrays that start 4 bytes past a 16-byte boundary take the
    # kernels' scalar paths; the rows are the same
    import torch
    x, y = synth.uniform_positions(20003, 24)
    q = np.arange(0, 20003, 3, dtype=np.int32)
    xs = torch.zeros(len(x) + 1, dtype=torch.float32, device="cuda")
    ys = torch.zeros(len(y) + 1, dtype=torch.float32, device="cuda")
    xs[1:] = torch.from_numpy(x).cuda()
    ys[1:] = torch.from_numpy(y).cuda()
    assert (xs[1:].data_ptr() % 16) != 0
    qd = dev(q)
    out_ids = torch.empty((len(q), 8), dtype=torch.int32, device="cuda")
    out_d2 = torch.empty((len(q), 8), dtype=torch.float32, device="cuda")
    desc = knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, 64, len(q))
    knnq.knn_query_static(desc, xs[1:].data_ptr(), ys[1:].data_ptr(), len(x), qd.data_ptr(),
                          None, None, len(q), 8, out_ids.data_ptr(), out_d2.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = (out_ids.cpu().numpy(), out_d2.cpu().numpy())
    assert same(got, regular_path(x, y, q, 8))


def test_static_rejects_sizes_beyond_its_scratch():
    lib = knnq.lib()
    desc = knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, 64, 10)
    st = lib.knn_query_static(ctypes.byref(desc), 1, 1, 65537, 1, None, None, 1, 4, 1, 1, None)
    assert st == knnq.KNN_ERR_INVALID
    assert "65536" in knnq.knn_last_error()
    st = lib.knn_query_static(ctypes.byref(desc), 1, 1, 100, 1, None, None, 70000, 4, 1, 1, None)
    assert st == knnq.KNN_ERR_INVALID
