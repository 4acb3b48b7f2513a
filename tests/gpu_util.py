"""Helpers for the GPU parity tests: run ticks through the C ABI and compare
with the oracle element by element (ids equal, squared distances equal as bit
patterns)."""
import numpy as np

import oracle


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a):
    torch, dev = torch_dev()
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def make_world(x0, y0, k_max=64, max_queries=None, **kw):
    from paper_1412_6170_gb300 import knnq
    return knnq.World(to_dev(x0), to_dev(y0), k_max=k_max, max_queries=max_queries, **kw)


def gpu_tick(world, t, k=None):
    """Run one synth.Tick through knn_tick; returns numpy (ids, d2)."""
    torch, _ = torch_dev()
    k = t.k if k is None else k
    ids, d2 = world.tick(k, to_dev(t.q_id), to_dev(t.upd_id), to_dev(t.upd_x),
                         to_dev(t.upd_y), to_dev(t.q_x), to_dev(t.q_y))
    torch.cuda.synchronize()
    if ids is None:
        return None, None
    return ids.cpu().numpy(), d2.cpu().numpy()


def assert_rows_equal(ids, d2, rid, rd2, rows=None, what=""):
    if rows is not None:
        ids, d2 = ids[rows], d2[rows]
    assert ids.shape == rid.shape, (ids.shape, rid.shape)
    bad = np.flatnonzero(~(np.all(ids == rid, axis=1)
                           & np.all(d2.view(np.uint32) == rd2.view(np.uint32), axis=1)))
    if bad.size:
        r = bad[0]
        raise AssertionError(
            f"{what}: {bad.size} rows differ; first row {r if rows is None else rows[r]}:\n"
            f" gpu ids {ids[r].tolist()}\n oracle  {rid[r].tolist()}\n"
            f" gpu d2 {d2[r].tolist()}\n oracle  {rd2[r].tolist()}")


def sample_rows(n_q, count, seed=0):
    """Sampled query rows: the first and last rows plus a seeded random subset."""
    if count >= n_q:
        return np.arange(n_q)
    r = np.random.default_rng(seed)
    s = np.unique(np.concatenate([np.arange(min(64, n_q)), np.arange(max(0, n_q - 64), n_q),
                                  r.choice(n_q, count, replace=False)]))
    return s


def oracle_rows(x, y, t, rows, k=None):
    k = t.k if k is None else k
    qx = None if t.q_x is None else t.q_x[rows]
    qy = None if t.q_y is None else t.q_y[rows]
    ids, d2, _ = oracle.knn(x, y, t.q_id[rows], k, qx, qy)
    return ids, d2
