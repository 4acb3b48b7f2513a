"""Batched multi-world ticks (knn_batch_tick) and the autotuner (GPU): the rows
are bit-identical to separate knn_tick calls and to the oracle."""
import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import knnq, synth
from tests.gpu_util import assert_rows_equal, sample_rows, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_batch_matches_single_ticks_and_oracle():
    torch, dev = torch_dev()
    ws = synth.many_worlds(n_worlds=24, seed=3, n_lo=50, n_hi=30000, ticks=3,
                           query_frac=(0.3, 1.0))
    batched = [knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n) for w in ws]
    single = [knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n) for w in ws]
    try:
        # fixed input/output buffers per world (reused by the first two ticks, so
        # the second batch call replays the recorded graph)
        bufs = []
        for w in ws:
            t = w.ticks[0]
            bufs.append({"uid": to_dev(t.upd_id), "ux": to_dev(t.upd_x), "uy": to_dev(t.upd_y),
                         "q": to_dev(t.q_id),
                         "oi": torch.empty((t.q_id.shape[0], w.k), dtype=torch.int32, device=dev),
                         "od": torch.empty((t.q_id.shape[0], w.k), dtype=torch.float32, device=dev)})
        xs = [(w.x0.copy(), w.y0.copy()) for w in ws]
        for ti in range(3):
            if ti == 2:  # new buffers: the batch is recorded again
                bufs = [{kk: v.clone() for kk, v in b.items()} for b in bufs]
            args = []
            for w, b in zip(ws, bufs):
                t = w.ticks[ti]
                b["ux"].copy_(to_dev(t.upd_x))
                b["uy"].copy_(to_dev(t.upd_y))
                if t.q_id.shape[0] == b["q"].shape[0]:
                    b["q"].copy_(to_dev(t.q_id))
                args.append(knnq.tick_args(w.k, b["q"], b["uid"], b["ux"], b["uy"],
                                           out_ids=b["oi"], out_d2=b["od"]))
            knnq.knn_batch_tick([bw.handle for bw in batched], args,
                                torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            for i, (w, b) in enumerate(zip(ws, bufs)):
                t = w.ticks[ti]
                q = b["q"].cpu().numpy()
                ids, d2 = single[i].tick(w.k, b["q"], to_dev(t.upd_id), to_dev(t.upd_x),
                                         to_dev(t.upd_y))
                torch.cuda.synchronize()
                gi, gd = b["oi"].cpu().numpy(), b["od"].cpu().numpy()
                assert np.array_equal(gi, ids.cpu().numpy()), f"world {i} tick {ti}"
                assert np.array_equal(gd.view(np.uint32), d2.cpu().numpy().view(np.uint32))
                x, y, _ = oracle.apply_updates(xs[i][0], xs[i][1], t.upd_id, t.upd_x, t.upd_y)
                xs[i] = (x, y)
                rows = sample_rows(q.shape[0], 300, seed=i)
                rid, rd2, _ = oracle.knn(x, y, q[rows], w.k)
                assert_rows_equal(gi, gd, rid, rd2, rows, what=f"world {i} tick {ti}")
        for bw in batched:
            assert bw.status()[0] == knnq.KNN_OK
    finally:
        for w in batched + single:
            w.close()


def test_autotune_keeps_results_exact():
    torch, dev = torch_dev()
    w = synth.skewed_moving(n=80000, k=16, ticks=1, seed=5, query_frac=0.5)
    t = w.ticks[0]
    world = knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=16, max_queries=t.q_id.shape[0])
    try:
        q = to_dev(t.q_id)
        chosen = world.autotune(16, q, trials=1)
        assert chosen["leaf_capacity"] > 0 and chosen["grid_level"] > 0
        assert world.get_tuning(t.q_id.shape[0], 16)["leaf_capacity"] == chosen["leaf_capacity"]
        ids, d2 = world.tick(16, q, to_dev(t.upd_id), to_dev(t.upd_x), to_dev(t.upd_y))
        torch.cuda.synchronize()
        x, y, _ = oracle.apply_updates(w.x0, w.y0, t.upd_id, t.upd_x, t.upd_y)
        rows = sample_rows(t.q_id.shape[0], 4000)
        rid, rd2, _ = oracle.knn(x, y, t.q_id[rows], 16)
        assert_rows_equal(ids.cpu().numpy(), d2.cpu().numpy(), rid, rd2, rows, what="autotuned")
    finally:
        world.close()


def test_batch_rejects_bad_lists():
    torch, dev = torch_dev()
    x = to_dev(np.random.default_rng(0).random(100).astype(np.float32))
    w = knnq.World(x, x, k_max=4, max_queries=100)
    try:
        a = knnq.tick_args(4, to_dev(np.arange(10, dtype=np.int32)),
                           out_ids=torch.empty((10, 4), dtype=torch.int32, device=dev),
                           out_d2=torch.empty((10, 4), dtype=torch.float32, device=dev))
        with pytest.raises(knnq.KnnError):
            knnq.knn_batch_tick([w.handle, w.handle], [a, a])
        bad = knnq.tick_args(5, to_dev(np.arange(10, dtype=np.int32)))
        with pytest.raises(knnq.KnnError):
            knnq.knn_batch_tick([w.handle], [bad])
    finally:
        w.close()
