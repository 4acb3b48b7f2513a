"""The batched expansion of knn_batch_tick (GPU): the worlds on the gathered
form skip their own expansion and one grid per list size expands the packets
of all of them, then one packet-walk grid per list size the packets they
handed back.  Every row of every world is compared with the oracle, over a
recorded tick and a replayed one, in a batch that mixes every list-size class,
worlds that hand packets back (fewer objects than k, coincident objects),
per-query list sizes, explicit centres outside the domain, a world without
queries, a world on the packet walk (batched by its own class) and a world
that keeps its own expansion (one warp per query).  The batch autotuner is
checked for exact rows after it chose."""
import numpy as np
import pytest

import oracle
from paper_1412_6170_gb300 import knnq, synth
from tests.gpu_util import assert_rows_equal, to_dev, torch_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _specs():
    """(name, x0, y0, k, tuning, query kind, per-query k) of the batch's worlds."""
    s = []
    x, y = synth.uniform_positions(50_000, 71)
    s.append(("uniform k=16", x, y, 16, None, "all", False))
    x, y = synth.clustered_positions(30_000, 72)
    s.append(("clustered k=4", x, y, 4, None, "all", False))
    x, y = synth.uniform_positions(3, 73)
    s.append(("3 objects k=8", x, y, 8, None, "all", False))
    s.append(("coincident k=8", np.full(50, 0.25, np.float32), np.full(50, 0.75, np.float32), 8,
              None, "all", False))
    x, y = synth.clustered_positions(20_000, 74)
    s.append(("clustered k=32 per-query k", x, y, 32, None, "half", True))
    x, y = synth.clustered_positions(20_000, 75)
    s.append(("explicit centres k=16", x, y, 16, None, "explicit", False))
    x, y = synth.uniform_positions(5_000, 76)
    s.append(("gathered k=48", x, y, 48, dict(expansion=4), "all", False))
    x, y = synth.uniform_positions(5_000, 77)
    s.append(("wide k=48", x, y, 48, None, "all", False))
    x, y = synth.uniform_positions(4_000, 78)
    s.append(("no queries k=8", x, y, 8, None, "none", False))
    x, y = synth.uniform_positions(8_000, 79)
    s.append(("walk k=8", x, y, 8, dict(expansion=1), "all", False))
    x, y = synth.uniform_positions(1, 80)
    s.append(("1 object k=4", x, y, 4, None, "all", False))
    return s


def _tick_inputs(n, kind, seed, tick):
    r = np.random.default_rng(1000 * seed + tick)
    if kind == "none":
        q = np.zeros(0, np.int32)
    elif kind == "half":
        q = np.sort(r.choice(n, max(1, n // 2), replace=False)).astype(np.int32)
    else:
        q = np.arange(n, dtype=np.int32)
    qx = qy = None
    if kind == "explicit":
        qx = np.clip(r.normal(0.5, 0.4, n), -0.5, 1.5).astype(np.float32)
        qy = np.clip(r.normal(0.5, 0.4, n), -0.5, 1.5).astype(np.float32)
        q = np.where(r.random(n) < 0.3, -1, q).astype(np.int32)
    return q, qx, qy


def test_batched_expansion_every_row_against_oracle():
    torch, dev = torch_dev()
    specs = _specs()
    worlds, bufs, state = [], [], []
    try:
        for i, (name, x0, y0, k, tuning, kind, perq) in enumerate(specs):
            n = len(x0)
            w = knnq.World(to_dev(x0), to_dev(y0), k_max=max(k, 4), max_queries=max(n, 1))
            if tuning:
                w.set_tuning(**tuning)
            worlds.append(w)
            state.append((x0.copy(), y0.copy()))
            q, qx, qy = _tick_inputs(n, kind, i, 0)
            nq = q.shape[0]
            qk = np.random.default_rng(500 + i).integers(0, k + 1, nq).astype(np.int32) \
                if perq else None
            bufs.append({"q": to_dev(q), "qx": to_dev(qx), "qy": to_dev(qy), "qk": to_dev(qk),
                         "uid": to_dev(np.arange(n, dtype=np.int32)),
                         "ux": to_dev(x0), "uy": to_dev(y0),
                         "oi": torch.empty((nq, k), dtype=torch.int32, device=dev),
                         "od": torch.empty((nq, k), dtype=torch.float32, device=dev),
                         "qk_np": qk, "q_np": q, "qx_np": qx, "qy_np": qy})
        handed_back = {}
        for tick in range(2):
            args = []
            for i, ((name, x0, y0, k, tuning, kind, perq), b) in enumerate(zip(specs, bufs)):
                n = len(x0)
                ux, uy = synth.random_walk(state[i][0], state[i][1], 1e-3, 90 + i, tick)
                b["ux"].copy_(to_dev(ux))
                b["uy"].copy_(to_dev(uy))
                q = b["q"] if b["q_np"].shape[0] else None
                args.append(knnq.tick_args(k, q, b["uid"], b["ux"], b["uy"], q_x=b["qx"],
                                           q_y=b["qy"], out_ids=b["oi"], out_d2=b["od"],
                                           q_k=b["qk"]))
                state[i] = (ux, uy)
            # tick 0 records the batch, tick 1 replays the recording
            knnq.knn_batch_tick([w.handle for w in worlds], args,
                                torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            for i, ((name, x0, y0, k, tuning, kind, perq), b, w) in enumerate(
                    zip(specs, bufs, worlds)):
                assert w.status()[0] == knnq.KNN_OK, (name, w.status())
                if b["q_np"].shape[0] == 0:
                    continue
                x, y = state[i]
                rid, rd2, _ = oracle.knn(x, y, b["q_np"], k, b["qx_np"], b["qy_np"])
                if perq:
                    keep = np.arange(k)[None, :] < b["qk_np"][:, None]
                    rid = np.where(keep, rid, -1).astype(np.int32)
                    rd2 = np.where(keep, rd2, np.float32(np.inf)).astype(np.float32)
                assert_rows_equal(b["oi"].cpu().numpy(), b["od"].cpu().numpy(), rid, rd2,
                                  what=f"{name} tick {tick}")
                handed_back[name] = w.expand_info()["handed_back"]
        # the worlds that cannot fill their lists went through the batched walk
        assert handed_back["3 objects k=8"] > 0, handed_back
        assert handed_back["1 object k=4"] > 0, handed_back
    finally:
        for w in worlds:
            w.close()


def test_batched_expansion_many_small_worlds_replays():
    # 64 small worlds of all list sizes, three ticks (record, replay, replay):
    # the batched rows equal separate knn_tick calls on twin worlds
    torch, dev = torch_dev()
    ws = synth.many_worlds(n_worlds=64, seed=11, n_lo=100, n_hi=20_000, ticks=3,
                           query_frac=(0.2, 1.0))
    batched = [knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n) for w in ws]
    single = [knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n) for w in ws]
    try:
        bufs = []
        for w in ws:
            t = w.ticks[0]
            bufs.append({"uid": to_dev(t.upd_id), "ux": to_dev(t.upd_x), "uy": to_dev(t.upd_y),
                         "q": to_dev(t.q_id),
                         "oi": torch.empty((t.q_id.shape[0], w.k), dtype=torch.int32, device=dev),
                         "od": torch.empty((t.q_id.shape[0], w.k), dtype=torch.float32,
                                           device=dev)})
        for ti in range(3):
            args = []
            for w, b in zip(ws, bufs):
                t = w.ticks[ti]
                b["ux"].copy_(to_dev(t.upd_x))
                b["uy"].copy_(to_dev(t.upd_y))
                args.append(knnq.tick_args(w.k, b["q"], b["uid"], b["ux"], b["uy"],
                                           out_ids=b["oi"], out_d2=b["od"]))
            knnq.knn_batch_tick([bw.handle for bw in batched], args,
                                torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            for i, (w, b) in enumerate(zip(ws, bufs)):
                t = w.ticks[ti]
                ids, d2 = single[i].tick(w.k, b["q"], to_dev(t.upd_id), to_dev(t.upd_x),
                                         to_dev(t.upd_y))
                torch.cuda.synchronize()
                assert_rows_equal(b["oi"].cpu().numpy(), b["od"].cpu().numpy(),
                                  ids.cpu().numpy(), d2.cpu().numpy(),
                                  what=f"world {i} tick {ti}")
    finally:
        for w in batched + single:
            w.close()


def test_batch_autotune_keeps_rows_exact_and_settings():
    # the batch autotuner times whole batches per list-size class; whatever it
    # keeps, the next batch's rows still match the oracle and each world's
    # settings are the ones it reported
    torch, dev = torch_dev()
    ws = synth.many_worlds(n_worlds=16, seed=21, n_lo=500, n_hi=40_000, ticks=2,
                           query_frac=(0.5, 1.0))
    worlds = [knnq.World(to_dev(w.x0), to_dev(w.y0), k_max=32, max_queries=w.n) for w in ws]
    try:
        bufs, args = [], []
        for w in ws:
            t = w.ticks[0]
            b = {"uid": to_dev(t.upd_id), "ux": to_dev(t.upd_x), "uy": to_dev(t.upd_y),
                 "q": to_dev(t.q_id),
                 "oi": torch.empty((t.q_id.shape[0], w.k), dtype=torch.int32, device=dev),
                 "od": torch.empty((t.q_id.shape[0], w.k), dtype=torch.float32, device=dev)}
            bufs.append(b)
            args.append(knnq.tick_args(w.k, b["q"], b["uid"], b["ux"], b["uy"], out_ids=b["oi"],
                                       out_d2=b["od"]))
        s = torch.cuda.current_stream().cuda_stream
        chosen = knnq.knn_batch_autotune([w.handle for w in worlds], args, trials=1, stream=s)
        assert len(chosen) == len(ws)
        for w, c, spec in zip(worlds, chosen, ws):
            t = w.get_tuning(spec.n, spec.k)
            if c["leaf_capacity"] > 0:
                assert t["leaf_capacity"] == c["leaf_capacity"], (t, c)
            assert c["expansion"] in (0, 1, 2, 4), c
        knnq.knn_batch_tick([w.handle for w in worlds], args, s)
        torch.cuda.synchronize()
        for i, (w, b) in enumerate(zip(ws, bufs)):
            t = w.ticks[0]
            x, y, _ = oracle.apply_updates(w.x0, w.y0, t.upd_id, t.upd_x, t.upd_y)
            rid, rd2, _ = oracle.knn(x, y, t.q_id, w.k)
            assert_rows_equal(b["oi"].cpu().numpy(), b["od"].cpu().numpy(), rid, rd2,
                              what=f"tuned world {i}")
            assert worlds[i].status()[0] == knnq.KNN_OK
    finally:
        for w in worlds:
            w.close()


def test_batch_after_a_world_is_replaced():
    # a batch recorded with world B, then B destroyed and a new world of the
    # same size created (possibly at the same handle address) and batched with
    # the same argument buffers: the batch is recorded again, rows stay exact
    torch, dev = torch_dev()
    r = np.random.default_rng(31)
    n = 20_000
    xa, ya = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    xb, yb = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
    q = to_dev(np.arange(n, dtype=np.int32))
    out = [(torch.empty((n, 8), dtype=torch.int32, device=dev),
            torch.empty((n, 8), dtype=torch.float32, device=dev)) for _ in range(2)]
    args = [knnq.tick_args(8, q, out_ids=o[0], out_d2=o[1]) for o in out]
    a = knnq.World(to_dev(xa), to_dev(ya), k_max=8, max_queries=n)
    b = knnq.World(to_dev(xb), to_dev(yb), k_max=8, max_queries=n)
    try:
        s = torch.cuda.current_stream().cuda_stream
        knnq.knn_batch_tick([a.handle, b.handle], args, s)
        torch.cuda.synchronize()
        b.close()
        xc, yc = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
        b = knnq.World(to_dev(xc), to_dev(yc), k_max=8, max_queries=n)
        for _ in range(2):
            knnq.knn_batch_tick([a.handle, b.handle], args, s)
            torch.cuda.synchronize()
            for (x, y), (oi, od) in zip(((xa, ya), (xc, yc)), out):
                rid, rd2, _ = oracle.knn(x, y, np.arange(n, dtype=np.int32), 8)
                assert_rows_equal(oi.cpu().numpy(), od.cpu().numpy(), rid, rd2)
    finally:
        a.close()
        b.close()


def test_batch_of_more_than_1024_worlds_in_one_class():
    # the device prefix over a class's worlds runs 1024 worlds at a time: 1100
    # small worlds of one list size, every row against the oracle
    torch, dev = torch_dev()
    r = np.random.default_rng(41)
    nw = 1100
    sizes = r.integers(20, 120, nw)
    worlds, data = [], []
    try:
        for i, n in enumerate(sizes):
            x, y = r.random(n).astype(np.float32), r.random(n).astype(np.float32)
            q = np.arange(n, dtype=np.int32)
            oi = torch.empty((n, 4), dtype=torch.int32, device=dev)
            od = torch.empty((n, 4), dtype=torch.float32, device=dev)
            worlds.append(knnq.World(to_dev(x), to_dev(y), k_max=4, max_queries=int(n)))
            data.append((x, y, q, to_dev(q), oi, od))
        args = [knnq.tick_args(4, dq, out_ids=oi, out_d2=od) for (_, _, _, dq, oi, od) in data]
        s = torch.cuda.current_stream().cuda_stream
        for _ in range(2):  # recorded, then replayed
            knnq.knn_batch_tick([w.handle for w in worlds], args, s)
            torch.cuda.synchronize()
        for i, (x, y, q, _, oi, od) in enumerate(data):
            rid, rd2, _ = oracle.knn(x, y, q, 4)
            assert_rows_equal(oi.cpu().numpy(), od.cpu().numpy(), rid, rd2, what=f"world {i}")
    finally:
        for w in worlds:
            w.close()
