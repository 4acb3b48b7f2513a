"""The multi-rank bench path on CPU: two gloo ranks run independent replicas,
the timed region's MAX over ranks reaches every rank, and the whole-job value
is every rank's units over the slowest rank's time (no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    mine = [10.0 + 5.0 * rank, 1.0 + rank]          # this rank's timings
    got = bench.max_over_ranks(mine, dist)
    dist.barrier()
    out.put((r, w, local, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, w, loc) for r, w, loc, _ in res] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, got in res:
        assert got == [15.0, 2.0]


def test_replicas_value_is_weak_scaling():
    import bench
    assert bench.replicas_value(1, 1_000_000, 0.5) == 2_000_000
    assert bench.replicas_value(4, 1_000_000, 0.5) == 8_000_000


@pytest.mark.parametrize("env,want", [({}, (0, 1, 0)),
                                      ({"RANK": "3", "WORLD_SIZE": "8", "LOCAL_RANK": "3"},
                                       (3, 8, 3))])
def test_dist_env(monkeypatch, env, want):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    assert bench.dist_env() == want
