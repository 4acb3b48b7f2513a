"""Benchmark: per-tick k-NN spatial join on 1M moving objects, k = 16.

Workload (one "step" = one tick = every hot-path stage): 1,000,000 objects
uniform in [0,1)^2 (seed 0); each tick every object moves by N(0, 1e-3) per
coordinate (clamped) and every object issues a k=16 query at its own position.
Ten ticks are generated once and stay resident in HBM; steps cycle through
them.  The L2 cache is flushed (a 256 MiB write) between timed steps, outside
the timed events.

Prints one JSON line.  ``e2e`` is the same metric through the host-buffer
API: pinned host arrays, every step's inputs copied in and rows copied out
inside the timed region, two ticks in flight (knn_tick_host_submit /
knn_tick_host_wait); ``e2e.by_mode`` adds the synchronous knn_tick_host.
``roofline`` reports the expansion kernel against the measured HBM copy
bandwidth and against instruction issue.  ``--impl reference`` times the CPU
oracle (brute force on the host cores) on a bounded sample of the same
workload instead.
Under torchrun each rank runs an independent replica of the workload on its
own GPU ("replicas only": one world does not shard); value = all ranks'
queries / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "queries/s (1M obj, k=16) + p99 tick latency: served vs plain, ids exact"
N_OBJ = 1_000_000
K = 16
N_TICKS = 10
WORKLOAD = "uniform 1M objects, k=16, all objects query, N(0,1e-3) moves, 10 ticks cycled"
# Algorithmic bytes per query of the expansion kernel (query 12 B + each object
# read once amortised 12 B * n/q + k results of 8 B).
ALGO_BYTES_PER_QUERY = 12 + 12 * N_OBJ / N_OBJ + 8 * K
FALLBACK_HBM_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback"


def expand_profile(kernel="k_expand_gather", source="knn_expand_gather.cu"):
    """Per-launch DRAM traffic and ALU-pipe use of the expansion kernel from the
    committed ncu summary, or None when the kernel source changed since that capture."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", f"{kernel}_uniform1M_k16.md")
    src = os.path.join(ROOT, "paper_1412_6170_gb300", "csrc", source)
    try:
        text = open(prof).read()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if re.search(r"source sha256[^:]*: *([0-9a-f]{16})", text).group(1) != h:
            return None
        traffic = int(re.search(r"traffic_bytes_per_launch: *(\d+)", text).group(1))
        alu = float(re.search(r"sm__inst_executed_pipe_alu[^|]*\| *([0-9.]+)", text).group(1))
        inst = int(re.search(r"warp_instructions_per_launch: *(\d+)", text).group(1))
        return {"traffic": traffic, "alu_pipe_pct": alu, "warp_inst": inst}
    except Exception:  # noqa: BLE001
        return None


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of per-rank timings (a barrier-synchronised MAX
    all-reduce; the data path itself has no collective)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]


def replicas_value(n_ranks, units_per_rank, max_seconds):
    """Whole-job throughput of independent replicas: every rank's units over the
    slowest rank's time (weak scaling)."""
    return n_ranks * units_per_rank / max_seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(workload, target_s: float = 12.0):
    """Time the oracle (brute force over all objects, all host cores) on a bounded
    sample of tick 1's queries; returns the cpu_baseline object."""
    import numpy as np

    import oracle
    t = workload.ticks[0]
    x, y, _ = oracle.apply_updates(workload.x0, workload.y0, t.upd_id, t.upd_x, t.upd_y)
    cores = os.cpu_count() or 1
    probe = min(t.q_id.shape[0], max(256, 32 * cores))
    t0 = time.perf_counter()
    oracle.knn(x, y, t.q_id[:probe], t.k)
    dt = time.perf_counter() - t0
    count = int(min(t.q_id.shape[0], max(probe, probe * target_s / max(dt, 1e-3))))
    rows = np.linspace(0, t.q_id.shape[0] - 1, count).astype(np.int64)
    t0 = time.perf_counter()
    oracle.knn(x, y, t.q_id[rows], t.k)
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{count} of tick 1's {t.q_id.shape[0]} queries (evenly spaced), "
                      f"brute force over all {workload.n} objects, {dt:.1f} s"}


def pct(v, q):
    v = sorted(float(x) for x in v)
    return v[min(len(v) - 1, int(round(q * (len(v) - 1))))]


def _json_default(o):
    """numpy scalars (and anything else with .item()) as plain JSON values."""
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(f"not JSON serializable: {type(o).__name__}")


def _spawn_map(fn, items):
    """Map over a spawn-context process pool (the GPU is in use in this process, so
    workers must not be forked from it)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)),
                                mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items))


def rows_vs_oracle(x, y, q_id, k, ids, d2, count=256, seed=0):
    """Sampled rows of one tick (numpy ids/d2 for all of q_id) against the oracle."""
    import numpy as np

    import oracle
    r = np.random.default_rng(seed)
    rows = np.unique(r.choice(q_id.shape[0], min(count, q_id.shape[0]), replace=False))
    rid, rd2, _ = oracle.knn(x, y, q_id[rows], k)
    return bool(np.array_equal(ids[rows], rid)
                and np.array_equal(d2[rows].view(np.uint32), rd2.view(np.uint32)))


def serving_config5(dev, n_worlds=64, loads=(0.5, 0.8, 0.95), n_req=1000, n_slots=8, seed=5,
                    check=True):
    """The serving workload: a Poisson stream of tick requests over 64 resident
    clustered worlds (10k-4M objects, k up to 64, 10-100 % of the objects query),
    served by the request loop under a device-memory budget below the worlds'
    total tick scratch (admission evicts idle worlds' scratch), against the same
    requests run one knn_tick at a time (plain).  Each request is a tick of one
    world: every object moves, a subset queries.  Offered loads are fractions of
    the plain capacity (1 / mean plain service time)."""
    import numpy as np
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    from functools import partial
    wl = _spawn_map(partial(synth.serving_world, seed=seed, n_worlds=n_worlds), range(n_worlds))
    ws = []
    for w in wl:
        t = w.ticks[0]
        x0, y0 = torch.from_numpy(w.x0).to(dev), torch.from_numpy(w.y0).to(dev)
        nq = t.q_id.shape[0]
        ws.append({"n": w.n, "k": w.k, "x": x0, "y": y0,
                   "ids": torch.from_numpy(t.upd_id).to(dev),
                   # two position sets used in turn: the tick's moves, then back
                   "pos": [(torch.from_numpy(t.upd_x).to(dev), torch.from_numpy(t.upd_y).to(dev)),
                           (x0, y0)],
                   "q": torch.from_numpy(t.q_id).to(dev),
                   "oi": torch.empty((nq, w.k), dtype=torch.int32, device=dev),
                   "od": torch.empty((nq, w.k), dtype=torch.float32, device=dev)})
    stream = torch.cuda.current_stream()
    total_q = sum(int(d["q"].shape[0]) for d in ws)

    def args_for(i, parity, out=None):
        d = ws[i]
        ux, uy = d["pos"][parity]
        oi, od = out if out is not None else (d["oi"], d["od"])
        return knnq.tick_args(d["k"], d["q"], d["ids"], ux, uy, out_ids=oi, out_d2=od)

    def plain_tick(worlds, i, a):
        knnq.knn_tick(worlds[i].handle, a.upd_id_dev, a.upd_x_dev, a.upd_y_dev, a.n_upd,
                      a.q_id_dev, None, None, a.n_q, a.k, a.out_ids_dev, a.out_d2_dev,
                      stream.cuda_stream)

    # plain service time of every world (graphs recorded first)
    plain = [knnq.World(d["x"], d["y"], k_max=d["k"], max_queries=d["n"]) for d in ws]
    for i in range(n_worlds):
        for par in (0, 1, 0, 1):
            plain_tick(plain, i, args_for(i, par))
    torch.cuda.synchronize()
    svc = []
    for i in range(n_worlds):
        t0 = time.perf_counter()
        plain_tick(plain, i, args_for(i, 0))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        plain_tick(plain, i, args_for(i, 1))
        torch.cuda.synchronize()
        svc.append(0.5 * (time.perf_counter() - t0))
        del t1
    mean_service = float(np.mean(svc))

    # request streams: a world drawn uniformly per request, Poisson arrivals
    plans = {}
    for li, load in enumerate(loads):
        r = np.random.default_rng(seed * 1000 + li)
        who = r.integers(0, n_worlds, n_req)
        gaps = r.exponential(mean_service / load, n_req)
        checked = set(int(v) for v in np.linspace(n_req // 8, n_req - 1, 4).astype(int))
        plans[load] = (who, np.cumsum(gaps) - gaps[0], checked)
    outs = {}  # (load, request) -> dedicated output tensors of a checked request

    def out_for(load, j, i):
        key = (load, j)
        if key not in outs:
            d = ws[i]
            outs[key] = {"plain": (torch.empty_like(d["oi"]), torch.empty_like(d["od"])),
                         "served": (torch.empty_like(d["oi"]), torch.empty_like(d["od"]))}
        return outs[key]

    def spin_until(t_abs):
        while time.perf_counter() < t_abs:
            pass

    parity = [0] * n_worlds
    results = {}
    for load in loads:
        who, arrive, checked = plans[load]
        par_seq = []
        for j in range(n_req):
            i = int(who[j])
            par_seq.append(parity[i])
            parity[i] ^= 1
        plans[load] = (who, arrive, checked, par_seq)
        for j in checked:  # graphs of the checked requests' own outputs, before timing
            i = int(who[j])
            plain[i].record_tick(ws[i]["k"], ws[i]["q"], ws[i]["ids"], *ws[i]["pos"][par_seq[j]],
                                 out_ids=out_for(load, j, i)["plain"][0],
                                 out_d2=out_for(load, j, i)["plain"][1])
        lat = []
        t_base = time.perf_counter() + 0.01
        for j in range(n_req):
            i = int(who[j])
            spin_until(t_base + arrive[j])
            o = out_for(load, j, i)["plain"] if j in checked else None
            plain_tick(plain, i, args_for(i, par_seq[j], o))
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - (t_base + arrive[j]))
        span = time.perf_counter() - t_base
        q = sum(int(ws[int(i)]["q"].shape[0]) for i in who)
        results[load] = {"plain": {"p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99),
                                   "queries_per_s_at_load": q / span}}
    # plain saturated: every request of the 0.8 stream back to back
    who, _, _, par_seq = plans[loads[len(loads) // 2]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(n_req):
        plain_tick(plain, int(who[j]), args_for(int(who[j]), par_seq[j]))
    torch.cuda.synchronize()
    sat_plain = time.perf_counter() - t0
    q_sat = sum(int(ws[int(i)]["q"].shape[0]) for i in who)
    for w in plain:
        w.close()
    del plain
    torch.cuda.synchronize()

    # the total tick scratch of the worlds, then a budget below it
    probe = knnq.knn_server_create(n_slots, 0)
    idx = [knnq.knn_server_add_world(probe, knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, d["k"],
                                                                d["n"]),
                                     d["x"].data_ptr(), d["y"].data_ptr(), d["n"]) for d in ws]
    for r in [knnq.knn_server_submit(probe, idx[i], args_for(i, 1)) for i in range(n_worlds)]:
        knnq.knn_server_wait(probe, r)
    st0 = knnq.knn_server_stats(probe)
    knnq.knn_server_destroy(probe)
    total_scratch = int(st0["scratch_bytes"])
    budget = max(int(1.5 * st0["largest_world_scratch"]), int(0.35 * total_scratch))
    srv = knnq.knn_server_create(n_slots, budget)
    idx = [knnq.knn_server_add_world(srv, knnq.knn_world_desc(0.0, 0.0, 1.0, 0, 0, d["k"], d["n"]),
                                     d["x"].data_ptr(), d["y"].data_ptr(), d["n"]) for d in ws]
    # warm-up: every world once on each position set (the worlds end where the
    # plain ones started each stream: parity bookkeeping as in the plain runs)
    for par in (0, 1):
        for r in [knnq.knn_server_submit(srv, idx[i], args_for(i, par)) for i in range(n_worlds)]:
            knnq.knn_server_wait(srv, r)
    base = knnq.knn_server_stats(srv)
    for load in loads:
        who, arrive, checked, par_seq = plans[load]
        before = knnq.knn_server_stats(srv)
        rids = []
        t_base = time.perf_counter() + 0.01
        for j in range(n_req):
            i = int(who[j])
            spin_until(t_base + arrive[j])
            o = out_for(load, j, i)["served"] if j in checked else None
            rids.append(knnq.knn_server_submit(srv, idx[i], args_for(i, par_seq[j], o)))
        lat = [knnq.knn_server_wait(srv, r) / 1e3 for r in rids]
        span = time.perf_counter() - t_base
        after = knnq.knn_server_stats(srv)
        q = sum(int(ws[int(i)]["q"].shape[0]) for i in who)
        results[load]["served"] = {"p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99),
                                   "queries_per_s_at_load": q / span,
                                   "admitted": after["admitted"] - before["admitted"],
                                   "evictions": after["evictions"] - before["evictions"]}
    who, _, _, par_seq = plans[loads[len(loads) // 2]]
    t0 = time.perf_counter()
    rids = [knnq.knn_server_submit(srv, idx[int(who[j])], args_for(int(who[j]), par_seq[j]))
            for j in range(n_req)]
    for r in rids:
        knnq.knn_server_wait(srv, r)
    sat_served = time.perf_counter() - t0
    st = knnq.knn_server_stats(srv)
    status_ok = all(knnq.knn_server_world_status(srv, j)[0] == knnq.KNN_OK for j in idx)
    knnq.knn_server_destroy(srv)
    torch.cuda.synchronize()

    # checked requests: served rows = plain rows, and sampled rows = the oracle
    same = True
    oracle_ok = True if check else None
    n_checked = 0
    for (load, j), o in outs.items():
        who, _, _, par_seq = plans[load]
        i = int(who[j])
        pi, pd = (t.cpu().numpy() for t in o["plain"])
        si, sd = (t.cpu().numpy() for t in o["served"])
        same = same and np.array_equal(pi, si) and np.array_equal(pd.view(np.uint32),
                                                                  sd.view(np.uint32))
        if check:
            w = wl[i]
            x, y = (w.ticks[0].upd_x, w.ticks[0].upd_y) if par_seq[j] == 0 else (w.x0, w.y0)
            oracle_ok = oracle_ok and rows_vs_oracle(x, y, w.ticks[0].q_id, w.k, si, sd,
                                                     count=128, seed=j)
        n_checked += 1
    for load in loads:
        results[load]["served_beats_plain_p99"] = \
            results[load]["served"]["p99_ms"] < results[load]["plain"]["p99_ms"]
    return {
        "workload": f"{n_worlds} resident clustered worlds, {sum(d['n'] for d in ws)} objects "
                    f"(10k-4M each, log-uniform), k in {{4,8,16,32,64}}, 10-100 % querying "
                    f"({total_q} queries if every world ticks once); {n_req} Poisson tick "
                    f"requests per offered load, a world drawn uniformly per request",
        "plain_mean_service_ms": 1e3 * mean_service,
        "served_config": {"stream_slots": n_slots, "hbm_budget_bytes": budget,
                          "worlds_total_scratch_bytes": total_scratch,
                          "largest_world_scratch_bytes": int(st0["largest_world_scratch"])},
        "by_load": {str(load): results[load] for load in loads},
        "saturated_queries_per_s": {"served": q_sat / sat_served, "plain": q_sat / sat_plain},
        "server_totals": {"admitted": st["admitted"] - base["admitted"],
                          "evictions": st["evictions"] - base["evictions"],
                          "completed": st["completed"]},
        "rows_checked": {"requests": n_checked, "served_equals_plain": bool(same),
                         "sampled_rows_equal_oracle": oracle_ok, "device_status_ok": status_ok},
    }


def skewed_config3(dev, ticks=10, rounds=3, seed=0, check=True):
    """The skewed workload: 4M objects, 90 % in 64 Gaussian hotspots, a fresh random
    25 % querying each tick, k = 32, N(0, 5e-4) moves; the ten ticks are replayed
    `rounds` times (each tick sets every position, so a replay is a valid tick) for
    per-tick latency, with per-stage events for the expansion's roofline."""
    import numpy as np
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    k, n = 32, 4_000_000
    w = synth.skewed_moving(n=n, k=k, ticks=ticks, seed=seed)
    x0, y0 = torch.from_numpy(w.x0).to(dev), torch.from_numpy(w.y0).to(dev)
    ids = torch.from_numpy(w.ticks[0].upd_id).to(dev)
    tk = [(torch.from_numpy(t.upd_x).to(dev), torch.from_numpy(t.upd_y).to(dev),
           torch.from_numpy(t.q_id).to(dev)) for t in w.ticks]
    nq = w.ticks[0].q_id.shape[0]
    oi = torch.empty((nq, k), dtype=torch.int32, device=dev)
    od = torch.empty((nq, k), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    world = knnq.World(x0, y0, k_max=k, max_queries=nq)
    world.set_profiling(True)
    stream = torch.cuda.current_stream()
    try:
        for t in range(ticks):  # warm-up: records the tick graphs
            world.tick(k, tk[t][2], ids, tk[t][0], tk[t][1], out_ids=oi, out_d2=od)
        torch.cuda.synchronize()
        ms, exp_ms = [], []
        for r in range(rounds):
            for t in range(ticks):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                world.tick(k, tk[t][2], ids, tk[t][0], tk[t][1], out_ids=oi, out_d2=od)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
                st_k = world.stage_times()
                exp_ms.append(st_k["expand"] + st_k["pass-on"])
        ok = None
        if check:
            t = w.ticks[ticks - 1]
            ok = rows_vs_oracle(t.upd_x, t.upd_y, t.q_id, k, oi.cpu().numpy(), od.cpu().numpy(),
                                count=2000, seed=3)
        info = world.expand_info()
        st = world.status()[0]
    finally:
        world.close()
    hbm, hbm_kind = peaks()
    bpq = 12 + 12 * n / nq + 8 * k
    e = statistics.median(exp_ms)
    return {"workload": f"{n} objects, 90% in 64 Gaussian hotspots (sigma 0.01), a random 25% "
                        f"({nq}) query each tick, k={k}, N(0,5e-4) moves, {ticks} ticks x "
                        f"{rounds} rounds, L2 flushed between ticks",
            "queries_per_s": nq * len(ms) / (sum(ms) / 1e3),
            "ms_per_tick": sum(ms) / len(ms), "p50_tick_ms": pct(ms, 0.5),
            "p99_tick_ms": pct(ms, 0.99), "ticks_timed": len(ms),
            "expand_ms": e,
            "expand_roofline": {"algorithmic_bytes_per_query": bpq,
                                "achieved_gbs": bpq * nq / (e / 1e3) / 1e9, "peak_gbs": hbm,
                                "peak_kind": hbm_kind,
                                "frac": bpq * nq / (e / 1e3) / 1e9 / hbm},
            "expand_form": info, "rows_vs_oracle": ok, "device_status_ok": st == knnq.KNN_OK}


def index_reuse_vs_rebuild(dev, ticks=20, max_age=8):
    """The headline workload with the paper's index reuse (leaves kept across ticks,
    rebuilt at least every max_age + 1 ticks) against a rebuild every tick; same
    moves, same rows (checked here on the last tick)."""
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    wl = synth.plain_uniform_moving(n=N_OBJ, k=K, ticks=N_TICKS, seed=0)
    ids = torch.from_numpy(wl.ticks[0].upd_id).to(dev)
    ux = [torch.from_numpy(t.upd_x).to(dev) for t in wl.ticks]
    uy = [torch.from_numpy(t.upd_y).to(dev) for t in wl.ticks]
    stream = torch.cuda.current_stream()
    out = {}
    rows = {}
    for name, age in (("rebuild every tick", 0), (f"reuse, max_age {max_age}", max_age)):
        x0, y0 = torch.from_numpy(wl.x0).to(dev), torch.from_numpy(wl.y0).to(dev)
        world = knnq.World(x0, y0, k_max=K, max_queries=N_OBJ)
        world.set_index_reuse(age)
        oi = torch.empty((N_OBJ, K), dtype=torch.int32, device=dev)
        od = torch.empty((N_OBJ, K), dtype=torch.float32, device=dev)
        try:
            for i in range(3):
                world.tick(K, ids, ids, ux[i % N_TICKS], uy[i % N_TICKS], out_ids=oi, out_d2=od)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(3, 3 + ticks):
                world.tick(K, ids, ids, ux[i % N_TICKS], uy[i % N_TICKS], out_ids=oi, out_d2=od)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / ticks
            out[name] = {"tick_ms": ms, "queries_per_s": N_OBJ / (ms * 1e-3)}
            rows[name] = (oi.cpu(), od.cpu())
        finally:
            world.close()
    a, b = rows.values()
    same = bool(torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32),
                                                        b[1].view(torch.int32)))
    return {"workload": f"{WORKLOAD}; {ticks} back-to-back ticks (no L2 flush)",
            "per_mode": out, "rows_identical": same}


def expansion_ablation(dev, ticks=3):
    """The headline workload's expansion in each form: tiles (the default for
    k = 16), gathered packets, packets walking the quadtree, one warp per query,
    and the paper's multi-pass iterative form; tick times, the first expansion
    kernel's time and the time of what finishes the packets it passed on, and
    whether the rows agree."""
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    wl = synth.plain_uniform_moving(n=N_OBJ, k=K, ticks=2, seed=5)
    ids = torch.from_numpy(wl.ticks[0].upd_id).to(dev)
    ux = [torch.from_numpy(t.upd_x).to(dev) for t in wl.ticks]
    uy = [torch.from_numpy(t.upd_y).to(dev) for t in wl.ticks]
    stream = torch.cuda.current_stream()
    out, rows = {}, {}
    for name, exp in (("tiles", 5), ("gathered packets", 4), ("packets", 1),
                      ("warp per query", 2), ("multi-pass iterative", 3)):
        x0, y0 = torch.from_numpy(wl.x0).to(dev), torch.from_numpy(wl.y0).to(dev)
        world = knnq.World(x0, y0, k_max=K, max_queries=N_OBJ)
        world.set_tuning(expansion=exp)
        world.set_profiling(True)
        oi = torch.empty((N_OBJ, K), dtype=torch.int32, device=dev)
        od = torch.empty((N_OBJ, K), dtype=torch.float32, device=dev)
        try:
            world.tick(K, ids, ids, ux[0], uy[0], out_ids=oi, out_d2=od)
            tick_ms, exp_ms, pass_ms = [], [], []
            for i in range(ticks):
                world.tick(K, ids, ids, ux[1 - i % 2], uy[1 - i % 2], out_ids=oi, out_d2=od)
                st = world.stage_times()
                tick_ms.append(sum(st.values()))
                exp_ms.append(st["expand"])
                pass_ms.append(st["pass-on"])
            out[name] = {"tick_ms": min(tick_ms), "expand_ms": min(exp_ms),
                         "pass_on_ms": min(pass_ms)}
            rows[name] = (oi.cpu(), od.cpu())
        finally:
            world.close()
    base = rows["packets"]
    for name, (a, b) in rows.items():
        out[name]["rows_identical_to_packets"] = bool(
            torch.equal(a, base[0]) and torch.equal(b.view(torch.int32), base[1].view(torch.int32)))
    return {"workload": f"{WORKLOAD}; {ticks} ticks per form", "per_form": out}


def brute_vs_indexed(dev, n_sample=16384):
    """The GPU brute-force baseline (every query against every object, as in the
    paper's comparison) against the indexed tick: on the 10k uniform k=8 world (all
    query) and on the headline world (1M uniform, k=16) with a sample of queries;
    rows compared for equality."""
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    stream = torch.cuda.current_stream()
    out = {}
    for name, wl, nq in (("10k uniform, k=8, all query", synth.plain_uniform_one_tick(), None),
                         ("1M uniform, k=16", synth.plain_uniform_moving(n=N_OBJ, k=K, ticks=1,
                                                                         seed=0), n_sample)):
        t = wl.ticks[0]
        n, k = wl.n, t.k
        x0, y0 = torch.from_numpy(wl.x0).to(dev), torch.from_numpy(wl.y0).to(dev)
        q_all = torch.from_numpy(t.q_id).to(dev)
        uid = torch.from_numpy(t.upd_id).to(dev)
        ux, uy = torch.from_numpy(t.upd_x).to(dev), torch.from_numpy(t.upd_y).to(dev)
        world = knnq.World(x0, y0, k_max=k, max_queries=int(q_all.shape[0]))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        try:
            oi = torch.empty((q_all.shape[0], k), dtype=torch.int32, device=dev)
            od = torch.empty((q_all.shape[0], k), dtype=torch.float32, device=dev)
            world.tick(k, q_all, uid, ux, uy, out_ids=oi, out_d2=od)  # positions after the move
            e0.record(stream)
            for _ in range(3):
                world.tick(k, q_all, out_ids=oi, out_d2=od)
            e1.record(stream)
            e1.synchronize()
            idx_ms = e0.elapsed_time(e1) / 3
            px, py = world.positions()
            q = q_all if nq is None else q_all[torch.linspace(0, q_all.shape[0] - 1, nq,
                                                                device=dev).long()]
            knnq.brute_force(px, py, k, q)  # warm
            e0.record(stream)
            bi, bd = knnq.brute_force(px, py, k, q)
            e1.record(stream)
            e1.synchronize()
            br_ms = e0.elapsed_time(e1)
            rows = q.long() if nq is not None else torch.arange(q.shape[0], device=dev)
            same = bool(torch.equal(bi, oi[rows]) and
                        torch.equal(bd.view(torch.int32), od[rows].view(torch.int32)))
            out[name] = {"indexed_queries_per_s": q_all.shape[0] / (idx_ms * 1e-3),
                         "brute_queries_per_s": q.shape[0] / (br_ms * 1e-3),
                         "brute_queries": int(q.shape[0]), "rows_identical": same}
        finally:
            world.close()
    return out


def k_sweep(dev, ks=(1, 4, 16, 32, 64, 128, 256, 512), iters=3):
    """Ticks of the 1M-uniform world (every object moves and queries) for k over the
    paper's range [1, 512]: queries/s per k and the expansion kernel used."""
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    wl = synth.plain_uniform_moving(n=N_OBJ, k=max(ks), ticks=2, seed=3)
    x0, y0 = torch.from_numpy(wl.x0).to(dev), torch.from_numpy(wl.y0).to(dev)
    ids = torch.from_numpy(wl.ticks[0].upd_id).to(dev)
    ux = [torch.from_numpy(t.upd_x).to(dev) for t in wl.ticks]
    uy = [torch.from_numpy(t.upd_y).to(dev) for t in wl.ticks]
    world = knnq.World(x0, y0, k_max=max(ks), max_queries=N_OBJ)
    stream = torch.cuda.current_stream()
    out = {}
    try:
        for k in ks:
            oi = torch.empty((N_OBJ, k), dtype=torch.int32, device=dev)
            od = torch.empty((N_OBJ, k), dtype=torch.float32, device=dev)
            world.tick(k, ids, ids, ux[0], uy[0], out_ids=oi, out_d2=od)
            world.tick(k, ids, ids, ux[1], uy[1], out_ids=oi, out_d2=od)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(iters):
                world.tick(k, ids, ids, ux[i % 2], uy[i % 2], out_ids=oi, out_d2=od)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / iters
            kernel = {1: "packets", 2: "warp per query", 4: "gathered packets", 5: "tiles"}.get(
                world.get_tuning(N_OBJ, k)["expansion"], "packets")
            out[str(k)] = {"tick_ms": ms, "queries_per_s": N_OBJ / (ms * 1e-3),
                           "expansion": kernel}
            del oi, od
    finally:
        world.close()
    return {"workload": "uniform 1M objects, every object moves N(0,1e-3) and queries, "
                        f"{iters} timed ticks per k", "per_k": out}


def batched_vs_plain(dev, n_worlds=256, seed=0, iters=5):
    """Many uneven worlds (1k-200k objects, uniform or clustered, k in {4,8,16,32}, all
    query): one knn_batch_tick (a recorded CUDA graph: the worlds' index stages side by
    side, then one batched expansion grid per list size) against one knn_tick per world,
    with the automatic settings and after knn_batch_autotune chose the settings per
    list-size class; the batched rows are compared with the plain ones, world by world."""
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    wl = synth.many_worlds(n_worlds=n_worlds, seed=seed, ticks=2)
    stream = torch.cuda.current_stream()
    data, worlds_b, worlds_p = [], [], []
    for w in wl:
        t = w.ticks[0]
        d = {"ids": torch.from_numpy(t.upd_id).to(dev), "ux": torch.from_numpy(t.upd_x).to(dev),
             "uy": torch.from_numpy(t.upd_y).to(dev), "q": torch.from_numpy(t.q_id).to(dev),
             "oi": torch.empty((t.q_id.shape[0], w.k), dtype=torch.int32, device=dev),
             "od": torch.empty((t.q_id.shape[0], w.k), dtype=torch.float32, device=dev),
             "pi": torch.empty((t.q_id.shape[0], w.k), dtype=torch.int32, device=dev),
             "pd": torch.empty((t.q_id.shape[0], w.k), dtype=torch.float32, device=dev)}
        data.append(d)
        x, y = torch.from_numpy(w.x0).to(dev), torch.from_numpy(w.y0).to(dev)
        worlds_b.append(knnq.World(x, y, k_max=w.k, max_queries=w.n))
        worlds_p.append(knnq.World(x, y, k_max=w.k, max_queries=w.n))
    args = [knnq.tick_args(w.k, d["q"], d["ids"], d["ux"], d["uy"], out_ids=d["oi"],
                           out_d2=d["od"]) for w, d in zip(wl, data)]
    pargs = [knnq.tick_args(w.k, d["q"], d["ids"], d["ux"], d["uy"], out_ids=d["pi"],
                            out_d2=d["pd"]) for w, d in zip(wl, data)]
    handles = [w.handle for w in worlds_b]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def batched_ms():
        knnq.knn_batch_tick(handles, args, stream.cuda_stream)  # (re)records the graph
        torch.cuda.synchronize()
        for _ in range(2):
            knnq.knn_batch_tick(handles, args, stream.cuda_stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(iters):
            knnq.knn_batch_tick(handles, args, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / iters

    def plain_pass():
        for w, a in zip(worlds_p, pargs):
            knnq.knn_tick(w.handle, a.upd_id_dev, a.upd_x_dev, a.upd_y_dev, a.n_upd, a.q_id_dev,
                          None, None, a.n_q, a.k, a.out_ids_dev, a.out_d2_dev, stream.cuda_stream)

    t0 = time.perf_counter()
    batch_default = batched_ms()
    record_s = time.perf_counter() - t0
    plain_pass()
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    for _ in range(iters):
        plain_pass()
    e1.record(stream)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1) / iters
    plain_host_ms = 1e3 * (time.perf_counter() - t0) / iters
    same_default = all(torch.equal(d["oi"], d["pi"]) and torch.equal(d["od"].view(torch.int32),
                                                                     d["pd"].view(torch.int32))
                       for d in data)
    # the batch autotuner (settings per list-size class, timed as whole batches),
    # then the batch again
    t0 = time.perf_counter()
    tunings = knnq.knn_batch_autotune(handles, args, trials=3, stream=stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    chosen = {}
    for w, t in zip(wl, tunings):
        c = chosen.setdefault(f"k={w.k}", {})
        key = f"expansion {t['expansion']} leaf_capacity {t['leaf_capacity']}"
        c[key] = c.get(key, 0) + 1
    batch_tuned = batched_ms()
    same_tuned = all(torch.equal(d["oi"], d["pi"]) and torch.equal(d["od"].view(torch.int32),
                                                                   d["pd"].view(torch.int32))
                     for d in data)
    q = sum(int(a.n_q) for a in args)
    for w in worlds_b + worlds_p:
        w.close()
    return {"workload": f"{n_worlds} worlds, {sum(w.n for w in wl)} objects, {q} queries per "
                        "batch tick; objects log-uniform in [1k, 200k], uniform or clustered, "
                        "k in {4,8,16,32}",
            "batched_ms": batch_tuned, "batched_default_ms": batch_default,
            "plain_ms": plain_ms, "plain_host_ms": plain_host_ms,
            "batched_queries_per_s": q / (batch_tuned / 1e3),
            "batched_default_queries_per_s": q / (batch_default / 1e3),
            "plain_queries_per_s": q / (plain_ms / 1e3), "graph_record_s": record_s,
            "autotune_s": tune_s, "autotune_chosen_forms": chosen,
            "rows_identical_to_plain": {"default": same_default, "tuned": same_tuned}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1412_6170_gb300 import synth
    w = synth.plain_uniform_moving(n=N_OBJ, k=K, ticks=1, seed=0)
    import numpy as np

    import oracle
    t = w.ticks[0]
    x, y, _ = oracle.apply_updates(w.x0, w.y0, t.upd_id, t.upd_x, t.upd_y)
    cores = os.cpu_count() or 1
    sample = max(64, 16 * cores)
    rows = np.linspace(0, N_OBJ - 1, sample).astype(np.int64)
    for _ in range(args.warmup):
        oracle.knn(x, y, t.q_id[rows[:cores]], K)
    times = []
    for s in range(args.steps):
        r = rows if s % 2 == 0 else rows[::-1]
        t0 = time.perf_counter()
        oracle.knn(x, y, t.q_id[r], K)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_objects": N_OBJ, "k": K,
                       "path": "cpu oracle (brute force)",
                       "step": f"{sample} sampled queries of one tick"},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{sample} evenly spaced queries per step over "
                                       f"{N_OBJ} objects"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_json_default), flush=True)


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1412_6170_gb300 import knnq, synth
    import __graft_entry__

    rank, world_size, local = dist_env()
    dist = None
    if world_size > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    knnq.lib()
    if args.only:
        # one comparison leg alone (its own JSON line), e.g. for a profiler
        legs = {"serving": lambda: serving_config5(dev, check=not args.no_check),
                "skewed": lambda: skewed_config3(dev, check=not args.no_check),
                "batching": lambda: batched_vs_plain(dev),
                "k_sweep": lambda: k_sweep(dev),
                "index_reuse": lambda: index_reuse_vs_rebuild(dev),
                "brute_force": lambda: brute_vs_indexed(dev),
                "expansion_ablation": lambda: expansion_ablation(dev)}
        if rank == 0:
            print(json.dumps({"leg": args.only, **legs[args.only]()}, default=_json_default),
                  flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    wl = synth.plain_uniform_moving(n=N_OBJ, k=K, ticks=N_TICKS, seed=0)
    stream = torch.cuda.current_stream()
    x0 = torch.from_numpy(wl.x0).to(dev)
    y0 = torch.from_numpy(wl.y0).to(dev)
    ids_d = torch.from_numpy(wl.ticks[0].upd_id).to(dev)          # 0..n-1, shared by ticks
    ux = [torch.from_numpy(t.upd_x).to(dev) for t in wl.ticks]
    uy = [torch.from_numpy(t.upd_y).to(dev) for t in wl.ticks]
    qid = ids_d
    out_ids = torch.empty((N_OBJ, K), dtype=torch.int32, device=dev)
    out_d2 = torch.empty((N_OBJ, K), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    world = knnq.World(x0, y0, k_max=K, max_queries=N_OBJ)
    world.set_profiling(True)
    # A simulation hands each tick's moves over in one of two device buffers
    # (double buffering); the move is copied into place before the step's
    # timed region, so inputs are resident in HBM when it starts.  knn_tick
    # records one graph per buffer and replays it.
    bx = [torch.empty_like(ux[0]) for _ in range(2)]
    by = [torch.empty_like(uy[0]) for _ in range(2)]

    def stage_inputs(i):
        bx[i % 2].copy_(ux[i % N_TICKS])
        by[i % 2].copy_(uy[i % N_TICKS])

    def tick(i):
        world.tick(K, qid, ids_d, bx[i % 2], by[i % 2], out_ids=out_ids, out_d2=out_d2)

    for i in range(args.warmup):
        stage_inputs(i)
        tick(i)
    torch.cuda.synchronize()
    st, bits = world.status()
    if st != knnq.KNN_OK:
        raise RuntimeError(f"device status {st} bits {bits} after warm-up")

    # quick exactness spot check of the last warm-up tick against the oracle
    spot = None
    if rank == 0 and not args.no_check:
        import oracle
        t = wl.ticks[(args.warmup - 1) % N_TICKS]
        rows = np.linspace(0, N_OBJ - 1, 512).astype(np.int64)
        x, y, _ = oracle.apply_updates(wl.x0, wl.y0, t.upd_id, t.upd_x, t.upd_y)
        rid, rd2, _ = oracle.knn(x, y, t.q_id[rows], K)
        gid = out_ids.cpu().numpy()[rows]
        gd2 = out_d2.cpu().numpy()[rows]
        spot = bool(np.array_equal(gid, rid) and np.array_equal(gd2.view(np.uint32),
                                                                rd2.view(np.uint32)))
        if not spot:
            raise RuntimeError("GPU result differs from the oracle on the spot check")

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stage_sums = None
    launches0 = world.launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for s in range(args.steps):
            stage_inputs(args.warmup + s)
            flush.zero_()
            a, b = ev[s]
            a.record(stream)
            tick(args.warmup + s)
            b.record(stream)
            b.synchronize()
            st_ms = world.stage_times()
            stage_sums = {k: stage_sums.get(k, 0.0) + v for k, v in st_ms.items()} \
                if stage_sums else dict(st_ms)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    launches = world.launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # tick latency over many ticks (same steps: moves copied in, L2 flushed, one
    # tick timed by events each)
    lat_ms = []
    for s in range(args.latency_ticks):
        stage_inputs(s)
        flush.zero_()
        a, b = ev[s % len(ev)]
        a.record(stream)
        tick(s)
        b.record(stream)
        b.synchronize()
        lat_ms.append(a.elapsed_time(b))
    total_ms = max_over_ranks([sum(step_ms)], dist, dev)[0]
    st, bits = world.status()
    if st != knnq.KNN_OK:
        raise RuntimeError(f"device status {st} bits {bits} after timed steps")

    # end-to-end through the public host-buffer API (pinned host arrays)
    import ctypes
    h_uid = torch.from_numpy(wl.ticks[0].upd_id).pin_memory()
    h_ux = [torch.from_numpy(t.upd_x).pin_memory() for t in wl.ticks[:2]]
    h_uy = [torch.from_numpy(t.upd_y).pin_memory() for t in wl.ticks[:2]]
    h_oid = torch.empty((N_OBJ, K), dtype=torch.int32).pin_memory()
    h_od = torch.empty((N_OBJ, K), dtype=torch.float32).pin_memory()
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    e2e_steps = max(3, min(args.steps, 20))

    def e2e_run(mode):
        # mode: how knn_tick_host uses the pinned arrays (bit 0 rows written in
        # place by the kernels, bit 1 inputs read in place; 0 stages both)
        world.set_host_io(write_rows=bool(mode & 1), read_inputs=bool(mode & 2))
        for i in range(2):  # warm-up (the first staged call allocates its buffers)
            knnq.knn_tick_host(world.handle, vp(h_uid), vp(h_ux[i]), vp(h_uy[i]), N_OBJ,
                               vp(h_uid), None, None, N_OBJ, K, vp(h_oid), vp(h_od),
                               stream.cuda_stream)
        torch.cuda.synchronize()
        t = []
        for s in range(e2e_steps):
            t0 = time.perf_counter()
            knnq.knn_tick_host(world.handle, vp(h_uid), vp(h_ux[s % 2]), vp(h_uy[s % 2]), N_OBJ,
                               vp(h_uid), None, None, N_OBJ, K, vp(h_oid), vp(h_od),
                               stream.cuda_stream)
            t.append(time.perf_counter() - t0)
        return max_over_ranks([sum(t)], dist, dev)[0]

    e2e_modes = {name: e2e_run(m) for name, m in
                 (("sync_staged", 0), ("sync_inputs_in_place", 2), ("sync_all_in_place", 3),
                  ("sync_rows_in_place", 1))}

    # pipelined: knn_tick_host_submit / knn_tick_host_wait with two sets of
    # output arrays; step s's rows are waited for (read) after step s + 1 is
    # submitted, so one tick's copies overlap the next one's search
    h_oid2 = [h_oid, torch.empty((N_OBJ, K), dtype=torch.int32).pin_memory()]
    h_od2 = [h_od, torch.empty((N_OBJ, K), dtype=torch.float32).pin_memory()]

    def e2e_pipelined(steps):
        prev = None
        for s in range(steps):
            tk = knnq.knn_tick_host_submit(world.handle, vp(h_uid), vp(h_ux[s % 2]),
                                           vp(h_uy[s % 2]), N_OBJ, vp(h_uid), None, None, N_OBJ,
                                           K, vp(h_oid2[s % 2]), vp(h_od2[s % 2]),
                                           stream.cuda_stream)
            if prev is not None:
                knnq.knn_tick_host_wait(world.handle, prev)
            prev = tk
        knnq.knn_tick_host_wait(world.handle, prev)

    e2e_pipelined(3)  # warm-up (allocates the two staging slots, records the graphs)
    # three timed runs (fill and drain inside each); the median is reported, so
    # one host-side hiccup in a run of a few milliseconds does not decide it
    e2e_runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pipelined(e2e_steps)
        e2e_runs.append(max_over_ranks([time.perf_counter() - t0], dist, dev)[0])
    e2e_total = sorted(e2e_runs)[1]
    e2e_modes = {"pipelined": e2e_total, **e2e_modes}
    # the rows that reached host memory in the last pipelined step, against
    # the oracle (every object moves every tick, so that tick's inputs alone
    # fix its rows)
    e2e_spot = None
    if rank == 0 and not args.no_check:
        import oracle
        last = (e2e_steps - 1) % 2
        t = wl.ticks[last]
        rows = np.linspace(0, N_OBJ - 1, 512).astype(np.int64)
        x, y, _ = oracle.apply_updates(wl.x0, wl.y0, t.upd_id, t.upd_x, t.upd_y)
        rid, rd2, _ = oracle.knn(x, y, t.q_id[rows], K)
        gid = h_oid2[last].numpy()[rows]
        gd2 = h_od2[last].numpy()[rows]
        e2e_spot = bool(np.array_equal(gid, rid) and np.array_equal(gd2.view(np.uint32),
                                                                    rd2.view(np.uint32)))
        if not e2e_spot:
            raise RuntimeError("host-buffer rows differ from the oracle on the spot check")
    form = world.get_tuning(N_OBJ, K)["expansion"]
    world.close()
    if rank != 0:
        return
    n_gpus = world_size
    value = replicas_value(n_gpus, N_OBJ * args.steps, total_ms / 1e3)
    p99 = pct(lat_ms, 0.99) if lat_ms else pct(step_ms, 0.99)
    p50 = pct(lat_ms, 0.5) if lat_ms else statistics.median(step_ms)
    exp_ms = stage_sums["expand"] / args.steps
    hbm, hbm_kind = peaks()
    achieved = ALGO_BYTES_PER_QUERY * N_OBJ / (exp_ms / 1e3) / 1e9
    kernel, source = {5: ("k_expand_tile", "knn_expand_tile.cu"),
                      4: ("k_expand_gather", "knn_expand_gather.cu")}.get(
                          form, ("k_expand", "knn_expand.cu"))
    prof = expand_profile(kernel, source)
    traffic = None if prof is None else prof["traffic"]
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_sum = clk.summary()
    clk_mhz = clk_sum.get("sm_mhz") or clk_sum.get("sm_max_mhz") or 2070.0
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": n_gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_objects": N_OBJ, "k": K, "queries_per_tick": N_OBJ,
                   "path": "plain (one knn_tick per tick; moves double-buffered on the "
                           "device, copied in before each step's timed region)",
                   "l2": "flushed between steps",
                   "parallelism": "replicas" if n_gpus > 1 else "single GPU"},
        "p50_tick_ms": p50, "p99_tick_ms": p99, "latency_ticks": len(lat_ms),
        "stages_ms": {k: v / args.steps for k, v in stage_sums.items()},
        "roofline": {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "peak_kind": hbm_kind, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": traffic,
                     "algorithmic_bytes_per_query": ALGO_BYTES_PER_QUERY,
                     "limiter": None if prof is None else
                     f"ALU pipe {prof['alu_pipe_pct']:.0f}% of peak (ncu); DRAM traffic "
                     "below the algorithmic bytes",
                     # the bound that binds: instruction issue (one warp
                     # instruction per cycle per scheduler, 4 per SM)
                     "issue": None if prof is None else {
                         "achieved": prof["warp_inst"] / (exp_ms / 1e3) / 1e9,
                         "peak": 4 * n_sms * clk_mhz / 1e3,
                         "unit": "G warp instructions/s",
                         "frac": prof["warp_inst"] / (exp_ms / 1e3) / 1e9
                         / (4 * n_sms * clk_mhz / 1e3),
                         "source": "smsp__inst_executed.sum per launch (ncu, same kernel "
                                   "source) over the live launch time; peak at the "
                                   "sampled SM clock"}},
        "e2e": {"value": replicas_value(n_gpus, N_OBJ * e2e_steps, e2e_total),
                "unit": "queries/s",
                "h2d_bytes_per_step": N_OBJ * 12 + N_OBJ * 4,
                "d2h_bytes_per_step": N_OBJ * K * 8,
                "api": "knn_tick_host_submit + knn_tick_host_wait (pinned host buffers, "
                       "two ticks in flight: each step's inputs copied in and rows copied "
                       "out inside the timed region, overlapping the next step's search; "
                       "the median of three timed runs of the same steps); "
                       "by_mode adds the synchronous knn_tick_host",
                "pipelined_runs_s": e2e_runs,
                "by_mode": {m: replicas_value(n_gpus, N_OBJ * e2e_steps, t)
                            for m, t in e2e_modes.items()},
                "exact_spot_check": e2e_spot},
        "gpu_launches": launches,
        "clocks": clk_sum,
        "exact_spot_check": spot,
        "wall_s": wall,
    }
    if not args.no_patterns:
        line["serving"] = serving_config5(dev, check=not args.no_check)
        line["skewed"] = skewed_config3(dev, check=not args.no_check)
        line["batching"] = batched_vs_plain(dev)
        line["k_sweep"] = k_sweep(dev)
        line["index_reuse"] = index_reuse_vs_rebuild(dev)
        line["brute_force"] = brute_vs_indexed(dev)
        line["expansion_ablation"] = expansion_ablation(dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line, default=_json_default), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the serving, skewed, batching and other comparison legs")
    ap.add_argument("--only", default=None,
                    choices=["serving", "skewed", "batching", "k_sweep", "index_reuse",
                             "brute_force", "expansion_ablation"],
                    help="run one comparison leg alone and print its JSON line")
    ap.add_argument("--latency-ticks", type=int, default=200,
                    help="ticks timed one by one for p50/p99 tick latency")
    args = ap.parse_args()
    if args.warmup < 1:
        args.warmup = 1
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
