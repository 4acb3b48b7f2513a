"""Seeded synthetic moving-object workloads.

This module only draws random numbers and lays out input arrays; it holds none
of the k-NN method's arithmetic.  The same bytes feed the CUDA path and the CPU
oracle, so both see identical inputs.

The paper (Section 5, Experimental Setup) generates uniform, Gaussian-hotspot
and road-network datasets with an external framework over 30 ticks, one query
per object per tick.  That generator is not available, so these seeded
stand-ins reproduce the shapes: positions in the unit square, per-tick random
displacements, clustered (hotspot) mixtures and query subsets.

Random source: splitmix64.  Stream ``(seed, stream)`` is the splitmix64
sequence started from ``state0 = mix(seed ^ mix(stream))``: value ``i`` is
``mix(state0 + (i + 1) * 0x9E3779B97F4A7C15)`` (mod 2**64), where ``mix`` is the
splitmix64 finaliser.

* uniform float32 in [0, 1):   ``(u >> 40) * 2**-24``  (exact in binary32)
* uniform float64 in (0, 1):   ``((u >> 11) + 0.5) * 2**-53``
* standard normal (float64):   Box-Muller, ``sqrt(-2 ln u1) * cos(2 pi u2)``
  with ``u1``/``u2`` the even/odd draws of one stream; the scaled result is
  rounded to float32 once.
* every position is clamped to ``[0, 1 - 2**-24]`` (the largest float32 below 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
F32_ONE_MINUS = np.float32(1.0 - 2.0 ** -24)

# Stream identifiers (stable; changing one changes every workload).
S_X, S_Y, S_CLUSTER_PICK, S_CLUSTER_ID, S_CX, S_CY, S_NX, S_NY = range(1, 9)
S_MOVE_X, S_MOVE_Y, S_QUERY_PICK = 101, 102, 103


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def u64_stream(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` splitmix64 draws of stream ``(seed, stream)`` starting at ``offset``."""
    s = _mix(np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))
    state0 = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) ^ s)[0]
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(state0 + idx * _GOLDEN)


def uniform_f32(seed: int, stream: int, count: int) -> np.ndarray:
    u = u64_stream(seed, stream, count)
    return (u >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -24)


def uniform_f64(seed: int, stream: int, count: int) -> np.ndarray:
    u = u64_stream(seed, stream, count)
    return ((u >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal_f64(seed: int, stream: int, count: int) -> np.ndarray:
    u = u64_stream(seed, stream, 2 * count)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    u2 = ((u[1::2] >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def clamp_unit(v: np.ndarray) -> np.ndarray:
    return np.clip(v.astype(np.float32), np.float32(0.0), F32_ONE_MINUS).astype(np.float32)


def uniform_positions(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    return uniform_f32(seed, S_X, n), uniform_f32(seed, S_Y, n)


def clustered_positions(n: int, seed: int, n_clusters: int = 64, sigma: float = 0.01,
                        frac_clustered: float = 0.9) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian hotspots (centres uniform, per-coordinate sigma) plus a uniform background."""
    pick = uniform_f64(seed, S_CLUSTER_PICK, n) < frac_clustered
    cid = (uniform_f64(seed, S_CLUSTER_ID, n) * n_clusters).astype(np.int64)
    cid = np.minimum(cid, n_clusters - 1)
    cx = uniform_f32(seed, S_CX, n_clusters).astype(np.float64)
    cy = uniform_f32(seed, S_CY, n_clusters).astype(np.float64)
    gx = cx[cid] + sigma * normal_f64(seed, S_NX, n)
    gy = cy[cid] + sigma * normal_f64(seed, S_NY, n)
    ux, uy = uniform_positions(n, seed)
    x = np.where(pick, clamp_unit(gx), ux).astype(np.float32)
    y = np.where(pick, clamp_unit(gy), uy).astype(np.float32)
    return x, y


def random_walk(x: np.ndarray, y: np.ndarray, sigma: float, seed: int, tick: int
                ) -> tuple[np.ndarray, np.ndarray]:
    """Per-coordinate N(0, sigma) displacement, then clamp to the square."""
    n = x.shape[0]
    s = seed * 1000003 + tick
    nx = x.astype(np.float64) + sigma * normal_f64(s, S_MOVE_X, n)
    ny = y.astype(np.float64) + sigma * normal_f64(s, S_MOVE_Y, n)
    return clamp_unit(nx), clamp_unit(ny)


def random_subset(n: int, count: int, seed: int, tick: int) -> np.ndarray:
    """``count`` distinct ids from [0, n) in random (caller) order."""
    u = u64_stream(seed * 1000003 + tick, S_QUERY_PICK, n)
    return np.argsort(u, kind="stable")[:count].astype(np.int32)


@dataclass
class Tick:
    """One tick's batch: updates applied in array order, then the queries.

    ``q_x``/``q_y`` None means each query is centred at its issuer's
    post-update position.
    """
    upd_id: np.ndarray
    upd_x: np.ndarray
    upd_y: np.ndarray
    q_id: np.ndarray
    k: int
    q_x: Optional[np.ndarray] = None
    q_y: Optional[np.ndarray] = None


@dataclass
class Workload:
    name: str
    n: int
    k: int
    x0: np.ndarray
    y0: np.ndarray
    ticks: list = field(default_factory=list)

    @property
    def n_ticks(self) -> int:
        return len(self.ticks)


def _empty_updates():
    return (np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32))


def plain_uniform_one_tick(n: int = 10_000, k: int = 8, seed: int = 0) -> Workload:
    """10k objects uniform in [0,1)^2, one tick, every object queries at its own position."""
    x, y = uniform_positions(n, seed)
    uid, ux, uy = _empty_updates()
    t = Tick(uid, ux, uy, np.arange(n, dtype=np.int32), k)
    return Workload(f"uniform n={n} k={k} 1 tick", n, k, x, y, [t])


def plain_uniform_moving(n: int = 1_000_000, k: int = 16, ticks: int = 10, seed: int = 0,
                         sigma: float = 1e-3) -> Workload:
    """Uniform objects; each tick every object moves by N(0, sigma) and every object queries."""
    x, y = uniform_positions(n, seed)
    w = Workload(f"uniform n={n} k={k} {ticks} ticks, N(0,{sigma:g}) moves, all query",
                 n, k, x, y)
    ids = np.arange(n, dtype=np.int32)
    cx, cy = x, y
    for t in range(1, ticks + 1):
        cx, cy = random_walk(cx, cy, sigma, seed, t)
        w.ticks.append(Tick(ids, cx, cy, ids, k))
    return w


def skewed_moving(n: int = 4_000_000, k: int = 32, ticks: int = 10, seed: int = 0,
                  sigma: float = 5e-4, query_frac: float = 0.25) -> Workload:
    """90% of objects in 64 Gaussian hotspots (sigma 0.01) + 10% uniform; a fresh random
    25% of the objects query each tick."""
    x, y = clustered_positions(n, seed)
    w = Workload(f"clustered n={n} k={k} {ticks} ticks, {query_frac:.0%} query", n, k, x, y)
    ids = np.arange(n, dtype=np.int32)
    cx, cy = x, y
    nq = int(round(n * query_frac))
    for t in range(1, ticks + 1):
        cx, cy = random_walk(cx, cy, sigma, seed, t)
        w.ticks.append(Tick(ids, cx, cy, random_subset(n, nq, seed, t), k))
    return w


def world_positions(n: int, seed: int, clustered: bool) -> tuple[np.ndarray, np.ndarray]:
    return clustered_positions(n, seed) if clustered else uniform_positions(n, seed)


def serving_world(i: int, seed: int = 0, n_worlds: int = 64, n_lo: int = 10_000,
                  n_hi: int = 4_000_000, ks=(4, 8, 16, 32, 64), query_frac=(0.1, 1.0),
                  sigma: float = 5e-4) -> "Workload":
    """World ``i`` of :func:`serving_worlds` (each world is drawn from its own streams,
    so the worlds can be generated independently, e.g. in worker processes)."""
    u = uniform_f64(seed, 202, 3 * n_worlds).reshape(n_worlds, 3)
    n = int(round(np.exp(np.log(n_lo) + u[i, 0] * (np.log(n_hi) - np.log(n_lo)))))
    k = int(ks[min(len(ks) - 1, int(u[i, 1] * len(ks)))])
    qf = query_frac[0] + u[i, 2] * (query_frac[1] - query_frac[0])
    ws = seed * 7919 + 5000 + i
    x, y = clustered_positions(n, ws)
    w = Workload(f"world {i}: n={n} k={k} clustered, {qf:.0%} query", n, k, x, y)
    cx, cy = random_walk(x, y, sigma, ws, 1)
    nq = max(1, int(round(n * qf)))
    w.ticks.append(Tick(np.arange(n, dtype=np.int32), cx, cy, random_subset(n, nq, ws, 1), k))
    return w


def serving_worlds(n_worlds: int = 64, seed: int = 0, map_fn=map, **kw) -> list:
    """Resident worlds of a serving loop: object counts log-uniform in [10k, 4M], all
    clustered as the 4M skewed workload, k drawn from {4, 8, 16, 32, 64}, a query
    fraction uniform in [0.1, 1]; one tick of N(0, 5e-4) moves of every object and a
    random subset of querying objects.  ``map_fn`` may be a process pool's map."""
    from functools import partial
    return list(map_fn(partial(serving_world, seed=seed, n_worlds=n_worlds, **kw),
                       range(n_worlds)))


def many_worlds(n_worlds: int = 256, seed: int = 0, n_lo: int = 1_000, n_hi: int = 200_000,
                ks=(4, 8, 16, 32), ticks: int = 2, sigma: float = 1e-3,
                query_frac=(1.0, 1.0)) -> list:
    """Independent worlds of uneven size: object counts log-uniform in [n_lo, n_hi],
    uniform or clustered (as the 4M skewed workload) by a coin flip, k drawn from ``ks``,
    a query fraction drawn uniformly from ``query_frac``; every tick moves every object
    by N(0, sigma) and a fresh random subset (or all) of the objects query."""
    u = uniform_f64(seed, 201, 4 * n_worlds).reshape(n_worlds, 4)
    out = []
    for i in range(n_worlds):
        n = int(round(np.exp(np.log(n_lo) + u[i, 0] * (np.log(n_hi) - np.log(n_lo)))))
        clustered = bool(u[i, 1] < 0.5)
        k = int(ks[min(len(ks) - 1, int(u[i, 2] * len(ks)))])
        qf = query_frac[0] + u[i, 3] * (query_frac[1] - query_frac[0])
        ws = seed * 7919 + i + 1
        x, y = world_positions(n, ws, clustered)
        w = Workload(f"world {i}: n={n} k={k} {'clustered' if clustered else 'uniform'}",
                     n, k, x, y)
        ids = np.arange(n, dtype=np.int32)
        cx, cy = x, y
        nq = max(1, int(round(n * qf)))
        for t in range(1, ticks + 1):
            cx, cy = random_walk(cx, cy, sigma, ws, t)
            q = ids if nq == n else random_subset(n, nq, ws, t)
            w.ticks.append(Tick(ids, cx, cy, q, k))
        out.append(w)
    return out
