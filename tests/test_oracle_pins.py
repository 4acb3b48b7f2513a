"""Pins for the brute-force k-NN oracle (CPU only).

Each test ties the oracle to something other than itself: closed-form lattice
distances, exhaustive enumeration of Def. 1 on tiny inputs in exact rational
arithmetic, the binary32 rounding sequence of the distance (no FMA), the
paper's batch semantics (Section 2.2), and invariants that any correct k-NN
result satisfies.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests import f32exact as fx


def rng(seed):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# Distance arithmetic


def test_sqdist_matches_exact_rounding_sequence():
    r = rng(1)
    pts = r.random((2000, 4)).astype(np.float32)
    pts[:500] *= np.float32(1e-3)  # small differences, subnormal-free
    for qx, qy, px, py in pts:
        want = fx.to_f32(fx.sqdist(qx, qy, px, py))
        got = np.float32(oracle.sqdist(qx, qy, px, py))
        assert got.view(np.uint32) == want.view(np.uint32), (qx, qy, px, py)


def test_sqdist_is_not_fused():
    """Find inputs where fma(dx,dx,dy*dy) rounds differently from the unfused
    expression; the oracle must give the unfused value."""
    r = rng(2)
    found = 0
    for _ in range(20000):
        qx, qy, px, py = r.random(4).astype(np.float32)
        plain = fx.sqdist(qx, qy, px, py)
        fused = fx.sqdist_fused(qx, qy, px, py)
        if plain != fused:
            got = np.float32(oracle.sqdist(qx, qy, px, py))
            assert got == fx.to_f32(plain)
            assert got != fx.to_f32(fused)
            found += 1
            if found >= 50:
                break
    assert found >= 50


def test_sqdist_symmetric_and_within_error_bound():
    """Both argument orders give the same value (round-to-nearest is symmetric),
    and the result is within 3 half-ulps (relative 2^-24 each) of the exact d^2."""
    r = rng(3)
    for qx, qy, px, py in r.random((2000, 4)).astype(np.float32):
        a = oracle.sqdist(qx, qy, px, py)
        b = oracle.sqdist(px, py, qx, qy)
        assert np.float32(a) == np.float32(b)
        ex = (fx.exact(qx) - fx.exact(px)) ** 2 + (fx.exact(qy) - fx.exact(py)) ** 2
        if ex == 0:
            assert a == 0
            continue
        rel = abs(Fraction(float(a)) - ex) / ex
        assert rel <= Fraction(3, 2 ** 24) * (1 + Fraction(1, 2 ** 20))


# --------------------------------------------------------------------------
# Closed form: integer lattice scaled by 1/64, every distance exact


def lattice(side=16):
    ii, jj = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    return (ii / 64.0).astype(np.float32), (jj / 64.0).astype(np.float32), ii, jj


@pytest.mark.parametrize("k", [1, 4, 5, 8, 12, 13, 20])
def test_lattice_closed_form(k):
    x, y, ii, jj = lattice()
    n = x.shape[0]
    qid = np.arange(n, dtype=np.int32)
    ids, d2, bad = oracle.knn(x, y, qid, k)
    assert bad == 0
    for s in range(n):
        # exact integer distances, ties broken by the object id
        keys = sorted(((ii[s] - ii[j]) ** 2 + (jj[s] - jj[j]) ** 2, j)
                      for j in range(n) if j != s)[:k]
        assert list(ids[s]) == [j for _, j in keys]
        assert list(d2[s]) == [np.float32(v / 4096.0) for v, _ in keys]


def test_lattice_first_ring_values():
    """Interior lattice point: four neighbours at 1/4096, four at 2/4096, four at 4/4096."""
    x, y, ii, jj = lattice()
    s = int(np.flatnonzero((ii == 7) & (jj == 7))[0])
    ids, d2, _ = oracle.knn(x, y, np.array([s], np.int32), 12)
    assert list(d2[0]) == [np.float32(v / 4096.0) for v in [1] * 4 + [2] * 4 + [4] * 4]
    # equal distances come in ascending id order
    for a in range(0, 12, 4):
        assert list(ids[0, a:a + 4]) == sorted(ids[0, a:a + 4])


# --------------------------------------------------------------------------
# Def. 1 by exhaustive enumeration of candidate result sets


def def1_by_enumeration(x, y, s, k, qx=None, qy=None):
    """The unique k-subset S of eligible objects whose every key is below every
    key outside S (Def. 1 with ties resolved by id), found by trying all subsets."""
    n = len(x)
    cx = x[s] if qx is None else qx
    cy = y[s] if qy is None else qy
    elig = [j for j in range(n) if j != s]
    key = {j: (fx.sqdist(cx, cy, x[j], y[j]), j) for j in elig}
    kk = min(k, len(elig))
    winners = []
    for S in itertools.combinations(elig, kk):
        inside = [key[j] for j in S]
        outside = [key[j] for j in elig if j not in S]
        if all(a < b for a in inside for b in outside):
            winners.append(sorted(inside))
    assert len(winners) == 1
    res = winners[0]
    ids = [j for _, j in res] + [-1] * (k - kk)
    d = [fx.to_f32(v) for v, _ in res] + [np.float32(np.inf)] * (k - kk)
    return ids, d


@pytest.mark.parametrize("seed", range(12))
def test_exhaustive_enumeration_tiny(seed):
    r = rng(100 + seed)
    n = int(r.integers(1, 9))
    if seed % 2 == 0:  # coarse grid: many exact ties and coincident points
        x = (r.integers(0, 4, n) / 4.0).astype(np.float32)
        y = (r.integers(0, 4, n) / 4.0).astype(np.float32)
    else:
        x = r.random(n).astype(np.float32)
        y = r.random(n).astype(np.float32)
    for k in range(1, n + 2):
        qid = np.arange(n, dtype=np.int32)
        ids, d2, bad = oracle.knn(x, y, qid, k)
        assert bad == 0
        for s in range(n):
            wid, wd = def1_by_enumeration(x, y, s, k)
            assert list(ids[s]) == wid
            assert [v.view(np.uint32) for v in d2[s]] == [v.view(np.uint32) for v in wd]


def test_anonymous_and_explicit_centres():
    r = rng(7)
    n = 7
    x = (r.integers(0, 3, n) / 2.0).astype(np.float32)
    y = (r.integers(0, 3, n) / 2.0).astype(np.float32)
    qx = np.array([0.5, 0.25, 1.0], np.float32)
    qy = np.array([0.5, 0.75, 0.0], np.float32)
    qid = np.array([-1, 3, -1], np.int32)
    for k in (1, 3, 6, 8):
        ids, d2, bad = oracle.knn(x, y, qid, k, qx, qy)
        assert bad == 0
        for i in range(3):
            wid, wd = def1_by_enumeration(x, y, int(qid[i]), k, qx[i], qy[i])
            assert list(ids[i]) == wid
            assert list(d2[i]) == wd


# --------------------------------------------------------------------------
# Invariants of any correct result


def random_cloud(n, seed):
    r = rng(seed)
    return r.random(n).astype(np.float32), r.random(n).astype(np.float32)


def test_prefix_and_disc_properties():
    n = 300
    x, y = random_cloud(n, 11)
    # add coincident objects and lattice duplicates to create ties
    x[:20] = x[20:40]
    y[:20] = y[20:40]
    qid = np.arange(n, dtype=np.int32)
    prev = None
    for k in (1, 2, 7, 16, 17, 40):
        ids, d2, _ = oracle.knn(x, y, qid, k)
        if prev is not None:
            pk = prev[0].shape[1]
            assert np.array_equal(ids[:, :pk], prev[0])
            assert np.array_equal(d2[:, :pk], prev[1])
        prev = (ids, d2)
        for s in range(0, n, 13):
            assert s not in ids[s]
            assert len(set(ids[s])) == k
            last = (Fraction(float(d2[s, -1])), int(ids[s, -1]))
            chosen = set(ids[s].tolist())
            for j in range(n):
                kj = (fx.sqdist(x[s], y[s], x[j], y[j]), j)
                if j == s:
                    continue
                if j in chosen:
                    assert kj <= last
                else:
                    assert kj > last


def test_permutation_invariance():
    n = 500
    x, y = random_cloud(n, 12)
    qid = np.arange(n, dtype=np.int32)
    ids, d2, _ = oracle.knn(x, y, qid, 9)
    perm = rng(13).permutation(n)            # object j is stored at slot perm[j]
    xp = np.empty_like(x)
    yp = np.empty_like(y)
    xp[perm] = x
    yp[perm] = y
    qidp = perm[qid].astype(np.int32)
    ids2, d22, _ = oracle.knn(xp, yp, qidp, 9)
    inv = np.argsort(perm)
    assert np.array_equal(d2, d22)
    # random float data: no distance ties, so relabelled ids agree exactly
    assert np.array_equal(ids, inv[ids2])


def test_full_sorted_list_when_k_is_n_minus_one():
    n = 60
    x, y = random_cloud(n, 14)
    ids, d2, _ = oracle.knn(x, y, np.arange(n, dtype=np.int32), n - 1)
    for s in range(n):
        keys = sorted((fx.sqdist(x[s], y[s], x[j], y[j]), j) for j in range(n) if j != s)
        assert list(ids[s]) == [j for _, j in keys]


def test_padding_and_degenerate_cases():
    # one object: every row is padding
    ids, d2, _ = oracle.knn(np.zeros(1, np.float32), np.zeros(1, np.float32),
                            np.array([0], np.int32), 3)
    assert list(ids[0]) == [-1, -1, -1] and np.all(np.isinf(d2))
    # n <= k: all others, then padding
    x = np.array([0.1, 0.2, 0.4], np.float32)
    y = np.zeros(3, np.float32)
    ids, d2, _ = oracle.knn(x, y, np.arange(3, dtype=np.int32), 4)
    assert list(ids[0]) == [1, 2, -1, -1]
    assert list(ids[2]) == [1, 0, -1, -1]
    # all objects coincident: every distance 0, ids ascending without the issuer
    x = np.full(10, 0.3, np.float32)
    ids, d2, _ = oracle.knn(x, x, np.arange(10, dtype=np.int32), 5)
    assert np.all(d2 == 0)
    assert list(ids[4]) == [0, 1, 2, 3, 5]
    # an anonymous query at an object's position keeps that object (distance 0)
    ids, d2, _ = oracle.knn(x, x, np.array([-1], np.int32), 2,
                            np.array([0.3], np.float32), np.array([0.3], np.float32))
    assert list(ids[0]) == [0, 1]


def test_invalid_queries_are_padded_and_counted():
    x, y = random_cloud(20, 15)
    qid = np.array([0, 25, -1, -2, 3], np.int32)
    ids, d2, bad = oracle.knn(x, y, qid, 2)
    assert bad == 3
    for i in (1, 2, 3):
        assert list(ids[i]) == [-1, -1]
    qx = np.array([0.5, np.nan], np.float32)
    ids, d2, bad = oracle.knn(x, y, np.array([-1, -1], np.int32), 2, qx, qx)
    assert bad == 1 and list(ids[1]) == [-1, -1] and ids[0, 0] >= 0


# --------------------------------------------------------------------------
# Batch semantics, Section 2.2


def test_updates_last_one_wins_and_invalid_skipped():
    x = np.zeros(5, np.float32)
    y = np.zeros(5, np.float32)
    uid = np.array([1, 3, 1, 7, -1, 2, 2], np.int32)
    ux = np.array([0.1, 0.3, 0.9, 0.5, 0.5, np.inf, 0.25], np.float32)
    uy = np.array([0.1, 0.3, 0.8, 0.5, 0.5, 0.0, 0.5], np.float32)
    nx, ny, bad = oracle.apply_updates(x, y, uid, ux, uy)
    assert bad == 3
    assert list(nx) == [0, np.float32(0.9), np.float32(0.25), np.float32(0.3), 0]
    assert list(ny) == [0, np.float32(0.8), np.float32(0.5), np.float32(0.3), 0]


def test_queries_see_post_update_positions():
    x = np.array([0.0, 0.5, 1.0], np.float32)
    y = np.zeros(3, np.float32)

    class T:
        upd_id = np.array([2], np.int32)
        upd_x = np.array([0.1], np.float32)
        upd_y = np.array([0.0], np.float32)
        q_id = np.array([0], np.int32)
        q_x = None
        q_y = None
        k = 1

    (ids, d2), = oracle.run_ticks(x, y, [T])
    assert ids[0, 0] == 2 and d2[0, 0] == np.float32(np.float32(0.1) * np.float32(0.1))


def test_threading_does_not_change_results():
    x, y = random_cloud(2000, 16)
    qid = np.arange(2000, dtype=np.int32)
    a = oracle.knn(x, y, qid, 8, n_threads=1)
    b = oracle.knn(x, y, qid, 8, n_threads=7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
