"""Pins for the Morton-code and PR-quadtree oracle (Section 4.1.1), CPU only."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def interleave_by_loop(cx, cy, L):
    """Morton code written out bit by bit: bit b of x -> bit 2b, of y -> bit 2b+1."""
    key = 0
    for b in range(L):
        key += ((cx >> b) & 1) * (4 ** b)
        key += ((cy >> b) & 1) * 2 * (4 ** b)
    return key


def test_morton_known_values():
    # level 1: quadrant numbering (x low bit, y high bit)
    assert oracle.morton_key(0.25, 0.25, 1) == 0
    assert oracle.morton_key(0.75, 0.25, 1) == 1
    assert oracle.morton_key(0.25, 0.75, 1) == 2
    assert oracle.morton_key(0.75, 0.75, 1) == 3
    # level 2: cell (3, 0) -> 0b0101, cell (0, 3) -> 0b1010
    assert oracle.morton_key(0.9, 0.1, 2) == 5
    assert oracle.morton_key(0.1, 0.9, 2) == 10
    # clamping outside the square
    assert oracle.morton_key(-1.0, 2.0, 2) == interleave_by_loop(0, 3, 2)
    assert oracle.morton_key(float("nan"), 0.9, 2) == interleave_by_loop(0, 3, 2)


def test_morton_matches_bit_loop_and_ancestor_rule():
    r = np.random.default_rng(0)
    L = 16
    for x, y in r.random((3000, 2)).astype(np.float32):
        cx = int(np.floor(np.float64(x) * 2 ** L))
        cy = int(np.floor(np.float64(y) * 2 ** L))
        key = oracle.morton_key(x, y, L)
        assert key == interleave_by_loop(cx, cy, L)
        # the level-l ancestor is floor(z / 4^(L-l)) (Section 4.1.1)
        for l in (1, 5, 9):
            assert key // 4 ** (L - l) == interleave_by_loop(cx >> (L - l), cy >> (L - l), l)


def read_example():
    spec = {}
    with open(os.path.join(GOLDEN, "leaf_order_example.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            head, *rest = line.split()
            spec[head] = [tuple(int(v) for v in t.split(",")) for t in rest] \
                if head != "l_deep" else int(rest[0])
    return spec


def test_paper_leaf_order_example():
    spec = read_example()
    L = spec["l_deep"]
    # one object in quadrants 0 and 3, one object in each child of quadrants 1 and 2;
    # th = 2 splits the root (10 objects) and quadrants 1, 2 (4 objects each)
    pts = [(0.25, 0.25), (0.75, 0.75)]
    for qx, qy in ((0.5, 0.0), (0.0, 0.5)):
        for cx, cy in ((0, 0), (1, 0), (0, 1), (1, 1)):
            pts.append((qx + 0.25 * cx + 0.125, qy + 0.25 * cy + 0.125))
    x = np.array([p[0] for p in pts], np.float32)
    y = np.array([p[1] for p in pts], np.float32)
    t = oracle.pr_quadtree(x, y, L, th=2)
    labels = [(int(l), int(z) * 4 ** (L - int(l))) for l, z in zip(t["level"], t["z"])]
    assert labels == spec["leaves"]
    pos = labels.index(spec["query"][0])
    assert labels[pos + 1:] == spec["right"]
    assert labels[:pos][::-1] == spec["left"]


def leaves_by_definition(x, y, L, th, min_level=0, emit_empty=False):
    """Brute force: count every quadrant of every level directly from the cell
    coordinates; a quadrant is a leaf when it is not split (count <= th and
    level >= min_level, or empty, or level L) while its parent is split."""
    cx = np.floor(x.astype(np.float64) * 2 ** L).astype(np.int64)
    cy = np.floor(y.astype(np.float64) * 2 ** L).astype(np.int64)

    def count(l, qx, qy):
        s = L - l
        return int(np.sum(((cx >> s) == qx) & ((cy >> s) == qy)))

    def split(l, c):
        return l < L and c > 0 and (c > th or l < min_level)

    out = []

    def visit(l, qx, qy):
        c = count(l, qx, qy)
        if split(l, c):
            for dy in (0, 1):
                for dx in (0, 1):
                    visit(l + 1, 2 * qx + dx, 2 * qy + dy)
        elif c > 0 or emit_empty:
            out.append((l, interleave_by_loop(qx, qy, l), c))

    visit(0, 0, 0)
    out.sort(key=lambda t: t[1] * 4 ** (L - t[0]))
    return out


@pytest.mark.parametrize("seed,th,min_level,emit_empty",
                         [(0, 1, 0, True), (1, 2, 0, False), (2, 3, 2, False),
                          (3, 5, 0, True), (4, 1, 3, False), (5, 8, 1, True)])
def test_leaves_match_definition_tiny(seed, th, min_level, emit_empty):
    r = np.random.default_rng(seed)
    L = 4
    n = int(r.integers(0, 40))
    x = (r.integers(0, 16, n) / 16.0 + r.random(n) / 64).astype(np.float32)
    y = (r.integers(0, 16, n) / 16.0 + r.random(n) / 64).astype(np.float32)
    if n > 6:
        x[:4] = x[4]
        y[:4] = y[4]   # duplicates that can only end at level L
    t = oracle.pr_quadtree(x, y, L, th, min_level, emit_empty)
    got = list(zip(t["level"].tolist(), t["z"].tolist(), t["count"].tolist()))
    assert got == leaves_by_definition(x, y, L, th, min_level, emit_empty)
    # intervals: consecutive in the sorted order, covering [0, n)
    st = t["start"][t["count"] > 0]
    ct = t["count"][t["count"] > 0]
    assert st[0] == 0 if n else True
    assert np.all(st[1:] == st[:-1] + ct[:-1])
    assert ct.sum() == n


@pytest.mark.parametrize("th", [1, 4, 32])
def test_quadtree_invariants_random(th):
    r = np.random.default_rng(th)
    n = 3000
    L = 16
    x = np.concatenate([r.random(n // 2), 0.3 + 0.01 * r.standard_normal(n // 2)])
    y = np.concatenate([r.random(n // 2), 0.6 + 0.01 * r.standard_normal(n // 2)])
    x = np.clip(x, 0, 1 - 2 ** -24).astype(np.float32)
    y = np.clip(y, 0, 1 - 2 ** -24).astype(np.float32)
    x[:50] = x[50]   # coincident objects force leaves at level L
    y[:50] = y[50]
    t = oracle.pr_quadtree(x, y, L, th, emit_empty=True)
    lv, z, st, ct = t["level"], t["z"].astype(np.int64), t["start"], t["count"]
    # leaves tile the domain
    assert sum(4 ** (L - int(l)) for l in lv) == 4 ** L
    # every leaf obeys the capacity unless it is at level L
    assert np.all((ct <= th) | (lv == L))
    assert np.any(lv == L) and ct[lv == L].max() >= 50
    # the parent of every non-root leaf holds more than th objects
    keys = np.array([oracle.morton_key(a, b, L) for a, b in zip(x, y)], np.int64)
    for l, zz in zip(lv, z):
        if l == 0:
            continue
        parent = zz >> 2
        assert np.sum((keys >> (2 * (L - l + 1))) == parent) > th
    # the sorted order is by key, then id
    order = t["order"]
    k_sorted = keys[order]
    assert np.all((k_sorted[1:] > k_sorted[:-1])
                  | ((k_sorted[1:] == k_sorted[:-1]) & (order[1:] > order[:-1])))
    # members of each leaf carry the leaf's code
    for l, zz, s, c in zip(lv, z, st, ct):
        if c:
            assert np.all((k_sorted[s:s + c] >> (2 * (L - l))) == zz)
