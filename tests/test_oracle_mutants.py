"""Planted mistakes: each mutant is a copy of the oracle's C source with one
plausible error, built on the CPU into a temporary library.  The pins must
reject every mutant, which shows that they constrain the oracle and not just
restate it.  The real oracle sources are never modified."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
from oracle import build as obuild
from tests import test_oracle_pins as P
from tests import test_oracle_quadtree as Q

MUTANTS = {
    "fused_distance": ("knn_oracle.c", "float dx2 = dx * dx;\n    float dy2 = dy * dy;\n    return dx2 + dy2;",
                       "return __builtin_fmaf(dx, dx, dy * dy);",
                       [P.test_sqdist_is_not_fused]),
    "wrong_operand": ("knn_oracle.c", "float dy = qy - py;", "float dy = qx - py;",
                      [P.test_sqdist_matches_exact_rounding_sequence]),
    "ties_by_descending_id": ("knn_oracle.c", "return a.id < b.id;", "return a.id > b.id;",
                              [lambda: P.test_lattice_closed_form(5)]),
    "heap_picks_smaller_child": ("knn_oracle.c",
                                 "if (r < size && key_less(h[m], h[r])) m = r;",
                                 "if (r < size && key_less(h[r], h[m])) m = r;",
                                 [lambda: P.test_lattice_closed_form(8)]),
    "issuer_not_excluded": ("knn_oracle.c", "if ((int32_t)j == issuer) continue;", "",
                            [lambda: P.test_exhaustive_enumeration_tiny(1)]),
    "first_update_wins": ("knn_oracle.c", "for (int64_t i = 0; i < n_upd; ++i) {",
                          "for (int64_t i = n_upd - 1; i >= 0; --i) {",
                          [P.test_updates_last_one_wins_and_invalid_skipped]),
    "zero_padding": ("knn_oracle.c", "out_d2[r] = INFINITY;", "out_d2[r] = 0.f;",
                     [P.test_padding_and_degenerate_cases]),
    "split_at_capacity": ("quadtree_oracle.c", "int split = (q.count > th ||",
                          "int split = (q.count >= th ||",
                          [lambda: Q.test_leaves_match_definition_tiny(1, 2, 0, False)]),
    "x_in_odd_bits": ("quadtree_oracle.c", "key |= ((cx >> b) & 1u) << (2 * b);",
                      "key |= ((cx >> b) & 1u) << (2 * b + 1); key ^= 0;",
                      [Q.test_morton_known_values]),
    "leaves_sorted_by_z": ("quadtree_oracle.c",
                           "return (uint64_t)q->z << (2 * (L_global_for_sort - q->level));",
                           "return (uint64_t)q->z;",
                           [Q.test_paper_leaf_order_example]),
}


def build_mutant(tmp_path, name):
    fname, old, new, _ = MUTANTS[name]
    d = tmp_path / name
    d.mkdir()
    for s in obuild.SOURCES + ["oracle.h"]:
        shutil.copy(os.path.join(obuild.HERE, s), d / s)
    src = (d / fname).read_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    (d / fname).write_text(src.replace(old, new))
    lib = d / "libmutant.so"
    subprocess.run(["gcc", *obuild.CFLAGS, "-o", str(lib),
                    *[str(d / s) for s in obuild.SOURCES], "-lm"], check=True)
    return str(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(tmp_path, monkeypatch, name):
    path = build_mutant(tmp_path, name)
    real = oracle.lib()
    mutant = ctypes.CDLL(path)
    for fn in ("oracle_apply_updates", "oracle_sqdist", "oracle_knn", "oracle_morton_key",
               "oracle_pr_quadtree"):
        getattr(mutant, fn).restype = getattr(real, fn).restype
        getattr(mutant, fn).argtypes = getattr(real, fn).argtypes
    monkeypatch.setattr(oracle, "_lib", mutant)
    caught = 0
    for pin in MUTANTS[name][3]:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught == len(MUTANTS[name][3]), f"pins did not reject mutant {name}"
