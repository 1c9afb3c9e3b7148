"""Mutation check of the oracle's pins (CPU only).

Each mutant plants one plausible mistake in a copy of the oracle's C source
(a strict comparison where the closed rule needs a non-strict one, a dropped
dimension, a wrong descent condition, a stale subtree bound, swapped
operands, an off-by-one in a binary search, a wrong tie order).  The copy is
compiled into a temporary library and the pin suite of ``test_oracle.py`` is
run against it: every mutant must fail at least one pin.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import tests.test_oracle as T

MUTANTS = {
    "closed_rule_strict_low": ("return xlo <= yhi && ylo <= xhi;", "return xlo < yhi && ylo <= xhi;"),
    "bf_drops_dimensions": ("for (int k = 0; k < d; ++k) {", "for (int k = 0; k < 1; ++k) {"),
    "itm_drops_last_dimension": ("for (int k = 1; k < q->d; ++k) {",
                                 "for (int k = 1; k < q->d - 1; ++k) {"),
    "right_descent_strict": ("(qh >= x->lo)", "(qh > x->lo)"),
    "prune_on_equal_upper": ("!(x->maxupper < ql)", "!(x->maxupper <= ql)"),
    "prune_on_equal_lower": ("!(x->minlower > qh)", "!(x->minlower >= qh)"),
    "walk_skips_left_subtrees": ("x = t->v[x].left;", "x = -1;"),
    "swapped_lo_hi_in_filter": ("intersect_1d(q->slo[si], q->shi[si],",
                                "intersect_1d(q->shi[si], q->slo[si],"),
    "maxupper_ignores_right_child": ("if (t->v[p->right].maxupper > mu) mu = t->v[p->right].maxupper;",
                                     ";"),
    "rotation_leaves_stale_bounds": ("    t->v[x].right = y;\n    it_fix(t, y);", "    t->v[x].right = y;"),
    "bits_count_le_off_by_one": ("if (v[mid] <= key) a = mid + 1; else b = mid;",
                                 "if (v[mid] < key) a = mid + 1; else b = mid;"),
    "tie_order_reversed": ("if (a->hi < b->hi) return 1;", "if (a->hi > b->hi) return 1;"),
}


def pins():
    yield lambda: [T.test_intersect_1d(*c) for c in [((0, 1), (1, 2), True, False),
                                                     ((1, 1), (1, 1), True, False)]]
    for d in (1, 2, 3):
        for k in (2, 3, 6):
            yield lambda d=d, k=k: T.test_lattice_closed_forms(d, k)
    yield lambda: T.test_fig1_worked_example(0)
    yield lambda: T.test_fig1_worked_example(1)
    for d in (1, 2, 3):
        for f in (0, 1):
            yield lambda d=d, f=f: T.test_bf_equals_itm_on_grids(d, f)
    yield T.test_bits_equals_itm_grid_ties
    yield T.test_tree_order_and_height
    yield T.test_invariants
    yield T.test_bf_equals_itm_clustered


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", str(so), str(path)])
    monkeypatch.setattr(oracle, "_lib", oracle.bind(ctypes.CDLL(str(so))))
    for pin in pins():
        try:
            pin()
        except AssertionError:
            return
    pytest.fail(f"mutant {name} passed every pin")
