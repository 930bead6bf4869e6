"""Pins for the oracle's full-grid stepper and tree (CPU only)."""
import math

import numpy as np
import pytest

from oracle import fullgrid as FG
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case
from tests.closed_forms import fourier_rk2


def test_tree_matches_paper_grouping_d6():
    # Section 2.2, eq. HTD: {1,2,3}|{4,5,6}, then {1}|{2,3} and {4}|{5,6}
    t = build_tree(6)
    assert t.n_nodes == 11
    groups = {(t.lo[k], t.hi[k]) for k in range(t.n_nodes)}
    for g in [(0, 6), (0, 3), (3, 6), (0, 1), (1, 3), (3, 4), (4, 6)]:
        assert g in groups
    assert t.children[0] == (1, 2)
    assert sum(t.is_leaf(k) for k in range(t.n_nodes)) == 6


@pytest.mark.parametrize("d", [2, 3, 5, 6, 7, 12])
def test_tree_node_count_and_depth(d):
    t = build_tree(d)
    assert t.n_nodes == 2 * d - 1
    assert max(t.depth) == math.ceil(math.log2(d))
    leaves = sorted(t.lo[k] for k in range(t.n_nodes) if t.is_leaf(k))
    assert leaves == list(range(d))


@pytest.mark.parametrize("d,n,steps", [(1, 16, 7), (2, 10, 5), (3, 8, 4)])
def test_stepper_matches_fourier_closed_form(d, n, steps):
    case = advection_case(d, n, seed=123 + d)
    u0 = FG.cp_to_full(np.ones(2), case.ic_factors())
    u = FG.rk2_steps(u0, case.c, [case.h] * d, case.dt, steps)
    ref = fourier_rk2(u0, case.c, case.h, case.dt, steps)
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_stepper_mass_conserved():
    case = advection_case(3, 8, seed=7)
    u0 = np.random.default_rng(0).standard_normal((8, 8, 8))
    u = FG.rk2_steps(u0, case.c, [case.h] * 3, case.dt, 6)
    assert abs(u.sum() - u0.sum()) <= 1e-12 * np.abs(u0).sum()


def test_stepper_second_order_vs_exact_shift():
    # u0 = exp(sin(x)), exact solution u0(x - c t); dt = 0.2 h, both errors O(h^2)
    c = 0.7
    errs = []
    for n in (32, 64, 128):
        h = 2 * math.pi / n
        x = np.arange(n) * h
        dt = 0.2 * h
        steps = int(round(1.0 / dt))
        T = steps * dt
        u = FG.rk2_steps(np.exp(np.sin(x)), [c], [h], dt, steps)
        errs.append(np.abs(u - np.exp(np.sin(x - c * T))).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5
