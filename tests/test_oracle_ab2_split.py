"""Pins for the oracle's split evaluation of the AB2 step (Section 3.2, the paragraph after eq.
AB2_): each sub-operation is followed by its own rank reduction.

Untruncated, both readings equal the full-grid AB2 step.  Truncated, each reduction T moves its
argument x by at most tol |x| (the HSVD bound when the rank cap does not bind), so the split
result differs from the exact AB2 step by at most the propagated sum of those moves, with
|S|_2 <= sum_i |A_i|_2 for the Kronecker-sum S = dt L."""
import numpy as np
import pytest

from oracle import fullgrid as FG
from oracle import ht as H
from oracle.problems import advection_A
from paper_1803_10270_gb300.inputs import advection_case


def _setup(d=4, n=6, seed=61):
    case = advection_case(d, n, seed=seed)
    A = advection_A(case)
    u0 = H.from_cp(np.ones(2), case.ic_factors())
    u1, _ = H.step_rk2_poly(u0, A, 0.0, 64)
    return case, A, u0, u1


@pytest.mark.parametrize("variant", ["argument", "difference"])
def test_split_untruncated_equals_full_grid_ab2(variant):
    case, A, u0, u1 = _setup()
    got, _ = H.step_ab2_split(u1, u0, A, 0.0, 64, variant)
    want = FG.ab2_step(H.to_full(u1), H.to_full(u0), case.c, case.h, case.dt)
    assert np.abs(H.to_full(got) - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_split_within_propagated_truncation_bound(tol):
    """The 'argument' split: e_w <= tol |3u - u_prev|; e_v <= tol |S w~| + |S| e_w;
    e <= tol |u + v~/2| + e_v / 2, against the exact step (w~, v~: the truncated values).  The
    'difference' split: e_w <= tol |u - u_prev|, e_a <= tol |S u|, e_b <= tol |S w~| + |S| e_w,
    e <= tol |u + a~ + b~/2| + e_a + e_b / 2."""
    case, A, u0, u1 = _setup(seed=62)
    S2 = sum(np.linalg.norm(Ai, 2) for Ai in A)
    full = H.to_full
    want = FG.ab2_step(full(u1), full(u0), case.c, case.h, case.dt)
    nrm = np.linalg.norm
    # argument
    got, _ = H.step_ab2_split(u1, u0, A, tol, 64, "argument")
    w = H.truncate(H.add(3.0, u1, -1.0, u0), tol, 64)[0]
    v = H.truncate(H.apply_kron_sum_poly(w, A, (0.0, 1.0)), tol, 64)[0]
    e_w = tol * nrm(3 * full(u1) - full(u0))
    e_v = tol * nrm(full(H.apply_kron_sum_poly(w, A, (0.0, 1.0)))) + S2 * e_w
    bound = tol * nrm(full(u1) + 0.5 * full(v)) + 0.5 * e_v
    assert nrm(full(got) - want) <= bound * (1 + 1e-9)
    # difference
    got, _ = H.step_ab2_split(u1, u0, A, tol, 64, "difference")
    w = H.truncate(H.add(1.0, u1, -1.0, u0), tol, 64)[0]
    a = H.truncate(H.apply_kron_sum_poly(u1, A, (0.0, 1.0)), tol, 64)[0]
    b = H.truncate(H.apply_kron_sum_poly(w, A, (0.0, 1.0)), tol, 64)[0]
    e_w = tol * nrm(full(u1) - full(u0))
    e_a = tol * nrm(full(H.apply_kron_sum_poly(u1, A, (0.0, 1.0))))
    e_b = tol * nrm(full(H.apply_kron_sum_poly(w, A, (0.0, 1.0)))) + S2 * e_w
    bound = tol * nrm(full(u1) + full(a) + 0.5 * full(b)) + e_a + 0.5 * e_b
    assert nrm(full(got) - want) <= bound * (1 + 1e-9)


def test_split_rejects_unknown_variant():
    case, A, u0, u1 = _setup()
    with pytest.raises(ValueError):
        H.step_ab2_split(u1, u0, A, 0.0, 64, "neither")
