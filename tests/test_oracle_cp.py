"""Pins for the CP / ALS oracle."""
import numpy as np
import pytest

from oracle import cp as C
from oracle import fullgrid as FG
from oracle import ht as H
from paper_1803_10270_gb300.inputs import advection_case, cp_random_factors
from tests.closed_forms import fourier_rk2


def test_cp_apply_matches_fourier():
    d, n = 3, 6
    case = advection_case(d, n, seed=3)
    x = C.CP(np.array([1.0, -0.4]), cp_random_factors([n] * d, 2, seed=1))
    A = [case.dt * (-case.c[i]) * H.central_diff_matrix(n, case.h) for i in range(d)]
    y = C.apply_kron_sum_rk2(x, A)
    assert y.rank == 2 * (1 + 2 * d + d * (d - 1) // 2)
    ref = fourier_rk2(C.to_full(x), case.c, case.h, case.dt, 1)
    assert np.abs(C.to_full(y) - ref).max() <= 1e-13 * np.abs(ref).max()


def test_mode_update_is_bruteforce_least_squares():
    d, n, r = 3, 4, 2
    rng = np.random.default_rng(0)
    y = C.CP(rng.uniform(0.5, 1.5, 5), [rng.standard_normal((n, 5)) for _ in range(d)])
    xf = [rng.standard_normal((n, r)) for _ in range(d)]
    Yfull = C.to_full(y)
    for k in range(d):
        Xk = C._mode_solve(y, xf, k)
        # unfold: Yfull[..] = sum_l X_k[i_k, l] prod_{j != k} X_j[i_j, l]
        others = [j for j in range(d) if j != k]
        Z = np.ones((1, r))
        for j in others:
            Z = np.einsum("al,bl->abl", Z, xf[j]).reshape(-1, r)
        # Z rows ordered with the earlier 'other' index slowest; match by transposing Yfull
        Yk = np.moveaxis(Yfull, k, 0).reshape(n, -1)
        sol, *_ = np.linalg.lstsq(Z, Yk.T, rcond=None)
        assert np.abs(sol.T - Xk).max() < 1e-10 * np.abs(sol).max()


def test_gs_residual_monotone_and_fixed_point():
    d, n = 4, 6
    rng = np.random.default_rng(2)
    y = C.CP(rng.uniform(0.5, 1.5, 7), [rng.standard_normal((n, 7)) for _ in range(d)])
    x0 = C.CP(np.ones(3), [rng.standard_normal((n, 3)) for _ in range(d)])
    prev = C.residual(y, x0)
    x = x0
    for _ in range(6):
        x, _ = C.als_sweeps(y, x, 1)
        cur = C.residual(y, x)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    # exact rank-3 target, init = truth: fixed point
    z = C.CP(np.array([2.0, 1.0, 0.5]), [rng.standard_normal((n, 3)) for _ in range(d)])
    xz, eps = C.als_sweeps(z, z, 2)
    assert np.abs(C.to_full(xz) - C.to_full(z)).max() < 1e-10 * np.abs(C.to_full(z)).max()
    assert eps[-1] < 1e-10


@pytest.mark.parametrize("variant", ["gs", "jacobi_damped"])
def test_rank1_target_recovered(variant):
    d, n = 3, 5
    rng = np.random.default_rng(4)
    truth = C.CP(np.array([3.0]), [rng.standard_normal((n, 1)) for _ in range(d)])
    init = C.CP(np.array([1.0]), [f + 0.3 * rng.standard_normal(f.shape) for f in truth.factors])
    sweeps = 30 if variant == "gs" else 200
    x, eps = C.als_sweeps(truth, init, sweeps, variant)
    ft = C.to_full(truth)
    assert np.linalg.norm(C.to_full(x) - ft) < 1e-8 * np.linalg.norm(ft)
    assert eps[-1] < eps[0]


def test_pad_keeps_tensor_when_padding_zero():
    d, n = 3, 4
    x = C.CP(np.array([1.0, 2.0]), cp_random_factors([n] * d, 2, seed=5))
    p = C.pad(x, 5, [np.zeros((n, 3))] * d)
    assert p.rank == 5
    assert np.abs(C.to_full(p) - C.to_full(x)).max() < 1e-12 * np.abs(C.to_full(x)).max()


def test_singular_gram_takes_the_shift_and_keeps_the_fit():
    """An initial guess with an all-zero column makes every Gamma_k exactly singular, so the
    Cholesky factorisation fails and the shift by 1e-14 tr(Gamma_k)/r (Section 2.1: ill-conditioned
    ALS systems are regularised, here only on failure) is taken.  The zero column then stays zero
    (its right-hand side vanishes) and the fit equals the rank-3 fit without it to rounding."""
    rng = np.random.default_rng(3)
    d, n = 3, 6
    y = C.CP(rng.uniform(0.5, 1.5, 5), [rng.standard_normal((n, 5)) for _ in range(d)])
    base = [rng.standard_normal((n, 3)) for _ in range(d)]
    x_zero = C.CP(np.ones(4), [np.hstack([b, np.zeros((n, 1))]) for b in base])
    G = np.ones((4, 4))
    for j in range(1, d):
        G *= x_zero.factors[j].T @ x_zero.factors[j]
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(G)
    a, _ = C.als_sweeps(y, C.CP(np.ones(3), [b.copy() for b in base]), 4)
    b, _ = C.als_sweeps(y, x_zero, 4)
    assert b.weights[3] == 0.0
    assert np.linalg.norm(C.to_full(a) - C.to_full(b)) <= 1e-12 * np.linalg.norm(C.to_full(a))


def test_damped_jacobi_sweep_is_a_quarter_step_from_one_iterate():
    """The parallel variant (Appendix B, Algorithm 1): every mode's minimiser V_k is taken from
    the same iterate (weights folded into the first factor) and each factor moves a quarter of
    the way, X_k <- X_k + (V_k - X_k) / 4; Algorithm 5's measure is max_k |V_k - X_k| / |X_k|.
    V_k by brute-force least squares on the unfolded full grid."""
    d, n, r = 3, 4, 2
    rng = np.random.default_rng(4)
    y = C.CP(rng.uniform(0.5, 1.5, 5), [rng.standard_normal((n, 5)) for _ in range(d)])
    x0 = C.CP(rng.uniform(0.5, 1.5, r), [rng.standard_normal((n, r)) for _ in range(d)])
    # the iterate: unit columns for k >= 1, every norm and weight folded into the first factor
    norms = [np.linalg.norm(f, axis=0) for f in x0.factors]
    it = [x0.factors[0] * (x0.weights * np.prod(norms[1:], axis=0))[None, :]]
    it += [x0.factors[k] / norms[k][None, :] for k in range(1, d)]
    Yfull = C.to_full(y)
    V = []
    for k in range(d):
        Z = np.ones((1, r))
        for j in (j for j in range(d) if j != k):
            Z = np.einsum("al,bl->abl", Z, it[j]).reshape(-1, r)
        sol, *_ = np.linalg.lstsq(Z, np.moveaxis(Yfull, k, 0).reshape(n, -1).T, rcond=None)
        V.append(sol.T)
    want = [it[k] + (V[k] - it[k]) / 4.0 for k in range(d)]
    x1, eps = C.als_sweeps(y, x0, 1, variant="jacobi_damped")
    ref = C.to_full(C.CP(np.ones(r), want))
    assert np.linalg.norm(C.to_full(x1) - ref) <= 1e-12 * np.linalg.norm(ref)
    e_want = max(np.linalg.norm(V[k] - it[k]) / np.linalg.norm(it[k]) for k in range(d))
    assert abs(eps[0] - e_want) <= 1e-10 * e_want


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_residual_equals_full_grid_norm(seed):
    """residual(y, x) (factor Grams, no grid) against |to_full(y) - to_full(x)|_F formed on the
    grid: the error that the ALS of Section 2.1 minimises.  Cases: a generic pair, a fit close
    to its target (cancellation in the Gram identity) and the exact fit (residual 0)."""
    d, n = 4, 5
    rng = np.random.default_rng(100 + seed)
    y = C.CP(rng.uniform(0.5, 1.5, 6), [rng.standard_normal((n, 6)) for _ in range(d)])
    x = C.CP(rng.uniform(0.5, 1.5, 3), [rng.standard_normal((n, 3)) for _ in range(d)])
    full = np.linalg.norm(C.to_full(y) - C.to_full(x))
    assert abs(C.residual(y, x) - full) <= 1e-12 * np.linalg.norm(C.to_full(y))
    # a fit within 1e-4 of its target: the identity still resolves the residual to
    # sqrt(eps) |y| (it subtracts Grams of size |y|^2)
    near = C.CP(y.weights.copy(), [f + 1e-4 * rng.standard_normal(f.shape) for f in y.factors])
    full = np.linalg.norm(C.to_full(y) - C.to_full(near))
    ny = np.linalg.norm(C.to_full(y))
    assert abs(C.residual(y, near) - full) <= 1e-7 * ny
    assert 0.5 * full < C.residual(y, near) < 2.0 * full
    assert C.residual(y, y) <= 1e-7 * ny
    # a scaled copy: |y - a y| = |1 - a| |y| exactly
    half = C.CP(0.5 * y.weights, [f.copy() for f in y.factors])
    assert abs(C.residual(y, half) - 0.5 * ny) <= 1e-12 * ny
