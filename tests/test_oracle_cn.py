"""Pins of the oracle's Crank-Nicolson CP-ALS step (Section 3.3, eqs. CNFDE, ALS2, ML, MR)."""
import numpy as np

from oracle import cn_als as CN
from oracle.cp import CP, to_full
from oracle.problems import kinetic_terms
from paper_1803_10270_gb300.inputs import kinetic_case


def rand_cp(rng, d, n, r):
    return CP(rng.uniform(0.5, 1.5, r), [rng.standard_normal((n, r)) for _ in range(d)])


def full_op(E, coefs, d, n):
    A = np.zeros((n ** d, n ** d))
    for c, Ee in zip(coefs, E):
        K = np.ones((1, 1))
        for F in Ee:
            K = np.kron(K, np.eye(n) if F is None else F)
        A += c * K
    return A


def test_mode_solve_equals_bruteforce_least_squares():
    """Each mode solve is the exact minimiser of |A x - B x_n| over that factor: the same V as
    a library least-squares solve on the full grid (A unfolded column by column)."""
    rng = np.random.default_rng(7)
    d, n, r = 3, 5, 2
    alphas = [0.7, -0.4]
    factors = [[rng.standard_normal((n, n)), None, np.diag(rng.standard_normal(n))],
               [None, np.outer(rng.standard_normal(n), rng.standard_normal(n)), rng.standard_normal((n, n))]]
    dt = 0.3
    xn = rand_cp(rng, d, n, 2)
    X = [rng.standard_normal((n, r)) for _ in range(d)]
    eta, zeta, E = CN.cn_terms(alphas, factors, dt, d)
    A = full_op(E, eta, d, n)
    b = full_op(E, zeta, d, n) @ to_full(xn).reshape(-1)
    for q in range(d):
        V = CN.mode_solve(X, xn, eta, zeta, E, q)
        cols = []
        for l in range(r):
            for i in range(n):
                Xi = [f.copy() for f in X]
                Xi[q] = np.zeros((n, r))
                Xi[q][i, l] = 1.0
                cols.append(A @ to_full(CP(np.ones(r), Xi)).reshape(-1))
        D = np.stack(cols, axis=1)                  # column i + n l
        v, *_ = np.linalg.lstsq(D, b, rcond=None)
        assert np.allclose(V, v.reshape(n, r, order="F"), rtol=1e-9, atol=1e-11 * np.abs(v).max()), q
        X[q] = V


def test_pure_relaxation_closed_form():
    """L = -nu I: the Crank-Nicolson step is x_n (1 - nu dt/2)/(1 + nu dt/2), reached exactly."""
    rng = np.random.default_rng(8)
    d, n, nu, dt = 4, 6, 1.3, 0.2
    xn = rand_cp(rng, d, n, 3)
    x, eps = CN.cn_als_step(xn, xn, [-nu], [[None] * d], dt, 2)
    g = (1 - 0.5 * nu * dt) / (1 + 0.5 * nu * dt)
    assert np.allclose(to_full(x), g * to_full(xn), rtol=0, atol=1e-12 * np.abs(to_full(xn)).max())
    assert eps[1] < 1e-24


def test_uniform_maxwellian_is_a_fixed_point():
    """f = M(v) (uniform in x) has L f = 0 for the linearised kinetic operator (transport of an
    x-constant and f - M rho = 0 with rho = 1), so A x = B f is solved by x = f."""
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    ones, m = np.ones(kc.n), kc.maxwellian()
    f = CP(np.ones(1), [ones[:, None]] * 3 + [m[:, None]] * 3)
    x, eps = CN.cn_als_step(f, f, alphas, factors, kc.dt, 2)
    assert np.allclose(to_full(x), to_full(f), rtol=0, atol=1e-13 * to_full(f).max())
    assert CN.cn_residual(x, f, alphas, factors, kc.dt) < 1e-13 * np.linalg.norm(to_full(f))


def test_residual_never_increases():
    rng = np.random.default_rng(9)
    kc = kinetic_case(4)
    alphas, factors = kinetic_terms(kc)
    xn = CP(np.ones(2), [np.abs(rng.standard_normal((4, 2))) + 0.2 for _ in range(6)])
    eta, zeta, E = CN.cn_terms(alphas, factors, kc.dt * 5, 6)
    X = [f * 1.1 for f in xn.factors]
    prev = CN.cn_residual(CP(np.ones(2), X), xn, alphas, factors, kc.dt * 5)
    for _ in range(2):
        for q in range(6):
            X[q] = CN.mode_solve(X, xn, eta, zeta, E, q)
            res = CN.cn_residual(CP(np.ones(2), X), xn, alphas, factors, kc.dt * 5)
            assert res <= prev * (1 + 1e-12) + 1e-15
            prev = res


def test_damped_jacobi_reaches_the_relaxation_closed_form():
    """The parallel variant (Appendix B, Algorithm 1: every mode from the same iterate, the
    increment damped by 1/4) converges to the same step as Gauss-Seidel: for L = -nu I the
    closed form (1 - nu dt/2)/(1 + nu dt/2) x_n; its increments shrink monotonically there."""
    rng = np.random.default_rng(10)
    d, n, nu, dt = 3, 5, 0.9, 0.3
    xn = rand_cp(rng, d, n, 2)
    x, eps = CN.cn_als_step(xn, xn, [-nu], [[None] * d], dt, 80, variant="jacobi_damped")
    g = (1 - 0.5 * nu * dt) / (1 + 0.5 * nu * dt)
    assert np.allclose(to_full(x), g * to_full(xn), rtol=0, atol=1e-10 * np.abs(to_full(xn)).max())
    above = [e for e in eps[1:] if e > 1e-24 * eps[0]]      # above the rounding floor
    assert all(b <= a * (1 + 1e-12) for a, b in zip(above, above[1:]))
    assert eps[-1] < 1e-24 * eps[0]


def test_damped_jacobi_step_is_a_stationary_point():
    """At convergence the parallel variant's iterate makes every mode's normal equations hold:
    solving any mode again leaves it unchanged (kinetic operator, n = 4, rank 2)."""
    kc = kinetic_case(4)
    alphas, factors = kinetic_terms(kc)
    rng = np.random.default_rng(11)
    xn = CP(np.ones(2), [np.abs(rng.standard_normal((4, 2))) + 0.2 for _ in range(6)])
    x, eps = CN.cn_als_step(xn, xn, alphas, factors, kc.dt, 400, variant="jacobi_damped")
    eta, zeta, E = CN.cn_terms(alphas, factors, kc.dt, 6)
    for q in range(6):
        V = CN.mode_solve(x.factors, xn, eta, zeta, E, q)
        assert np.allclose(V, x.factors[q], rtol=1e-10, atol=1e-12 * np.abs(V).max()), q
