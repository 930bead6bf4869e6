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


# ---- moments of the kinetic solution (Section 4.2: density, mean velocity, temperature) ----
def grid_moments(f, kc):
    """x-averaged density, momentum and second moment of a full-grid f on (x1,x2,x3,v1,v2,v3):
    the discrete forms of the paper's <rho>, <rho><u> and sum_v |v|^2 f (eqs. rho0, u0, T0)."""
    v = kc.vgrid()
    w = (kc.hx / (2 * np.pi)) ** 3 * kc.hv ** 3
    V = np.meshgrid(v, v, v, indexing="ij")
    fv = f.reshape((kc.n ** 3,) + (kc.n,) * 3).sum(axis=0)      # sum over the x points
    rho = w * fv.sum()
    mom = np.array([w * (Vd * fv).sum() for Vd in V])
    e2 = w * ((V[0] ** 2 + V[1] ** 2 + V[2] ** 2) * fv).sum()
    return rho, mom, e2


def test_exact_crank_nicolson_moment_recursions():
    """The discrete kinetic operator keeps the x-averaged mass (periodic central differences sum
    to zero over x, and sum_v h^3 M = 1), relaxes the momentum at rate nu (sum_v v M = 0 on the
    symmetric grid) and the second moment E towards 3 c2 rho (c2 = sum_j h v_j^2 m_j).  Hence the
    exact Crank-Nicolson step, A f1 = B f0 solved on the full grid with the oracle's eta / zeta,
    keeps rho and multiplies the momentum and E - 3 c2 rho by g = (1 - nu dt/2) / (1 + nu dt/2),
    for any f0 (here the x-dependent kinetic initial condition, n = 4).  A sign error in eta or
    zeta, a transposed Maxwellian projector or a lost term breaks one of the three."""
    from paper_1803_10270_gb300.inputs import kinetic_ic
    kc = kinetic_case(4)
    alphas, factors = kinetic_terms(kc)
    dt = 5 * kc.dt
    eta, zeta, E = CN.cn_terms(alphas, factors, dt, 6)
    A = full_op(E, eta, 6, kc.n)
    B = full_op(E, zeta, 6, kc.n)
    w, F = kinetic_ic(kc)
    f = to_full(CP(w, F)).reshape(-1)
    g = (1 - 0.5 * kc.nu * dt) / (1 + 0.5 * kc.nu * dt)
    c2 = kc.hv * float(np.sum(kc.vgrid() ** 2 * kc.maxwellian()))
    rho0, mom0, e0 = grid_moments(f, kc)
    assert np.abs(mom0).max() > 1e-3 * rho0          # a state away from equilibrium
    for step in range(1, 4):
        f = np.linalg.solve(A, B @ f)
        rho, mom, e2 = grid_moments(f, kc)
        assert abs(rho - rho0) <= 1e-13 * rho0, step
        assert np.allclose(mom, g ** step * mom0, rtol=1e-11, atol=1e-13 * rho0), step
        assert abs((e2 - 3 * c2 * rho) - g ** step * (e0 - 3 * c2 * rho0)) <= 1e-12 * e0, step


def test_x_uniform_relaxation_reaches_the_closed_form():
    """An x-uniform f0 = 1 x 1 x 1 x g1(v1) g2(v2) g3(v3) sees no transport, so the exact
    Crank-Nicolson step is f1 = g f0 + (1 - g) rho M (rho = sum_v h^3 f0): rank 2.  The CP-ALS
    step of rank 2 from the guess [f0, 0.3 M] reaches it to rounding, so its moments follow the
    recursions above exactly (n = 8, dt = 5x the explicit step, 5 sweeps)."""
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    v, m, ones = kc.vgrid(), kc.maxwellian(), np.ones(kc.n)
    f0 = CP(np.ones(1), [ones[:, None]] * 3 +
            [(m * (1 + 0.3 * v))[:, None], (m * (1 - 0.2 * v + 0.05 * v * v))[:, None], m[:, None]])
    dt = 5 * kc.dt
    g = (1 - 0.5 * kc.nu * dt) / (1 + 0.5 * kc.nu * dt)
    rho = float(np.prod([kc.hv * f0.factors[3 + k][:, 0].sum() for k in range(3)]))
    Mx = to_full(CP(np.ones(1), [ones[:, None]] * 3 + [m[:, None]] * 3))
    exact = g * to_full(f0) + (1 - g) * rho * Mx
    x0 = CP(np.array([1.0, 0.3]),
            [np.concatenate([f0.factors[k], (ones if k < 3 else m)[:, None]], axis=1) for k in range(6)])
    x, _ = CN.cn_als_step(f0, x0, alphas, factors, dt, 5)
    assert np.linalg.norm(to_full(x) - exact) <= 1e-13 * np.linalg.norm(exact)
    r0, p0, _ = grid_moments(to_full(f0), kc)
    r1, p1, _ = grid_moments(to_full(x), kc)
    assert abs(r1 - r0) <= 1e-13 * r0
    assert np.allclose(p1, g * p0, rtol=1e-11, atol=1e-13 * r0)


def test_equilibrium_moments_stay_constant():
    """The paper's steady-state check: from the Maxwellian f_eq, CP-ALS Crank-Nicolson steps keep
    the average density, velocity and temperature (eqs. rho0, u0, T0) at their initial values."""
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    ones, m = np.ones(kc.n), kc.maxwellian()
    f = CP(np.ones(1), [ones[:, None]] * 3 + [m[:, None]] * 3)
    r0, p0, e0 = grid_moments(to_full(f), kc)
    x = f
    for _ in range(3):
        x, _ = CN.cn_als_step(x, x, alphas, factors, 5 * kc.dt, 3)
    r, p, e2 = grid_moments(to_full(x), kc)
    assert abs(r - r0) <= 1e-13 * r0
    assert np.abs(p).max() <= 1e-14 * r0 and np.abs(p0).max() <= 1e-14 * r0
    t0, t = e0 / (3 * r0), (e2 - (p ** 2).sum() / r) / (3 * r)     # |v - <u>|^2 form of eq. T0
    assert abs(t - t0) <= 1e-13 * t0
