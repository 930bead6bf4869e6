"""Oracle pins for the variable-coefficient advection operator (Section 4.1, eq. PDE-advR,
Table tab:ordering0): the paper's term table, the operator on a shifted Gaussian against its
closed form, the HEUN2 stepper against the exact semi-discrete flow exp(t L_h) (second order in
dt), and the characteristic solution at the paper's evaluation point."""
import math
import os

import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import varcoef_terms
from paper_1803_10270_gb300.inputs import varcoef_case
from tests.closed_forms import varcoef_exact, varcoef_L_shifted_gaussian

HERE = os.path.dirname(__file__)


def read_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "varcoef_operator_terms.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_varcoef_terms_follow_the_paper_table():
    """Term q of the oracle's operator is row q of Table tab:ordering0 (N = 3): coefficient
    -C_jk and the 1-D factors identity / derivative / multiplication by z / z times derivative."""
    case = varcoef_case(3, 10, zmax=4.0)
    alphas, factors = varcoef_terms(case)
    n, h, z = case.n, case.h, case.z()
    D = np.zeros((n, n))
    for j in range(n):
        D[j, (j + 1) % n] = 1.0 / (2.0 * h)
        D[j, (j - 1) % n] = -1.0 / (2.0 * h)
    named = {"d": D, "z": np.diag(z), "zd": np.diag(z) @ D}
    rows = read_rows()
    assert len(rows) == len(alphas) == 9
    for q, row in enumerate(rows):
        assert int(row[0]) == q + 1
        j, k = int(row[1][2]) - 1, int(row[1][3]) - 1          # "-Cjk"
        assert alphas[q] == -case.C[j, k]
        for i, tok in enumerate(row[2:]):
            if tok == "1":
                assert factors[q][i] is None
            else:
                assert np.array_equal(factors[q][i], named[tok]), f"term {q + 1} dim {i}"


def ht_of_gaussian(case, mu):
    fac = [np.exp(-(case.z() - m) ** 2)[:, None] for m in mu]
    return OH.from_cp(np.ones(1), fac)


def fd_error_bound(case, mu):
    """Pointwise bound of |L_h g - L g| for g = prod_i g_i(z_i), g_i = exp(-(z_i - mu_i)^2): the
    central difference of g_j errs by at most (h^2 / 6) times the largest third derivative of
    g_j on [z_j - h, z_j + h] (Taylor), times the transport speed |(C z)_j| and the other
    factors g_i(z_i)."""
    h, z, N = case.h, case.z(), case.N
    s = np.linspace(-1.0, 1.0, 401) * h
    loc = []
    for m in mu:
        x = (z[:, None] + s[None, :]) - m
        loc.append(np.abs((-8 * x ** 3 + 12 * x) * np.exp(-x ** 2)).max(axis=1))
    gs = [np.exp(-(z - m) ** 2) for m in mu]
    Zs = np.meshgrid(*([z] * N), indexing="ij")
    b = np.zeros(Zs[0].shape)
    for j in range(N):
        speed = np.abs(sum(case.C[j, k] * Zs[k] for k in range(N)))
        term = np.ones(Zs[0].shape)
        for i in range(N):
            shape = [1] * N
            shape[i] = -1
            term = term * (loc[i] if i == j else gs[i]).reshape(shape)
        b += speed * term
    return b * h ** 2 / 6.0


@pytest.mark.parametrize("N,n", [(2, 96), (3, 40)])
def test_varcoef_operator_on_shifted_gaussian(N, n):
    """L_h g against the closed form 2 g (C z).(z - mu): within the central-difference bound
    everywhere (plus 1e-10 for the periodic wrap at the box edge, where g is about e^-29 and the
    stencil reaches the opposite side); with C transposed (a plausible index slip) the same
    comparison fails."""
    case = varcoef_case(N, n, zmax=6.0)
    mu = [0.5, -0.3, 0.2][:N]
    u = ht_of_gaussian(case, mu)
    alphas, factors = varcoef_terms(case)
    Lu = OH.to_full(OH.apply_separable(u, alphas, factors))
    exact = varcoef_L_shifted_gaussian([case.z()] * N, case.C, mu)
    bound = fd_error_bound(case, mu)
    err = np.abs(Lu - exact)
    assert np.all(err <= 1.01 * bound + 1e-10)
    # planted transposition in the oracle's coefficients
    case_t = varcoef_case(N, n, zmax=6.0)
    case_t.C = case.C.T.copy()
    a_t, f_t = varcoef_terms(case_t)
    Lt = OH.to_full(OH.apply_separable(u, a_t, f_t))
    assert np.any(np.abs(Lt - exact) > 10.0 * (bound + 1e-10))


def dense_L(case):
    alphas, factors = varcoef_terms(case)
    n = case.n
    M = np.zeros((n ** case.N, n ** case.N))
    for a, fs in zip(alphas, factors):
        K = np.ones((1, 1))
        for f in fs:
            K = np.kron(K, np.eye(n) if f is None else f)
        M += a * K
    return M


def test_varcoef_heun2_against_semidiscrete_flow():
    """N = 2: HEUN2 steps of the HT oracle (tolerance 1e-13, no rank cap) against the exact
    semi-discrete solution exp(T L_h) u0 (a library matrix exponential): the error is second
    order in dt (halving dt divides it by about 4)."""
    from scipy.linalg import expm
    case = varcoef_case(2, 40, zmax=5.0)
    alphas, factors = varcoef_terms(case)
    u0 = OH.from_cp(np.ones(1), case.ic_factors())
    dt = case.dt
    T = 12 * dt
    exact = (expm(T * dense_L(case)) @ OH.to_full(u0).reshape(-1)).reshape(case.n, case.n)
    errs = []
    for K in (12, 24):
        u = u0
        for _ in range(K):
            u, _ = OH.step_heun2(u, alphas, factors, T / K, 1e-13, 40)
        errs.append(float(np.abs(OH.to_full(u) - exact).max()))
    assert errs[1] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_varcoef_characteristic_solution_at_z_star():
    """N = 2 at the paper's evaluation point (grid point nearest z* = (h, h), h = 0.6988...):
    HEUN2 with tolerance 1e-10 to t = 0.5 against f0(exp(-tC) z), within 0.5% (the central
    difference's h^2 error at h = 0.1, about 0.2% here, dominates); the initial value matches
    exactly."""
    case = varcoef_case(2, 100, zmax=5.0)
    alphas, factors = varcoef_terms(case)
    u = OH.from_cp(np.ones(1), case.ic_factors())
    i = case.star_index()
    zp = np.array([case.z()[i]] * 2)
    assert abs(OH.to_full(u)[i, i] - varcoef_exact(0.0, case.C, zp)) < 1e-15
    steps = int(math.ceil(0.5 / case.dt))
    dt = 0.5 / steps
    for _ in range(steps):
        u, _ = OH.step_heun2(u, alphas, factors, dt, 1e-10, 40)
    f_num = OH.to_full(u)[i, i]
    f_ex = varcoef_exact(0.5, case.C, zp)
    assert abs(f_num - f_ex) / f_ex < 0.005, (f_num, f_ex)
