"""The 6-D advection steps at the bench's full size (n = 64), HT and CP routes, pinned by the fully
discrete Fourier closed form on sampled modes, without a 64^6 grid.

A single Fourier coefficient u^(q) = n^-d sum_x u(x) exp(-i q.x) of an HT tensor is a contraction
of its leaves with one separable vector per dimension, so it is evaluated on the format.  The
periodic central difference multiplies exp(i k x) by i sin(k h)/h, so K RK2 steps give
u^_K(q) = R(dt lam(q))^K u^_0(q), lam(q) = -i sum_j c_j sin(q_j h)/h, R(z) = 1 + z + z^2/2, and the
initial condition sum_m prod_i exp(sin(x_i + phi_mi)) has u^_0(q) = sum_m prod_i a^_mi(q_i) from
1-D DFTs.  Untruncated steps must reach it to rounding; truncated steps (the bench's tol 1e-8,
r_max 32) within n^-d/2 times the accumulated HSVD error bound (Parseval).
"""
import math

import numpy as np

from oracle import ht as OH
from oracle.problems import advection_A
from paper_1803_10270_gb300.inputs import advection_case


def fourier_coefficient(u, q, x):
    """u^(q) of an HT tensor: the leaves contracted with exp(-i q_i x)/n_i, then up the tree
    (eq. HTD: B_t[a, b, c] couples basis a of the first child with b of the second)."""
    tr = u.tree
    val = {}
    for t in sorted(range(tr.n_nodes), key=lambda t: -tr.depth[t]):
        X = u.node[t]
        if tr.is_leaf(t):
            i = tr.lo[t]
            val[t] = (np.exp(-1j * q[i] * x) / len(x)) @ X
        else:
            a, b = tr.children[t]
            if t == 0:
                return complex(val[a] @ X @ val[b])
            val[t] = np.einsum("a,b,abc->c", val[a], val[b], X)
    raise RuntimeError("unreachable")


def closed_form(case, q, steps):
    n, h, x = case.n, case.h, case.x()
    ic = case.ic_factors()
    u0 = 0.0
    for m in range(case.n_terms):
        term = 1.0 + 0.0j
        for i in range(case.d):
            term *= np.fft.fft(ic[i][:, m])[q[i] % n] / n
        u0 += term
    lam = -1j * sum(case.c[j] * math.sin(q[j] * h) / h for j in range(case.d))
    z = case.dt * lam
    return (1.0 + z + 0.5 * z * z) ** steps * u0


def sample_modes(d, count, seed):
    rng = np.random.default_rng(seed)
    qs = [np.zeros(d, dtype=int)] + [np.eye(d, dtype=int)[i] * s for i in range(d) for s in (1, -2)]
    qs += [rng.integers(-4, 5, d) for _ in range(count)]
    return qs


def test_untruncated_steps_match_fourier_modes_at_n64():
    """Three exact RK2-polynomial applies (ranks 2 -> 6 -> 18 -> 54) of the bench workload."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    u = OH.from_cp(np.ones(case.n_terms), case.ic_factors())
    for _ in range(3):
        u = OH.apply_kron_sum_rk2(u, A)
    assert max(u.ranks()[1:]) == 54
    x = case.x()
    scale = abs(closed_form(case, np.zeros(6, dtype=int), 0))
    for q in sample_modes(6, 24, seed=5):
        got = fourier_coefficient(u, q, x)
        ref = closed_form(case, q, 3)
        assert abs(got - ref) <= 1e-13 * scale, q


def test_truncated_bench_steps_within_the_hsvd_bound():
    """Five steps of the bench's HT route (tol 1e-8, r_max 32): every sampled coefficient lies
    within n^-d/2 sum_k g^(K-1-k) e_k of the exact one, e_k = sqrt(sum_t discarded_t^2) the HSVD
    bound of step k's truncation and g = max_q |R(dt lam(q))| the growth of later steps."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    u = OH.from_cp(np.ones(case.n_terms), case.ic_factors())
    theta = case.dt * sum(abs(c) for c in case.c) / case.h
    g = math.sqrt(1.0 + theta ** 4 / 4.0)           # |R(i s)| = sqrt(1 + s^4/4), |s| <= theta
    K, bound = 5, 0.0
    for _ in range(K):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 32)
        e_k = math.sqrt(sum(v * v for v in rep.discarded.values()))
        # the rank rule: each of the 2d - 2 non-root nodes (the root's children counted twice)
        # discards at most (tol |v|)^2 / (2d - 3) when r_max does not bind
        assert max(rep.ranks) < 32
        assert e_k <= 1e-8 * rep.norm * math.sqrt(10.0 / 9.0) * (1 + 1e-12)
        bound = bound * g + e_k
    assert 0.0 < bound
    x = case.x()
    tol = bound / 64.0 ** 3 * 1.01 + 1e-14 * abs(closed_form(case, np.zeros(6, dtype=int), 0))
    worst = 0.0
    for q in sample_modes(6, 24, seed=6):
        err = abs(fourier_coefficient(u, q, x) - closed_form(case, q, K))
        worst = max(worst, err)
        assert err <= tol, q
    assert worst > 0.0


def cp_fourier_coefficient(x, q):
    """x^(q) of a CP tensor: sum_l w_l prod_i (DFT of factor column l of dimension i at q_i) / n."""
    term = np.asarray(x.weights, dtype=np.complex128).copy()
    for i, F in enumerate(x.factors):
        n = F.shape[0]
        term *= np.fft.fft(F, axis=0)[q[i] % n] / n
    return complex(term.sum())


def test_cp_route_at_n64_against_fourier_modes():
    """The CP route at the bench size: the exact apply y = p(dt L) x (rank 2 (1 + 2d + d(d-1)/2)
    = 56) has y^(q) = R(dt lam(q)) x^(q) to rounding, and the fitted rank-24 x after 5 Gauss-Seidel
    sweeps lies within n^-d/2 (|y - x| + the Gram-difference rounding floor) of it on every
    sampled mode, |y - x| the oracle's reported residual."""
    from oracle import cp as OC
    from paper_1803_10270_gb300.inputs import cp_padding
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    x = OC.CP(np.ones(case.n_terms), case.ic_factors())
    y = OC.apply_kron_sum_rk2(x, A)
    assert y.rank == 56
    h = case.h
    scale = abs(cp_fourier_coefficient(x, np.zeros(6, dtype=int)))
    qs = sample_modes(6, 24, seed=7)
    for q in qs:
        lam = -1j * sum(case.c[j] * math.sin(q[j] * h) / h for j in range(6))
        z = case.dt * lam
        ref = (1.0 + z + 0.5 * z * z) * cp_fourier_coefficient(x, q)
        assert abs(cp_fourier_coefficient(y, q) - ref) <= 1e-13 * scale, q
    pad = cp_padding([64] * 6, 22, seed=0x5EED + 1, scale=1e-3)
    x1, _ = OC.step_rk2(x, A, 24, pad, 5)
    res = OC.residual(y, x1)
    ny = OC.residual(y, OC.CP(np.zeros(1), [np.zeros((64, 1))] * 6))
    floor = 4.0 * math.sqrt(2.2e-16) * 2.0 * ny                 # |.|^2 formed from Gram sums
    for q in qs:
        err = abs(cp_fourier_coefficient(x1, q) - cp_fourier_coefficient(y, q))
        assert err <= (res + floor) / 64.0 ** 3 * 1.01, q


def test_twelve_dim_n128_steps_match_fourier_modes():
    """The 12-D workload (n = 128, depth-4 tree, rank-3 initial condition): two untruncated
    RK2-polynomial applies (ranks 3 -> 9 -> 27) reach the closed form to rounding, and five of the
    bench's truncated steps (tol 1e-8, r_max 64) stay within the HSVD bound, on sampled modes."""
    case = advection_case(12, 128, n_terms=3, seed_offset=4)
    A = advection_A(case)
    x = case.x()
    u0 = OH.from_cp(np.ones(case.n_terms), case.ic_factors())
    scale = abs(closed_form(case, np.zeros(12, dtype=int), 0))
    u = u0
    for _ in range(2):
        u = OH.apply_kron_sum_rk2(u, A)
    assert max(u.ranks()[1:]) == 27
    qs = sample_modes(12, 24, seed=8)
    for q in qs:
        assert abs(fourier_coefficient(u, q, x) - closed_form(case, q, 2)) <= 1e-13 * scale, q
    theta = case.dt * sum(abs(c) for c in case.c) / case.h
    g = math.sqrt(1.0 + theta ** 4 / 4.0)
    u, bound = u0, 0.0
    for _ in range(5):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 64)
        assert max(rep.ranks) < 64
        bound = bound * g + math.sqrt(sum(v * v for v in rep.discarded.values()))
    tol = bound / 128.0 ** 6 * 1.01 + 1e-14 * scale
    for q in qs:
        assert abs(fourier_coefficient(u, q, x) - closed_form(case, q, 5)) <= tol, q


def test_tensor_train_route_at_n64_matches_fourier_modes():
    """The same steps on the linear (tensor-train) dimension tree: three untruncated applies to
    rounding and five truncated bench steps within the HSVD bound, on sampled modes."""
    from oracle.tree import build_tree
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    x = case.x()
    u0 = OH.from_cp(np.ones(case.n_terms), case.ic_factors(), build_tree(6, "linear"))
    scale = abs(closed_form(case, np.zeros(6, dtype=int), 0))
    qs = sample_modes(6, 24, seed=9)
    u = u0
    for _ in range(3):
        u = OH.apply_kron_sum_rk2(u, A)
    for q in qs:
        assert abs(fourier_coefficient(u, q, x) - closed_form(case, q, 3)) <= 1e-13 * scale, q
    theta = case.dt * sum(abs(c) for c in case.c) / case.h
    g = math.sqrt(1.0 + theta ** 4 / 4.0)
    u, bound = u0, 0.0
    for _ in range(5):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 32)
        assert max(rep.ranks) < 32
        bound = bound * g + math.sqrt(sum(v * v for v in rep.discarded.values()))
    tol = bound / 64.0 ** 3 * 1.01 + 1e-14 * scale
    for q in qs:
        assert abs(fourier_coefficient(u, q, x) - closed_form(case, q, 5)) <= tol, q


def test_ab2_route_at_n64_matches_fourier_modes():
    """The AB2 scheme (eq. AB2_) of the bench's ab2 line at n = 64: started by one RK2 step, each
    mode follows w_{k+1} = (1 + 3z/2) w_k - (z/2) w_{k-1}, z = dt lam(q).  Three AB2 steps with
    the sums formed exactly and no truncation (node ranks 2 -> 6 -> 16 -> 44 -> 120) reach it to
    rounding on sampled modes."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    x = case.x()
    h = case.h
    u_prev = OH.from_cp(np.ones(case.n_terms), case.ic_factors())
    u = OH.apply_kron_sum_rk2(u_prev, A)
    for _ in range(3):
        u, u_prev = OH.add(1.0, OH.apply_kron_sum_poly(u, A, (1.0, 1.5)), 1.0,
                           OH.apply_kron_sum_poly(u_prev, A, (0.0, -0.5))), u
    assert max(u.ranks()[1:]) == 120
    scale = abs(closed_form(case, np.zeros(6, dtype=int), 0))
    for q in sample_modes(6, 24, seed=10):
        z = case.dt * (-1j) * sum(case.c[j] * math.sin(q[j] * h) / h for j in range(6))
        w0 = closed_form(case, q, 0)
        w1 = (1.0 + z + 0.5 * z * z) * w0
        for _ in range(3):
            w1, w0 = (1.0 + 1.5 * z) * w1 - 0.5 * z * w0, w1
        assert abs(fourier_coefficient(u, q, x) - w1) <= 1e-13 * scale, q
