"""Pins for the HT oracle (apply, add, orthogonalise, HSVD truncation, scalars)."""
import itertools
import math

import numpy as np
import pytest

from oracle import fullgrid as FG
from oracle import ht as H
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case, normal_arrays
from oracle.problems import advection_A
from tests.closed_forms import apply_node_projector, fourier_ab2, fourier_rk2, matricize


def random_ht(d, n, rank, seed, leaf_rank=None):
    tree = build_tree(d)
    ns = [n] * d if np.isscalar(n) else list(n)
    rk = {}
    for t in range(tree.n_nodes):
        rk[t] = 1 if t == 0 else (leaf_rank if (leaf_rank and tree.is_leaf(t)) else rank)
    shapes = []
    for t in range(tree.n_nodes):
        if tree.is_leaf(t):
            shapes.append((ns[tree.lo[t]], rk[t]))
        else:
            a, b = tree.children[t]
            shapes.append((rk[a], rk[b]) if t == 0 else (rk[a], rk[b], rk[t]))
    arrs = normal_arrays(shapes, seed)
    u = H.HT(tree, ns)
    for t in range(tree.n_nodes):
        u.node[t] = arrs[t]
    return u


def adv_ops(case, d=None):
    d = d or case.d
    return [case.dt * (-case.c[i]) * H.central_diff_matrix(case.n, case.h) for i in range(d)]


def test_from_cp_matches_bruteforce():
    case = advection_case(4, 5, n_terms=3, seed=11)
    fac = case.ic_factors()
    w = np.array([1.0, -0.5, 2.0])
    u = H.from_cp(w, fac)
    assert np.abs(H.to_full(u) - FG.cp_to_full(w, fac)).max() < 1e-12 * np.abs(FG.cp_to_full(w, fac)).max()


@pytest.mark.parametrize("d,n", [(2, 7), (3, 6), (4, 5), (5, 4)])
def test_apply_rk2_matches_fourier_closed_form(d, n):
    case = advection_case(d, n, seed=40 + d)
    u = random_ht(d, n, 3, seed=d)
    v = H.apply_kron_sum_rk2(u, adv_ops(case))
    ref = fourier_rk2(H.to_full(u), case.c, case.h, case.dt, 1)
    assert v.ranks()[1:] == [9] * (2 * d - 2)
    assert np.abs(H.to_full(v) - ref).max() <= 1e-13 * np.abs(ref).max()
    # 1^T D = 0 => mass is conserved exactly by the apply
    assert abs(H.mass(v) - H.mass(u)) <= 1e-12 * np.abs(H.to_full(u)).sum()


def test_apply_separable_matches_dense_kronecker():
    d, n = 3, 4
    rng = np.random.default_rng(9)
    u = random_ht(d, n, 2, seed=3)
    alphas = [0.7, -1.3, 0.25]
    fac = [[rng.standard_normal((n, n)) if rng.random() < 0.7 else None for _ in range(d)] for _ in alphas]
    v = H.apply_separable(u, alphas, fac)
    # dense operator on vec(u) with first index fastest: kron(A_{d-1}, ..., A_0)
    Op = np.zeros((n ** d, n ** d))
    for a, f in zip(alphas, fac):
        K = np.ones((1, 1))
        for i in range(d):
            Ai = np.eye(n) if f[i] is None else f[i]
            K = np.kron(Ai, K)
        Op += a * K
    ref = (Op @ H.to_full(u).reshape(-1, order="F")).reshape([n] * d, order="F")
    assert np.abs(H.to_full(v) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_add_and_inner_and_norm():
    u = random_ht(4, 5, 2, seed=1)
    w = random_ht(4, 5, 3, seed=2)
    s = H.add(0.3, u, -1.7, w)
    fu, fw = H.to_full(u), H.to_full(w)
    assert np.abs(H.to_full(s) - (0.3 * fu - 1.7 * fw)).max() < 1e-12 * np.abs(fw).max()
    assert abs(H.inner(u, w) - np.sum(fu * fw)) < 1e-10 * np.linalg.norm(fu) * np.linalg.norm(fw)
    assert abs(H.norm(u) - np.linalg.norm(fu)) < 1e-12 * np.linalg.norm(fu)
    assert abs(H.mass(u) - fu.sum()) < 1e-10 * np.abs(fu).sum()


def test_orthogonalize_preserves_tensor_and_orthonormal_bases():
    u = random_ht(5, 4, 3, seed=8)
    o = H.orthogonalize(u)
    assert np.abs(H.to_full(o) - H.to_full(u)).max() < 1e-12 * np.abs(H.to_full(u)).max()
    for t in range(1, o.tree.n_nodes):
        Ut = H.node_basis(o, t)
        assert np.abs(Ut.T @ Ut - np.eye(Ut.shape[1])).max() < 1e-12


def test_truncate_d2_is_eckart_young():
    rng = np.random.default_rng(21)
    M = rng.standard_normal((12, 9)) @ np.diag(np.logspace(0, -6, 9)) @ rng.standard_normal((9, 10))
    tree = build_tree(2)
    u = H.HT(tree, [12, 10])
    u.node[1] = M.copy()
    u.node[2] = np.eye(10)
    u.node[0] = np.eye(10)
    for k in (1, 3, 5):
        w, rep = H.truncate(u, 0.0, k)
        Uf, s, Vt = np.linalg.svd(M)
        best = (Uf[:, :k] * s[:k]) @ Vt[:k]
        assert rep.ranks[1] == k and rep.ranks[2] == k
        assert np.abs(H.to_full(w) - best).max() < 1e-12 * s[0]
        assert abs(np.linalg.norm(H.to_full(w) - M) - math.sqrt(np.sum(s[k:] ** 2))) < 1e-12 * s[0]


@pytest.mark.parametrize("d,r", [(4, 2), (6, 3), (5, 1)])
def test_truncate_recovers_exact_separable(d, r):
    rng = np.random.default_rng(d * 10 + r)
    fac = [rng.standard_normal((5, r)) for _ in range(d)]
    w = rng.uniform(0.5, 2.0, r)
    u = H.from_cp(w, fac)
    # pad ranks with an exactly cancelling copy to make the representation redundant
    u2 = H.add(1.0, u, 0.0, H.from_cp(w, [rng.standard_normal((5, r)) for _ in range(d)]))
    t, rep = H.truncate(u2, 1e-12, 10)
    full = FG.cp_to_full(w, fac)
    assert max(rep.ranks[1:]) <= r
    if r == 1:
        assert rep.ranks[1:] == [1] * (2 * d - 2)
    assert np.abs(H.to_full(t) - full).max() <= 1e-12 * np.abs(full).max()


def _bruteforce_hsvd(full, tree, ranks):
    """T(u) = prod_{deepest level} pi_t ... prod_{level 1} pi_t u with pi_t from full SVDs."""
    out = full.copy()
    proj = {}
    for t in range(1, tree.n_nodes):
        Mt = matricize(full, tree.dims(t))
        Uf, s, _ = np.linalg.svd(Mt, full_matrices=False)
        proj[t] = (Uf[:, :ranks[t]] @ Uf[:, :ranks[t]].T, s)
    for level in tree.levels()[1:]:
        for t in level:
            out = apply_node_projector(out, tree.dims(t), proj[t][0])
    return out, proj


def test_truncate_equals_bruteforce_projectors_and_singular_values():
    u = random_ht(4, 4, 3, seed=77)
    full = H.to_full(u)
    for rmax in (1, 2):
        w, rep = H.truncate(u, 0.0, rmax)
        ref, proj = _bruteforce_hsvd(full, u.tree, rep.ranks)
        for t in range(1, u.tree.n_nodes):
            s = proj[t][1]
            m = min(len(s), len(rep.sigma[t]))
            assert np.abs(rep.sigma[t][:m] - s[:m]).max() < 1e-12 * s[0]
        assert np.abs(H.to_full(w) - ref).max() < 1e-12 * np.abs(full).max()


@pytest.mark.parametrize("tol,rmax", [(1e-2, 50), (1e-4, 50), (1e-1, 3)])
def test_truncate_error_bounds_and_idempotence(tol, rmax):
    d = 5
    case = advection_case(d, 6, seed=5)
    u = H.apply_kron_sum_rk2(random_ht(d, 6, 3, seed=4), adv_ops(case))
    w, rep = H.truncate(u, tol, rmax)
    err = np.linalg.norm(H.to_full(w) - H.to_full(u))
    c1, c2 = u.tree.children[0]
    e = [rep.discarded[t] for t in range(1, u.tree.n_nodes) if t != c2]
    assert max(e) <= err * (1 + 1e-10) + 1e-12
    assert err <= math.sqrt(sum(x * x for x in e)) * (1 + 1e-10) + 1e-12
    if rmax == 50:
        assert err <= tol * rep.norm * (1 + 1e-10)
    w2, rep2 = H.truncate(w, 0.0, 100)   # keep every nonzero direction
    assert np.abs(H.to_full(w2) - H.to_full(w)).max() < 1e-11 * np.abs(H.to_full(w)).max()
    w3, rep3 = H.truncate(w, tol, rmax)
    assert rep3.ranks == rep.ranks
    assert np.abs(H.to_full(w3) - H.to_full(w)).max() < 1e-10 * np.abs(H.to_full(w)).max()


def test_rank_rule():
    s = np.array([10.0, 1.0, 0.1, 0.01])
    assert H.choose_rank(s, 0.0, 9) == 4
    assert H.choose_rank(s, 0.011, 9) == 3
    assert H.choose_rank(s, math.sqrt(0.1 ** 2 + 0.01 ** 2) + 1e-12, 9) == 2
    assert H.choose_rank(s, 1e3, 9) == 1
    assert H.choose_rank(s, 0.0, 2) == 2


def _orthogonal_diagonal(d, n, s, seed):
    """u = sum_k s_k prod_i Q_i[:, k] with orthonormal Q_i: every node matricisation of u has the
    singular values s (a diagonal tensor in orthonormal bases)."""
    rng = np.random.default_rng(seed)
    Q = [np.linalg.qr(rng.standard_normal((n, len(s))))[0] for _ in range(d)]
    return H.from_cp(np.asarray(s, dtype=float), Q)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_rank_rule_splits_the_budget_over_2d_minus_3_edges(d):
    """The rank rule's budget (tol |u|)^2 / (2d - 3): every node of an orthogonally diagonal
    tensor has the spectrum s = (1, 0.1, 0.01, 0.001), and tol is set inside the window where
    the tail after two values fits the budget with 2d - 3 edges but not with 2d - 2, so every
    node keeps exactly two (d = 2 is the matrix case, a single edge)."""
    s = np.array([1.0, 0.1, 0.01, 0.001])
    u = _orthogonal_diagonal(d, 6, s, seed=70 + d)
    e = 2 * d - 3
    tail2 = float(np.sum(s[2:] ** 2)) / float(np.sum(s ** 2))
    tol = math.sqrt(tail2 * (e + 0.5))          # tail2 <= tol^2 / e, tail2 > tol^2 / (e + 1)
    t, rep = H.truncate(u, tol, 10)
    assert rep.ranks[1:] == [2] * (2 * d - 2)
    for t_ in range(1, 2 * d - 1):
        assert np.allclose(rep.sigma[t_][:4], s, rtol=1e-12)


def test_root_children_share_one_rank():
    """The two children of the root share one spectrum, and the rank is chosen once for both:
    with a 3-point leaf on one side and a rank-5 node on the other, tolerance 0 keeps three
    directions on both sides (the other side's factor also carries two singular values at the
    rounding level, which a separate choice at tolerance 0 would keep) and reproduces u."""
    tree = build_tree(3)
    c1, c2 = tree.children[0]
    ns = [3, 6, 6]
    ranks = {0: 1, c1: 3, c2: 5}
    for t in range(tree.n_nodes):
        if t not in ranks:
            ranks[t] = 3
    shapes = []
    for t in range(tree.n_nodes):
        if tree.is_leaf(t):
            shapes.append((ns[tree.lo[t]], ranks[t]))
        else:
            a, b = tree.children[t]
            shapes.append((ranks[a], ranks[b]) if t == 0 else (ranks[a], ranks[b], ranks[t]))
    arrs = normal_arrays(shapes, 71)
    u = H.HT(tree, ns)
    for t in range(tree.n_nodes):
        u.node[t] = arrs[t]
    assert u.ranks()[c1] == 3 and u.ranks()[c2] == 5
    t, rep = H.truncate(u, 0.0, 10)
    assert rep.ranks[c1] == rep.ranks[c2] == 3
    full = H.to_full(u)
    assert np.abs(H.to_full(t) - full).max() <= 1e-12 * np.abs(full).max()


def test_kinetic_operator_dense_and_conservation():
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case
    kc = kinetic_case(4, nu=1.0)
    alphas, factors = kinetic_terms(kc)
    u = random_ht(6, 4, 2, seed=12)
    v = H.apply_separable(u, alphas, factors)
    fu = H.to_full(u)
    # direct evaluation of -v.grad_x f - nu f + nu M rho on the grid
    D = H.central_diff_matrix(4, kc.hx)
    vg = kc.vgrid()
    ref = -kc.nu * fu
    for i in range(3):
        dfi = np.moveaxis(np.tensordot(D, fu, axes=(1, i)), 0, i)
        shape = [1] * 6
        shape[3 + i] = 4
        ref -= vg.reshape(shape) * dfi
    rho = np.einsum("abcijk,i,j,k->abc", fu, kc.weights(), kc.weights(), kc.weights())
    m = kc.maxwellian()
    ref += kc.nu * np.einsum("abc,i,j,k->abcijk", rho, m, m, m)
    assert np.abs(H.to_full(v) - ref).max() < 1e-12 * np.abs(ref).max()
    # weighted mass of L f vanishes (transport: 1^T D = 0; collision: sum h_v m = 1)
    assert abs(H.mass(v)) < 1e-11 * np.abs(fu).sum()


def test_heun2_matches_full_grid_rk2_without_truncation():
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case
    kc = kinetic_case(4, nu=1.0)
    alphas, factors = kinetic_terms(kc)
    u = random_ht(6, 4, 2, seed=13)
    w, _ = H.step_heun2(u, alphas, factors, kc.dt, 0.0, 10 ** 6)
    fu = H.to_full(u)
    Lf = lambda f: H.to_full(H.apply_separable(H.HT(u.tree, u.n, {t: a for t, a in _ht_of(f, u).node.items()}), alphas, factors))
    # full-grid Heun with dense operator
    Op = np.zeros((4 ** 6, 4 ** 6))
    for a, f in zip(alphas, factors):
        K = np.ones((1, 1))
        for i in range(6):
            K = np.kron(np.eye(4) if f[i] is None else f[i], K)
        Op += a * K
    x = fu.reshape(-1, order="F")
    xs = x + kc.dt * Op @ x
    xn = 0.5 * x + 0.5 * (xs + kc.dt * Op @ xs)
    assert np.abs(H.to_full(w).reshape(-1, order="F") - xn).max() < 1e-11 * np.abs(xn).max()


def _ht_of(f, like):
    return like


def test_apply_poly_matches_full_grid_polynomial():
    """apply_kron_sum_poly == q(dt L) on the full grid for degree 0, 1, 2 coefficient sets."""
    d, n = 4, 6
    case = advection_case(d, n, seed=51)
    A = advection_A(case)
    u = random_ht(d, n, 3, seed=52)
    full = H.to_full(u)
    Lu = FG.apply_L(full, case.c, case.h)
    LLu = FG.apply_L(Lu, case.c, case.h)
    for q in [(0.7,), (1.0, 1.5), (0.0, -0.5), (1.0, 1.0, 0.5), (0.3, -2.0, 0.25)]:
        want = q[0] * full
        if len(q) > 1:
            want = want + q[1] * case.dt * Lu
        if len(q) > 2:
            want = want + q[2] * case.dt ** 2 * LLu
        got = H.to_full(H.apply_kron_sum_poly(u, A, q))
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def test_ab2_full_grid_matches_fourier_recurrence():
    """The full-grid AB2 stepper reproduces the per-mode two-step recurrence (eq. AB2_)."""
    d, n = 3, 8
    case = advection_case(d, n, seed=53)
    u0 = H.to_full(H.from_cp(np.ones(2), case.ic_factors()))
    u1 = FG.rk2_step(u0, case.c, case.h, case.dt)
    a, b = u0, u1
    for _ in range(5):
        a, b = b, FG.ab2_step(b, a, case.c, case.h, case.dt)
    want = fourier_ab2(u0, u1, case.c, case.h, case.dt, 5)
    assert np.abs(b - want).max() <= 1e-12 * np.abs(want).max()


def test_ab2_ht_step_untruncated_matches_full_grid():
    """step_ab2 with tol 0 and a rank cap above the exact rank equals the full-grid AB2 step;
    with a tolerance it stays within the HSVD bound of the exact sum."""
    d, n = 4, 6
    case = advection_case(d, n, seed=54)
    A = advection_A(case)
    u0 = H.from_cp(np.ones(2), case.ic_factors())
    u1, _ = H.step_rk2_poly(u0, A, 0.0, 64)
    u2, rep = H.step_ab2(u1, u0, A, 0.0, 64)
    want = FG.ab2_step(H.to_full(u1), H.to_full(u0), case.c, case.h, case.dt)
    got = H.to_full(u2)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    tol = 1e-4
    u2t, rep = H.step_ab2(u1, u0, A, tol, 64)
    err = np.linalg.norm(H.to_full(u2t) - want)
    assert err <= tol * np.linalg.norm(want) * (1 + 1e-9)
