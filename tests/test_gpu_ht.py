"""GPU parity of the HT path (ht_apply, ht_truncate, ht_step, ht_from_cp, ht_mass,
ht_inner) against the FP64 CPU oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A, kinetic_terms
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case, kinetic_case
from tests.helpers import min_gap, random_ht, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1803_10270_gb300 import build as B
    B.build()
    from paper_1803_10270_gb300 import htgpu
    htgpu.load()
    return htgpu


def to_gpu(G, u: OH.HT, cap):
    t = G.HTTensor(u.tree.d, u.n, cap)
    t.upload(u.node)
    return t


def from_gpu(t, tree) -> OH.HT:
    return OH.HT(tree, list(t.n), t.download())


def sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("d,n,r", [(2, 7, 3), (4, 6, 3), (5, [5, 7, 4, 9, 6], 2), (6, 8, 4)])
def test_apply_rk2poly_exact(G, d, n, r):
    u = random_ht(d, n, r, seed=100 + d)
    ns = u.n
    case = advection_case(d, ns[0], seed=7 + d)
    hs = [2 * math.pi / m for m in ns]
    A = [case.dt * (-case.c[i]) * OH.central_diff_matrix(ns[i], hs[i]) for i in range(d)]
    ref = OH.apply_kron_sum_rk2(u, A)
    ctx = G.Context(d, ns, cap=r, max_terms=d)
    gu = to_gpu(G, u, r)
    gv = G.HTTensor(d, ns, 3 * r)
    G.ht_apply(ctx, gu, G.advection_op(case.c, hs), case.dt, G.HT_APPLY_RK2POLY, gv)
    sync()
    got = gv.download()
    assert gv.ranks()[1:2 * d - 1] == [3 * r] * (2 * d - 2)
    for t in range(u.tree.n_nodes):
        np.testing.assert_allclose(got[t], ref.node[t], rtol=0, atol=1e-13 * np.abs(ref.node[t]).max())


def test_apply_general_separable_kinetic(G):
    kc = kinetic_case(5)
    alphas, factors = kinetic_terms(kc)
    u = random_ht(6, 5, 2, seed=3)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [5] * 6, cap=2, max_terms=5)
    gu = to_gpu(G, u, 2)
    for mode in (G.HT_APPLY_L, G.HT_APPLY_EULER):
        if mode == G.HT_APPLY_L:
            ref = OH.apply_separable(u, alphas, factors)
            cap = 5 * 2
        else:
            dt = kc.dt
            ref = OH.apply_separable(u, [1.0] + [dt * a for a in alphas], [[None] * 6] + factors)
            cap = 6 * 2
        gv = G.HTTensor(6, [5] * 6, cap)
        G.ht_apply(ctx, gu, kop.op, kc.dt, mode, gv)
        sync()
        got = gv.download()
        for t in range(u.tree.n_nodes):
            np.testing.assert_allclose(got[t], ref.node[t], rtol=0, atol=1e-13 * max(1.0, np.abs(ref.node[t]).max()))


@pytest.mark.parametrize("d,n,r,tol,rmax", [
    (2, 9, 6, 1e-3, 4),
    (3, 6, 5, 1e-4, 8),
    (4, 5, 6, 1e-2, 3),
    (5, [4, 6, 5, 7, 3], 5, 1e-3, 6),
    (6, 7, 5, 1e-2, 4),
    (6, 6, 4, 0.0, 16),
    (7, 4, 3, 1e-2, 3),
])
def test_truncate_parity(G, d, n, r, tol, rmax):
    u = random_ht(d, n, r, seed=200 + d, scale_decay=0.5)
    ref, rep = OH.truncate(u, tol, rmax)
    assert min_gap(rep, rep.ranks) > 1 + 1e-6
    ctx = G.Context(d, u.n, cap=max(r, rmax), max_terms=1)
    gu = to_gpu(G, u, max(r, rmax))
    out = G.HTTensor(d, u.n, max(r, rmax))
    import torch
    sig = torch.zeros(31 * 64, dtype=torch.float64, device="cuda")
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.ht_truncate(ctx, gu, tol, rmax, out, sigma=sig, sig_stride=64, norm=nrm)
    sync()
    ctx.check()
    assert out.ranks() == rep.ranks
    got = from_gpu(out, u.tree)
    assert rel_err(got, ref) < TOL64
    assert abs(float(nrm[0]) - rep.norm) < 1e-12 * rep.norm
    s = sig.cpu().numpy().reshape(31, 64)
    for t in range(1, u.tree.n_nodes):
        m = min(len(rep.sigma[t]), 64)
        ref_s = rep.sigma[t][:m]
        assert np.abs(s[t, :len(ref_s)] - ref_s).max() <= 1e-12 * rep.norm


def test_truncate_in_place_and_rank1(G):
    rng = np.random.default_rng(5)
    fac = [rng.standard_normal((6, 1)) for _ in range(5)]
    u = OH.from_cp(np.array([2.0]), fac)
    pad = OH.add(1.0, u, 0.0, random_ht(5, 6, 2, seed=9))   # redundant rank-3 representation
    ctx = G.Context(5, [6] * 5, cap=4, max_terms=1)
    g = to_gpu(G, pad, 4)
    G.ht_truncate(ctx, g, 1e-12, 4, g)   # out aliases the input
    sync()
    assert g.ranks()[1:] == [1] * 8
    assert rel_err(from_gpu(g, pad.tree), u) < TOL64


def test_step_rk2poly_adv6d_n16_ten_steps(G):
    """6-D advection, n=16, HT r_max=8, tol 1e-8, RK2, dt=0.2h, 10 steps, FP64."""
    case = advection_case(6, 16, seed_offset=0)
    A = advection_A(case)
    u = OH.from_cp(np.ones(2), case.ic_factors())
    ctx = G.Context(6, [16] * 6, cap=8, max_terms=6)
    g = to_gpu(G, u, 8)
    op = G.advection_op(case.c, case.h)
    for step in range(10):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 8)
        G.ht_step(ctx, g, op, case.dt, 1e-8, 8)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        e = rel_err(from_gpu(g, u.tree), u)
        assert e < TOL64, f"step {step}: {e:.3e}"


def test_step_rk2poly_adv6d_n64_shape_three_steps(G):
    """6-D advection at n=64, r_max=32 (the ranks settle near 6), 3 steps vs oracle."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    u = OH.from_cp(np.ones(2), case.ic_factors())
    ctx = G.Context(6, [64] * 6, cap=32, max_terms=6)
    g = to_gpu(G, u, 32)
    op = G.advection_op(case.c, case.h)
    for step in range(3):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 32)
        G.ht_step(ctx, g, op, case.dt, 1e-8, 32)
        sync()
        assert g.ranks() == rep.ranks
        assert rel_err(from_gpu(g, u.tree), u) < TOL64


def test_step_heun2_kinetic_small(G):
    kc = kinetic_case(6)
    alphas, factors = kinetic_terms(kc)
    u = random_ht(6, 6, 2, seed=31, scale_decay=0.3)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [6] * 6, cap=6, max_terms=5)
    g = to_gpu(G, u, 6)
    for step in range(2):
        u, reps = OH.step_heun2(u, alphas, factors, kc.dt, 1e-6, 6)
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 6, scheme=G.HT_SCHEME_HEUN2)
        sync()
        assert g.ranks() == reps[1].ranks
        assert rel_err(from_gpu(g, u.tree), u) < TOL64


def test_from_cp_mass_inner(G):
    import torch
    case = advection_case(5, 6, n_terms=3, seed=4)
    fac = case.ic_factors()
    w = np.array([1.0, -0.5, 0.25])
    ref = OH.from_cp(w, fac)
    ctx = G.Context(5, [6] * 5, cap=3, max_terms=1)
    x = G.CPTensor(5, [6] * 5, 3)
    x.upload(w, fac)
    h = G.HTTensor(5, [6] * 5, 3)
    G.ht_from_cp(ctx, x, h)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    G.ht_mass(ctx, h, out[0:1])
    v = random_ht(5, 6, 2, seed=1)
    hv = to_gpu(G, v, 3)
    G.ht_inner(ctx, h, hv, out[1:2])
    sync()
    assert rel_err(from_gpu(h, ref.tree), ref) < 1e-14
    assert abs(float(out[0]) - OH.mass(ref)) <= 1e-12 * abs(OH.mass(ref))
    assert abs(float(out[1]) - OH.inner(ref, v)) <= 1e-11 * OH.norm(ref) * OH.norm(v)


def test_capacity_and_argument_errors(G):
    ctx = G.Context(4, [5] * 4, cap=3, max_terms=1)
    u = G.HTTensor(4, [5] * 4, 3)
    small = G.HTTensor(4, [5] * 4, 2)
    with pytest.raises(G.HTError) as e:
        G.ht_truncate(ctx, u, 1e-3, 3, small)     # rmax > out capacity
    assert e.value.status == G.HT_ERR_CAPACITY
    case = advection_case(4, 5, seed=1)
    with pytest.raises(G.HTError) as e:
        G.ht_apply(ctx, u, G.advection_op(case.c, case.h), 0.1, G.HT_APPLY_RK2POLY, small)
    assert e.value.status == G.HT_ERR_CAPACITY
    other = G.HTTensor(4, [6] * 4, 3)
    with pytest.raises(G.HTError) as e:
        G.ht_step(ctx, other, G.advection_op(case.c, case.h), 0.1, 1e-3, 3)
    assert e.value.status == G.HT_ERR_ARG
