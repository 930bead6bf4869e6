"""GPU parity on the linear dimension tree, the tensor-train format as a special case of HT
(Section 2.2): truncation, RK2 advection steps (the shape of the 6-D n = 16 configuration),
HEUN2 kinetic steps, and a 12-D tree eleven levels deep, against the FP64 oracle."""
import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A, kinetic_terms
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case, kinetic_case
from tests.helpers import random_ht, rel_err

pytestmark = pytest.mark.gpu
TOL64 = 1e-10
LINEAR = 1


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


def sync():
    import torch
    torch.cuda.synchronize()


def to_gpu(G, u, cap):
    t = G.HTTensor(u.tree.d, u.n, cap, tree=LINEAR)
    t.upload(u.node)
    return t


def from_gpu(t, tree):
    return OH.HT(tree, list(t.n), t.download())


def test_linear_tree_numbering_matches_oracle(G):
    for d in (2, 5, 12, 16):
        ti = G.tree_info(d, LINEAR)
        to = build_tree(d, "linear")
        assert ti.lo == to.lo and ti.hi == to.hi and ti.depth == to.depth


@pytest.mark.parametrize("rel_tol,rmax", [(1e-6, 8), (1e-10, 8), (0.0, 4)])
def test_tt_truncate(G, rel_tol, rmax):
    d, n, r = 6, 10, 8
    u = random_ht(d, n, r, seed=31, scale_decay=0.6, kind="linear")
    ref, rep = OH.truncate(u, rel_tol, rmax)
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1, tree=LINEAR)
    g = to_gpu(G, u, r)
    out = G.HTTensor(d, [n] * d, r, tree=LINEAR)
    G.ht_truncate(ctx, g, rel_tol, rmax, out)
    sync()
    ctx.check()
    assert out.ranks() == rep.ranks
    assert rel_err(from_gpu(out, u.tree), ref) < TOL64


def test_tt_rk2_advection_steps(G):
    d, n, cap = 6, 16, 8
    case = advection_case(d, n, seed_offset=0)
    A = advection_A(case)
    u = OH.from_cp(np.ones(2), case.ic_factors(), tree=build_tree(d, "linear"))
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1, tree=LINEAR)
    g = to_gpu(G, u, cap)
    op = G.advection_op(case.c, case.h)
    for step in range(10):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, cap)
        G.ht_step(ctx, g, op, case.dt, 1e-8, cap)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"


def test_tt_kinetic_heun2_steps(G):
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    rng = np.random.default_rng(5)
    F = [np.abs(rng.standard_normal((8, 2))) + 0.1 for _ in range(6)]
    u = OH.from_cp(np.array([1.0, 0.3]), F, tree=build_tree(6, "linear"))
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [8] * 6, cap=8, max_terms=5, tree=LINEAR)
    g = to_gpu(G, u, 8)
    for step in range(2):
        u, reps = OH.step_heun2(u, alphas, factors, kc.dt, 1e-8, 8)
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-8, 8, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        assert g.ranks() == reps[1].ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"


def test_tt_twelve_dim_deep_tree(G):
    """d = 12 on the linear tree: eleven levels of bottom-up QRs and top-down complements."""
    d, n, cap = 12, 6, 6
    case = advection_case(d, n, n_terms=3, seed_offset=4)
    A = advection_A(case)
    tree = build_tree(d, "linear")
    assert max(tree.depth) == 11
    u = OH.from_cp(np.ones(3), case.ic_factors(), tree=tree)
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1, tree=LINEAR)
    g = to_gpu(G, u, cap)
    op = G.advection_op(case.c, case.h)
    for step in range(3):
        u, rep = OH.step_rk2_poly(u, A, 1e-6, cap)
        G.ht_step(ctx, g, op, case.dt, 1e-6, cap)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"
