"""GPU parity at exactly the configurations the bench times: the AB2 and tensor-train lines on
the 6-D n = 64 advection workload, the full 256-instance ragged batch (one launch per step for
all instances; sampled instances against the oracle, every instance checked for finite values
and its rank cap), and the implicit Crank-Nicolson CP-ALS step on the kinetic workload."""
import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case
from tests.helpers import rel_err

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


def sync():
    import torch
    torch.cuda.synchronize()


def test_ab2_adv6d_n64(G):
    """AB2 on the 6-D n = 64 advection workload (r_max 32, tol 1e-8): RK2 start, 3 AB2 steps."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 1e-8, 32)
    ctx = G.Context(6, [64] * 6, cap=32, max_terms=2)
    gu = G.HTTensor(6, [64] * 6, 32)
    gu.upload(u1.node)
    gp = G.HTTensor(6, [64] * 6, 32)
    gp.upload(u0.node)
    op = G.advection_op(case.c, case.h)
    ref, prev = u1, u0
    for step in range(3):
        nxt, rep = OH.step_ab2(ref, prev, A, 1e-8, 32)
        prev, ref = ref, nxt
        G.ht_step_ab2(ctx, gu, gp, op, case.dt, 1e-8, 32)
        sync()
        ctx.check()
        assert gu.ranks() == rep.ranks, f"step {step}"
        assert rel_err(OH.HT(ref.tree, list(ref.n), gu.download()), ref) < TOL64, f"step {step}"


def test_tensor_train_adv6d_n64(G):
    """The same workload on the linear (tensor-train) tree, 3 RK2 steps."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    u = OH.from_cp(np.ones(2), case.ic_factors(), tree=build_tree(6, "linear"))
    ctx = G.Context(6, [64] * 6, cap=32, max_terms=1, tree=1)
    g = G.HTTensor(6, [64] * 6, 32, tree=1)
    g.upload(u.node)
    op = G.advection_op(case.c, case.h)
    for step in range(3):
        u, rep = OH.step_rk2_poly(u, A, 1e-8, 32)
        G.ht_step(ctx, g, op, case.dt, 1e-8, 32)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        assert rel_err(OH.HT(u.tree, list(g.n), g.download()), u) < TOL64, f"step {step}"


def test_full_ragged_batch(G):
    """The bench's batch: 256 instances (n from {32..128}, r_max from 8..48), two batched RK2
    steps; the largest-grid and largest-cap instances and a seeded sample against the oracle."""
    from paper_1803_10270_gb300.inputs import batched_advection_cases
    cases = batched_advection_cases(256, 6)
    ctxs, tens, ops = [], [], []
    for n, rmax, case in cases:
        ctxs.append(G.Context(6, [n] * 6, cap=rmax, max_terms=1))
        t = G.HTTensor(6, [n] * 6, rmax)
        t.upload(OH.from_cp(np.ones(2), case.ic_factors()).node)
        tens.append(t)
        ops.append(G.advection_op(case.c, case.h))
    b = G.Batch(ctxs, tens)
    for _ in range(2):
        b.step(ops, [c.dt for _, _, c in cases], [1e-8] * 256, [r for _, r, _ in cases])
    sync()
    for c in ctxs:
        c.check()
    ns = [n for n, _, _ in cases]
    caps = [r for _, r, _ in cases]
    rng = np.random.default_rng(12)
    pick = sorted({int(np.argmax(ns)), int(np.argmax(caps))} | set(int(i) for i in rng.choice(256, 4, replace=False)))
    for i in pick:
        n, rmax, case = cases[i]
        u = OH.from_cp(np.ones(2), case.ic_factors())
        A = advection_A(case)
        for _ in range(2):
            u, rep = OH.step_rk2_poly(u, A, 1e-8, rmax)
        assert tens[i].ranks() == rep.ranks, f"instance {i}"
        assert rel_err(OH.HT(u.tree, list(tens[i].n), tens[i].download()), u) < TOL64, f"instance {i}"
    for i, t in enumerate(tens):
        rk = t.ranks()
        assert max(rk[1:]) <= caps[i]
        assert all(np.isfinite(a).all() for a in t.download().values()), f"instance {i}"
    b.close()
    for c in ctxs:
        c.close()


def test_cn_kinetic_bench_config(G):
    """The implicit line: kinetic operator, n = 16, the seeded initial condition (CP rank 6),
    dt 5x the explicit step, 5 Gauss-Seidel sweeps, one step against the oracle."""
    import torch
    from oracle import cn_als as CN
    from oracle.cp import CP, to_full
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(16)
    w, F = kinetic_ic(kc)
    alphas, factors = kinetic_terms(kc)
    xn = CP(np.asarray(w), [np.asarray(f) for f in F])
    ref, eps_ref = CN.cn_als_step(xn, xn, alphas, factors, 5 * kc.dt, 5)
    r = len(w)
    ctx = G.Context(6, [16] * 6, cap=r, max_terms=5)
    kop = G.KineticOp(kc)
    gn = G.CPTensor(6, [16] * 6, r)
    gn.upload(w, F)
    gx = G.CPTensor(6, [16] * 6, r)
    gx.upload(w, F)
    eps = torch.zeros(5, dtype=torch.float64, device="cuda")
    G.cp_cn_als_step(ctx, gn, kop.op, 5 * kc.dt, gx, 5, eps=eps)
    sync()
    ctx.check()
    gw, gf = gx.download()
    got = CP(gw, gf)
    full_ref = to_full(ref)
    assert np.linalg.norm(to_full(got) - full_ref) / np.linalg.norm(full_ref) < 1e-10
    assert np.allclose(eps.cpu().numpy(), eps_ref, rtol=1e-6, atol=1e-14 * max(eps_ref))
