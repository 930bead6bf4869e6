"""The mixed-precision form (HT_PREC_MIXED): every dense contraction of the HSVD truncation on the
tensor cores (BF16 digit planes, FP32 accumulation), QR R factors, node SVDs, thresholds and the
X_t Y_t = I refinement of the kept subspaces in FP64.  Bar: relative error <= 1e-6 against the FP64
oracle at every step compared, and against the FP64 GPU form (itself within 1e-10 of the oracle,
tests/test_gpu_workloads.py) at every step of the longer runs and at their final time."""
import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A
from paper_1803_10270_gb300.inputs import advection_case, batched_advection_cases
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6


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
    t = G.HTTensor(u.tree.d, u.n, cap)
    t.upload(u.node)
    return t


def from_gpu(t, tree):
    return OH.HT(tree, list(t.n), t.download())


def test_mixed_rejects_bad_slice_counts(G):
    for bad in (1, 5):
        with pytest.raises(G.HTError):
            G.Context(4, [6] * 4, cap=4, max_terms=1, precision=G.HT_PREC_MIXED, mixed_slices=bad)


@pytest.mark.parametrize("slices", [4])
def test_mixed_12d_n128_against_oracle(G, slices):
    """12-D advection at full size (n = 128, r_max 64, tol 1e-8, the separable rank-3 initial
    condition): five mixed steps, each against the oracle's step.  (Three slices, 2^-23 per
    contraction, measured 9e-7 after one step and 3.8e-6 after five: too coarse for this
    tolerance, hence the default of four.)"""
    d, n, cap = 12, 128, 64
    case = advection_case(d, n, n_terms=3, seed_offset=4)
    A = advection_A(case)
    u = OH.from_cp(np.ones(3), case.ic_factors())
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1, precision=G.HT_PREC_MIXED, mixed_slices=slices)
    g = to_gpu(G, u, cap)
    op = G.advection_op(case.c, case.h)
    errs = []
    for step in range(5):
        u, _ = OH.step_rk2_poly(u, A, 1e-8, cap)
        G.ht_step(ctx, g, op, case.dt, 1e-8, cap)
        sync()
        ctx.check()
        errs.append(rel_err(from_gpu(g, u.tree), u))
    print(f"12-D mixed ({slices} slices) vs oracle per step: " + " ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= TOL_MIXED


def _run_pair(G, d, n, cap, max_terms, u0, op, dt, tol, steps, scheme, slices=4, every=1):
    """The same run in the FP64 and the mixed form; relative error of mixed vs FP64 at every
    `every`-th step and at the last."""
    tree = u0.tree
    c64 = G.Context(d, [n] * d, cap=cap, max_terms=max_terms)
    cmx = G.Context(d, [n] * d, cap=cap, max_terms=max_terms, precision=G.HT_PREC_MIXED, mixed_slices=slices)
    g64 = to_gpu(G, u0, cap)
    gmx = to_gpu(G, u0, cap)
    errs = []
    for step in range(steps):
        G.ht_step(c64, g64, op, dt, tol, cap, scheme=scheme)
        G.ht_step(cmx, gmx, op, dt, tol, cap, scheme=scheme)
        if (step + 1) % every == 0 or step == steps - 1:
            sync()
            c64.check()
            cmx.check()
            errs.append(rel_err(from_gpu(gmx, tree), from_gpu(g64, tree)))
    c64.close()
    cmx.close()
    return errs


def test_mixed_adv6d_n64_200_steps_against_fp64(G):
    """6-D advection n = 64 (r_max 32, tol 1e-8), the configuration's 200 RK2 steps: mixed against
    the FP64 GPU form every 10 steps and at the final time; three steps against the oracle."""
    d, n, cap = 6, 64, 32
    case = advection_case(d, n, seed_offset=1)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    op = G.advection_op(case.c, case.h)
    # against the oracle
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1, precision=G.HT_PREC_MIXED)
    g = to_gpu(G, u0, cap)
    u = u0
    for step in range(3):
        u, _ = OH.step_rk2_poly(u, A, 1e-8, cap)
        G.ht_step(ctx, g, op, case.dt, 1e-8, cap)
        sync()
        assert rel_err(from_gpu(g, u.tree), u) <= TOL_MIXED, f"step {step}"
    ctx.close()
    errs = _run_pair(G, d, n, cap, 1, u0, op, case.dt, 1e-8, 200, G.HT_SCHEME_RK2POLY, every=10)
    print("6-D n=64 mixed vs FP64 every 10 steps: " + " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) <= TOL_MIXED


def test_mixed_kinetic_n64_full_size(G):
    """The kinetic workload at full size (n = 64, r_max 64, five terms, HEUN2, tol 1e-6): two mixed
    steps against the oracle, then 20 steps against the FP64 GPU form (node factors 250-370 columns
    wide, the stage sums' 3960 x 252 matrices)."""
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(64)
    w, F = kinetic_ic(kc)
    u0 = OH.from_cp(w, F)
    alphas, factors = kinetic_terms(kc)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [64] * 6, cap=64, max_terms=5, precision=G.HT_PREC_MIXED)
    g = to_gpu(G, u0, 64)
    u = u0
    for step in range(2):
        u, _ = OH.step_heun2(u, alphas, factors, kc.dt, 1e-6, 64)
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        e = rel_err(from_gpu(g, u.tree), u)
        print(f"kinetic mixed vs oracle, step {step + 1}: {e:.2e}")
        assert e <= TOL_MIXED
    ctx.close()
    errs = _run_pair(G, 6, 64, 64, 5, u0, kop.op, kc.dt, 1e-6, 20, G.HT_SCHEME_HEUN2, every=2)
    print("kinetic mixed vs FP64 every 2 steps: " + " ".join(f"{e:.1e}" for e in errs))
    assert max(errs) <= TOL_MIXED


def test_mixed_batch_matches_single_instances(G):
    """A ragged batch of eight advection instances in the mixed form (one tensor-core launch per
    contraction list for all instances) against each instance stepped alone in the mixed form,
    and against the oracle."""
    import torch
    cases = batched_advection_cases(8)
    ctxs, us, ref_ctx, ref_us, ops, orc = [], [], [], [], [], []
    for (n, rmax, case) in cases:
        u0 = OH.from_cp(np.ones(2), case.ic_factors())
        for lst_c, lst_u in ((ctxs, us), (ref_ctx, ref_us)):
            lst_c.append(G.Context(6, [n] * 6, cap=rmax, max_terms=1, precision=G.HT_PREC_MIXED))
            lst_u.append(to_gpu(G, u0, rmax))
        ops.append(G.advection_op(case.c, case.h))
        orc.append(u0)
    b = G.Batch(ctxs, us)
    dts = [c.dt for (_, _, c) in cases]
    for step in range(3):
        b.step(ops, dts, [1e-8] * 8, [r for (_, r, _) in cases])
        for i, (n, rmax, case) in enumerate(cases):
            G.ht_step(ref_ctx[i], ref_us[i], ops[i], case.dt, 1e-8, rmax)
            orc[i], _ = OH.step_rk2_poly(orc[i], advection_A(case), 1e-8, rmax)
    torch.cuda.synchronize()
    for i in range(8):
        tree = orc[i].tree
        a, r = from_gpu(us[i], tree), from_gpu(ref_us[i], tree)
        assert rel_err(a, r) <= 1e-12, f"instance {i}"
        assert rel_err(a, orc[i]) <= TOL_MIXED, f"instance {i}"
    b.close()
