"""GPU parity of the paper's two-step explicit scheme (eq. AB2_) through ht_step_ab2."""
import numpy as np
import pytest

from oracle import fullgrid as FG
from oracle import ht as OH
from oracle.problems import advection_A
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


def upload(G, u: OH.HT, cap):
    t = G.HTTensor(u.tree.d, u.n, cap)
    t.upload(u.node)
    return t


def test_ab2_steps_match_oracle(G):
    """6-D advection, n=16, r_max 8, tol 1e-8: RK2 start step, then 6 AB2 steps vs the oracle."""
    case = advection_case(6, 16, seed_offset=0)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 1e-8, 8)
    ctx = G.Context(6, [16] * 6, cap=8, max_terms=2)
    gu = upload(G, u1, 8)
    gp = upload(G, u0, 8)
    op = G.advection_op(case.c, case.h)
    ref, prev = u1, u0
    for step in range(6):
        nxt, rep = OH.step_ab2(ref, prev, A, 1e-8, 8)
        prev, ref = ref, nxt
        G.ht_step_ab2(ctx, gu, gp, op, case.dt, 1e-8, 8)
        sync()
        ctx.check()
        assert gu.ranks() == rep.ranks, f"step {step}"
        assert rel_err(OH.HT(ref.tree, list(ref.n), gu.download()), ref) < TOL64, f"step {step}"
        assert rel_err(OH.HT(prev.tree, list(prev.n), gp.download()), prev) < TOL64, f"step {step} (u_prev)"


def test_ab2_untruncated_equals_full_grid(G):
    d, n = 4, 6
    case = advection_case(d, n, seed=61)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 0.0, 24)
    cap = 24
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=2)
    gu = upload(G, u1, cap)
    gp = upload(G, u0, cap)
    G.ht_step_ab2(ctx, gu, gp, G.advection_op(case.c, case.h), case.dt, 0.0, cap)
    sync()
    want = FG.ab2_step(OH.to_full(u1), OH.to_full(u0), case.c, case.h, case.dt)
    got = OH.to_full(OH.HT(u1.tree, list(u1.n), gu.download()))
    # exact up to rounding: singular values at the rounding level of |u| (64 eps |u|) are
    # dropped even at tolerance 0, which moves T(u) at that level only
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_ab2_argument_errors(G):
    d, n = 4, 6
    case = advection_case(d, n, seed=62)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    op = G.advection_op(case.c, case.h)
    ctx = G.Context(d, [n] * d, cap=4, max_terms=2)
    gu = upload(G, u0, 4)
    with pytest.raises(G.HTError):
        G.ht_step_ab2(ctx, gu, gu, op, case.dt, 1e-8, 4)          # u_prev must be its own tensor
    small = G.Context(d, [n] * d, cap=4, max_terms=1)            # truncation input 3 cap < 4 cap
    gp = upload(G, u0, 4)
    with pytest.raises(G.HTError):
        G.ht_step_ab2(small, gu, gp, op, case.dt, 1e-8, 4)


def test_ht_add_matches_oracle(G):
    """ht_add: a u + b w exactly (ranks add, block-diagonal transfers), against the oracle's add."""
    from tests.helpers import random_ht
    d, n = 4, 7
    u = random_ht(d, n, 3, seed=71)
    w = random_ht(d, n, 2, seed=72)
    ref = OH.add(1.7, u, -0.3, w)
    ctx = G.Context(d, [n] * d, cap=5, max_terms=1)
    gu, gw = upload(G, u, 5), upload(G, w, 5)
    out = G.HTTensor(d, [n] * d, 10)
    G.ht_add(ctx, 1.7, gu, -0.3, gw, out)
    sync()
    got = OH.HT(u.tree, [n] * d, out.download())
    assert out.ranks()[1:] == [5] * (2 * d - 2)
    full = OH.to_full
    assert np.abs(full(got) - full(ref)).max() <= 1e-14 * np.abs(full(ref)).max()
    with pytest.raises(G.HTError):
        G.ht_add(ctx, 1.0, gu, 1.0, gw, G.HTTensor(d, [n] * d, 8))     # out->cap < 5 + 5


@pytest.mark.parametrize("variant,name", [(0, "argument"), (1, "difference")])
def test_ab2_split_steps_match_oracle(G, variant, name):
    """The split evaluation of the AB2 step (Section 3.2, after eq. AB2_), both readings: 6-D
    advection n = 16, r_max 8, tol 1e-8, an RK2 start step and 5 split steps, ranks and tensors
    (u and u_prev) against the oracle's step_ab2_split."""
    case = advection_case(6, 16, seed_offset=0)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 1e-8, 8)
    ctx = G.Context(6, [16] * 6, cap=8, max_terms=1)
    gu, gp = upload(G, u1, 8), upload(G, u0, 8)
    op = G.advection_op(case.c, case.h)
    ref, prev = u1, u0
    for step in range(5):
        nxt, reps = OH.step_ab2_split(ref, prev, A, 1e-8, 8, name)
        prev, ref = ref, nxt
        G.ht_step_ab2_split(ctx, gu, gp, op, case.dt, 1e-8, 8, variant)
        sync()
        ctx.check()
        assert gu.ranks() == reps[-1].ranks, f"step {step}"
        assert rel_err(OH.HT(ref.tree, list(ref.n), gu.download()), ref) < TOL64, f"step {step}"
        assert rel_err(OH.HT(prev.tree, list(prev.n), gp.download()), prev) < TOL64, f"step {step} (u_prev)"


@pytest.mark.parametrize("variant", [0, 1])
def test_ab2_split_untruncated_equals_full_grid(G, variant):
    d, n = 4, 6
    case = advection_case(d, n, seed=63)
    A = advection_A(case)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 0.0, 24)
    cap = 24
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1)
    gu, gp = upload(G, u1, cap), upload(G, u0, cap)
    G.ht_step_ab2_split(ctx, gu, gp, G.advection_op(case.c, case.h), case.dt, 0.0, cap, variant)
    sync()
    want = FG.ab2_step(OH.to_full(u1), OH.to_full(u0), case.c, case.h, case.dt)
    got = OH.to_full(OH.HT(u1.tree, list(u1.n), gu.download()))
    assert np.linalg.norm(got - want) <= 1e-11 * np.linalg.norm(want)


def test_ab2_split_adv6d_n64_against_oracle(G):
    """The 6-D advection workload at n = 64 (r_max 32, tol 1e-8): three split steps of each reading
    against the oracle, and the cancellation study's quantity, the distance of each split result
    from the exact-sum step ht_step_ab2 after the same steps (within a few tol |u|)."""
    case = advection_case(6, 64, seed_offset=1)
    A = advection_A(case)
    op = G.advection_op(case.c, case.h)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    u1, _ = OH.step_rk2_poly(u0, A, 1e-8, 32)
    exact, eprev = u1, u0
    for _ in range(3):
        nxt, _ = OH.step_ab2(exact, eprev, A, 1e-8, 32)
        eprev, exact = exact, nxt
    for variant, name in ((0, "argument"), (1, "difference")):
        ctx = G.Context(6, [64] * 6, cap=32, max_terms=1)
        gu, gp = upload(G, u1, 32), upload(G, u0, 32)
        ref, prev = u1, u0
        for step in range(3):
            nxt, _ = OH.step_ab2_split(ref, prev, A, 1e-8, 32, name)
            prev, ref = ref, nxt
            G.ht_step_ab2_split(ctx, gu, gp, op, case.dt, 1e-8, 32, variant)
        sync()
        ctx.check()
        got = OH.HT(ref.tree, list(ref.n), gu.download())
        assert rel_err(got, ref) < TOL64, name
        assert rel_err(got, exact) < 20 * 1e-8, name
        ctx.close()
