"""GPU parity for the variable-coefficient advection operator (Section 4.1, eq. PDE-advR, Table
tab:ordering0): HEUN2 steps (a truncation after each stage) of ht_step with the N^2-term
operator against the FP64 oracle, ranks and entries."""
import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import varcoef_terms
from paper_1803_10270_gb300.inputs import varcoef_case
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


@pytest.mark.parametrize("N,n,zmax,cap,steps", [(2, 48, 6.0, 8, 6), (3, 20, 5.0, 4, 3)])
def test_varcoef_heun2_steps(G, N, n, zmax, cap, steps):
    case = varcoef_case(N, n, zmax=zmax)
    alphas, factors = varcoef_terms(case)
    u = OH.from_cp(np.ones(1), case.ic_factors())
    vop = G.VarCoefOp(case)
    ctx = G.Context(N, [n] * N, cap=cap, max_terms=N * N)
    g = G.HTTensor(N, [n] * N, cap)
    g.upload(u.node)
    for step in range(steps):
        u, reps = OH.step_heun2(u, alphas, factors, case.dt, 1e-8, cap)
        G.ht_step(ctx, g, vop.op, case.dt, 1e-8, cap, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        assert g.ranks() == reps[1].ranks, f"step {step}"
        assert rel_err(OH.HT(u.tree, list(g.n), g.download()), u) < TOL64, f"step {step}"


def test_varcoef_apply_matches_oracle(G):
    """ht_apply (EULER: u + dt L u, block diagonal, rank (1 + N^2) k) entry for entry."""
    N, n = 3, 12
    case = varcoef_case(N, n, zmax=4.0)
    alphas, factors = varcoef_terms(case)
    rng = np.random.default_rng(3)
    u = OH.from_cp(rng.standard_normal(2), [rng.standard_normal((n, 2)) for _ in range(N)])
    vop = G.VarCoefOp(case)
    ctx = G.Context(N, [n] * N, cap=2, max_terms=N * N)
    g = G.HTTensor(N, [n] * N, 2)
    g.upload(u.node)
    out = G.HTTensor(N, [n] * N, 2 * (N * N + 1))
    G.ht_apply(ctx, g, vop.op, 0.3, G.HT_APPLY_EULER, out)
    sync()
    ctx.check()
    ref = OH.apply_separable(u, [1.0] + [0.3 * a for a in alphas], [[None] * N] + factors)
    got = OH.HT(u.tree, list(out.n), out.download())
    assert np.allclose(OH.to_full(got), OH.to_full(ref), rtol=0, atol=1e-12 * np.abs(OH.to_full(ref)).max())


def test_varcoef_paper_grid_tiny_row_blocks(G):
    """The paper's 2-D grid ([-60, 60)^2, 600 nodes): the leaf matrices (600 rows) are reduced
    in row blocks, and the blocks far from the origin hold only the Gaussian's tails (entries
    down to 1e-300, squares below the normal range), where an unscaled Householder vector would
    overflow tau = 2 / (v.v).  Three HEUN2 steps against the oracle."""
    N, n, cap = 2, 600, 12
    case = varcoef_case(N, n)
    alphas, factors = varcoef_terms(case)
    u = OH.from_cp(np.ones(1), case.ic_factors())
    vop = G.VarCoefOp(case)
    ctx = G.Context(N, [n] * N, cap=cap, max_terms=N * N)
    g = G.HTTensor(N, [n] * N, cap)
    g.upload(u.node)
    for step in range(3):
        u, reps = OH.step_heun2(u, alphas, factors, case.dt, 1e-8, cap)
        G.ht_step(ctx, g, vop.op, case.dt, 1e-8, cap, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        assert g.ranks() == reps[1].ranks, f"step {step}"
        assert rel_err(OH.HT(u.tree, list(g.n), g.download()), u) < TOL64, f"step {step}"
