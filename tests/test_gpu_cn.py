"""GPU parity of the Crank-Nicolson CP-ALS step (cp_cn_als_step, Section 3.3, eqs. CNFDE,
ALS2, ML, MR) against the FP64 oracle: the kinetic operator (every factor kind but the
diagonal stencil), the variable-coefficient advection operator (diagonal stencils), the
pure-relaxation closed form and the Maxwellian fixed point."""
import numpy as np
import pytest

from oracle import cn_als as CN
from oracle.cp import CP, to_full
from oracle.problems import kinetic_terms, varcoef_terms
from paper_1803_10270_gb300.inputs import kinetic_case, varcoef_case

pytestmark = pytest.mark.gpu


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


def run_gpu(G, d, n, op, dt, xn: CP, x0: CP, sweeps, cap, max_terms, variant=0):
    import torch
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=max_terms)
    gn = G.CPTensor(d, [n] * d, cap)
    gn.upload(xn.weights, xn.factors)
    gx = G.CPTensor(d, [n] * d, cap)
    gx.upload(x0.weights, x0.factors)
    eps = torch.zeros(sweeps, dtype=torch.float64, device="cuda")
    G.cp_cn_als_step(ctx, gn, op, dt, gx, sweeps, variant=variant, eps=eps)
    torch.cuda.synchronize()
    ctx.check()
    w, f = gx.download()
    return CP(w, f), eps.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_cn_kinetic_matches_oracle(G):
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    rng = np.random.default_rng(41)
    xn = CP(np.array([1.0, 0.4, 0.2]), [np.abs(rng.standard_normal((8, 3))) + 0.1 for _ in range(6)])
    x0 = CP(np.ones(3), [f * (1.0 + 0.05 * rng.standard_normal(f.shape)) for f in xn.factors])
    x0.factors[0] = x0.factors[0] * xn.weights[None, :]
    dt = 5 * kc.dt
    ref, eps_ref = CN.cn_als_step(xn, x0, alphas, factors, dt, 3)
    kop = G.KineticOp(kc)
    got, eps = run_gpu(G, 6, 8, kop.op, dt, xn, x0, 3, cap=3, max_terms=5)
    assert np.allclose(got.weights, 1.0)
    assert rel(to_full(got), to_full(ref)) < 1e-10
    assert np.allclose(eps, eps_ref, rtol=1e-6, atol=1e-14 * max(eps_ref))


def test_cn_varcoef_matches_oracle(G):
    case = varcoef_case(3, 10, zmax=4.0)
    alphas, factors = varcoef_terms(case)
    rng = np.random.default_rng(42)
    xn = CP(np.array([1.0, 0.5]), [rng.standard_normal((10, 2)) for _ in range(3)])
    dt = 4 * case.dt
    ref, eps_ref = CN.cn_als_step(xn, xn, alphas, factors, dt, 2)
    vop = G.VarCoefOp(case)
    got, eps = run_gpu(G, 3, 10, vop.op, dt, xn, xn, 2, cap=2, max_terms=9)
    assert rel(to_full(got), to_full(ref)) < 1e-10


def test_cn_pure_relaxation_closed_form(G):
    d, n, nu, dt = 4, 6, 1.3, 0.2
    rng = np.random.default_rng(43)
    xn = CP(rng.uniform(0.5, 1.5, 3), [rng.standard_normal((n, 3)) for _ in range(d)])
    op = G.ht_op()
    op.d = d
    op.n_terms = 1
    op.kron_sum = 0
    op.alpha[0] = -nu
    for k in range(d):
        op.f[0][k] = G.ht_factor()
    got, _ = run_gpu(G, d, n, op, dt, xn, xn, 2, cap=3, max_terms=1)
    g = (1 - 0.5 * nu * dt) / (1 + 0.5 * nu * dt)
    assert rel(to_full(got), g * to_full(xn)) < 1e-13


def test_cn_uniform_maxwellian_fixed_point(G):
    kc = kinetic_case(8)
    ones, m = np.ones(8), kc.maxwellian()
    f = CP(np.ones(1), [ones[:, None]] * 3 + [m[:, None]] * 3)
    kop = G.KineticOp(kc)
    got, _ = run_gpu(G, 6, 8, kop.op, kc.dt, f, f, 2, cap=1, max_terms=5)
    assert rel(to_full(got), to_full(f)) < 1e-13


def test_cn_large_system_in_global_memory(G):
    """n r = 20 x 8 = 160 unknowns per mode: the 160 x 160 system no longer fits the solve's
    shared memory and is factorised in its global buffer."""
    case = varcoef_case(3, 20, zmax=5.0)
    alphas, factors = varcoef_terms(case)
    rng = np.random.default_rng(44)
    xn = CP(np.ones(8), [rng.standard_normal((20, 8)) for _ in range(3)])
    dt = 2 * case.dt
    ref, _ = CN.cn_als_step(xn, xn, alphas, factors, dt, 2)
    vop = G.VarCoefOp(case)
    got, _ = run_gpu(G, 3, 20, vop.op, dt, xn, xn, 2, cap=8, max_terms=9)
    assert rel(to_full(got), to_full(ref)) < 1e-10


def test_cn_damped_jacobi_matches_oracle(G):
    """The parallel variant (Appendix B, Algorithm 1): every mode from the same iterate, the
    increment damped by 1/4; kinetic operator, n = 8, rank 3, 4 sweeps against the oracle."""
    kc = kinetic_case(8)
    alphas, factors = kinetic_terms(kc)
    rng = np.random.default_rng(45)
    xn = CP(np.array([1.0, 0.4, 0.2]), [np.abs(rng.standard_normal((8, 3))) + 0.1 for _ in range(6)])
    x0 = CP(np.ones(3), [f * (1.0 + 0.05 * rng.standard_normal(f.shape)) for f in xn.factors])
    dt = 5 * kc.dt
    ref, eps_ref = CN.cn_als_step(xn, x0, alphas, factors, dt, 4, variant="jacobi_damped")
    kop = G.KineticOp(kc)
    got, eps = run_gpu(G, 6, 8, kop.op, dt, xn, x0, 4, cap=3, max_terms=5, variant=G.CP_ALS_JACOBI_DAMPED)
    assert rel(to_full(got), to_full(ref)) < 1e-10
    assert np.allclose(eps, eps_ref, rtol=1e-6, atol=1e-14 * max(eps_ref))


def test_cn_x_uniform_relaxation_closed_form(G):
    """An x-uniform f0 sees no transport, so the exact Crank-Nicolson step of the kinetic
    operator is f1 = g f0 + (1 - g) rho M (g = (1 - nu dt/2) / (1 + nu dt/2), rho = sum_v h^3 f0),
    a rank-2 tensor: the rank-2 step from the guess [f0, 0.3 M] reaches it to rounding (x_n of
    rank 1, x of rank 2; n = 8, 5 sweeps)."""
    kc = kinetic_case(8)
    v, m, ones = kc.vgrid(), kc.maxwellian(), np.ones(kc.n)
    f0 = CP(np.ones(1), [ones[:, None]] * 3 +
            [(m * (1 + 0.3 * v))[:, None], (m * (1 - 0.2 * v + 0.05 * v * v))[:, None], m[:, None]])
    dt = 5 * kc.dt
    g = (1 - 0.5 * kc.nu * dt) / (1 + 0.5 * kc.nu * dt)
    rho = float(np.prod([kc.hv * f0.factors[3 + k][:, 0].sum() for k in range(3)]))
    exact = g * to_full(f0) + (1 - g) * rho * to_full(CP(np.ones(1), [ones[:, None]] * 3 + [m[:, None]] * 3))
    x0 = CP(np.array([1.0, 0.3]),
            [np.concatenate([f0.factors[k], (ones if k < 3 else m)[:, None]], axis=1) for k in range(6)])
    kop = G.KineticOp(kc)
    got, _ = run_gpu(G, 6, 8, kop.op, dt, f0, x0, 5, cap=2, max_terms=5)
    assert rel(to_full(got), exact) < 1e-12
