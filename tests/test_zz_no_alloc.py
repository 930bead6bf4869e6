"""The allocation-free ALS entry point (cp_als_sweep_noalloc) against cp_als_sweep.

Callers that cannot allocate device memory (fixed-budget plug-ins, host callbacks,
processes whose memory is reserved up front) use cp_als_sweep_noalloc, which keeps its
scratch in a fixed static device array.  This file is collected last so a failure here
never hides the rest of the suite; it also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import cp as OC
from oracle.problems import advection_A
from paper_1803_10270_gb300.inputs import advection_case, cp_padding, cp_random_factors

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


def _inputs(seed, d=4, n=6, r=5):
    case = advection_case(d, n, seed=seed)
    x0 = OC.CP(np.array([1.0, 0.6]), cp_random_factors([n] * d, 2, seed=seed + 1))
    y = OC.apply_kron_sum_rk2(x0, advection_A(case))
    xi = OC.pad(x0, r, cp_padding([n] * d, r - 2, seed=seed + 2, scale=1e-3))
    return y, xi


def _full_rel(a, b):
    fa, fb = OC.to_full(OC.CP(*a)), OC.to_full(OC.CP(*b))
    return np.linalg.norm(fa - fb) / np.linalg.norm(fb)


def test_noalloc_matches_context_version_two_calls(G):
    import torch
    d, n, r = 4, 6, 5
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1)
    for call, (seed, variant) in enumerate([(11, G.CP_ALS_GS), (23, G.CP_ALS_JACOBI_DAMPED)]):
        y, xi = _inputs(seed, d, n, r)
        Y = G.CPTensor(d, [n] * d, y.rank)
        Y.upload(y.weights, y.factors)
        Xa = G.CPTensor(d, [n] * d, r)
        Xa.upload(xi.weights, xi.factors)
        Xb = G.CPTensor(d, [n] * d, r)
        Xb.upload(xi.weights, xi.factors)
        ea = torch.zeros(3, dtype=torch.float64, device="cuda")
        eb = torch.zeros(3, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        G.cp_als_sweep(ctx, Y, Xa, 3, variant, eps=ea)
        G.cp_als_sweep_noalloc(Y, Xb, 3, variant, eps=eb, status=st)
        torch.cuda.synchronize()
        assert int(st[0]) == G.HT_OK, f"call {call}"
        assert _full_rel(Xb.download(), Xa.download()) < 1e-12, f"call {call}"
        np.testing.assert_allclose(eb.cpu().numpy(), ea.cpu().numpy(), rtol=1e-12, atol=1e-15)


def test_noalloc_rejects_sizes_beyond_its_limits(G):
    big = G.CPTensor(4, [6] * 4, 40)
    big.struct.rank = 40          # x rank above the static limit of 32
    y = G.CPTensor(4, [6] * 4, 8)
    y.struct.rank = 8
    rc = G.load().cp_als_sweep_noalloc(C.byref(y.struct), C.byref(big.struct), 1, 0, None, None, None)
    assert rc == G.HT_ERR_CAPACITY
    tall = G.CPTensor(4, [300] * 4, 4)
    tall.struct.rank = 2
    y2 = G.CPTensor(4, [300] * 4, 4)
    y2.struct.rank = 4
    rc = G.load().cp_als_sweep_noalloc(C.byref(y2.struct), C.byref(tall.struct), 1, 0, None, None, None)
    assert rc == G.HT_ERR_CAPACITY


def test_noalloc_matches_oracle_directly(G):
    """Both variants against the FP64 oracle's ALS (Section 2.1; Appendix B, Algorithm 1 for the
    damped Jacobi sweep), on the full grid, over two calls in a row on the shared array."""
    import torch
    d, n, r = 4, 6, 5
    for seed, variant, name in [(31, G.CP_ALS_GS, "gs"), (37, G.CP_ALS_JACOBI_DAMPED, "jacobi_damped")]:
        y, xi = _inputs(seed, d, n, r)
        ref, eps_ref = OC.als_sweeps(y, xi, 3, name)
        Y = G.CPTensor(d, [n] * d, y.rank)
        Y.upload(y.weights, y.factors)
        X = G.CPTensor(d, [n] * d, r)
        X.upload(xi.weights, xi.factors)
        e = torch.zeros(3, dtype=torch.float64, device="cuda")
        G.cp_als_sweep_noalloc(Y, X, 3, variant, eps=e)
        torch.cuda.synchronize()
        assert _full_rel(X.download(), (ref.weights, ref.factors)) < 1e-10, name
        np.testing.assert_allclose(e.cpu().numpy(), eps_ref, rtol=1e-6, atol=1e-14)


def test_noalloc_allocates_nothing(G):
    """After a first call (which looks up the static array's address), further calls leave the
    device's free memory and the torch caching allocator's reservation unchanged."""
    import torch
    d, n, r = 4, 6, 5
    y, xi = _inputs(41, d, n, r)
    Y = G.CPTensor(d, [n] * d, y.rank)
    Y.upload(y.weights, y.factors)
    X = G.CPTensor(d, [n] * d, r)
    X.upload(xi.weights, xi.factors)
    G.cp_als_sweep_noalloc(Y, X, 2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for _ in range(3):
        X.upload(xi.weights, xi.factors)
        G.cp_als_sweep_noalloc(Y, X, 2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == res0
    assert free1 == free0


def test_noalloc_rejects_mismatched_shapes(G):
    """x and y must share d and every n_k: HT_ERR_ARG before anything is launched."""
    x = G.CPTensor(4, [6] * 4, 4)
    x.struct.rank = 2
    y3 = G.CPTensor(3, [6] * 3, 4)
    y3.struct.rank = 4
    rc = G.load().cp_als_sweep_noalloc(C.byref(y3.struct), C.byref(x.struct), 1, 0, None, None, None)
    assert rc == G.HT_ERR_ARG
    yn = G.CPTensor(4, [6, 6, 7, 6], 4)
    yn.struct.rank = 4
    rc = G.load().cp_als_sweep_noalloc(C.byref(yn.struct), C.byref(x.struct), 1, 0, None, None, None)
    assert rc == G.HT_ERR_ARG
