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
