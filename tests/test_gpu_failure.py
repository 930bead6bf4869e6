"""Failure detection without a GPU fault: the grid barrier that separates the phases of the
persistent ALS kernel waits a bounded time.  A CTA that never arrives makes the others give up
and report HT_ERR_TIMEOUT through the device error word; the device stays usable."""
import numpy as np
import pytest

from oracle import cp as OC
from oracle.problems import advection_A
from paper_1803_10270_gb300.inputs import advection_case, cp_random_factors

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


def test_barrier_passes_when_every_cta_arrives(G):
    assert G.selftest_grid_barrier(24, -1) == G.HT_OK
    assert G.selftest_grid_barrier(1, -1) == G.HT_OK


def test_barrier_times_out_on_a_missing_cta_and_device_stays_usable(G):
    import torch
    assert G.selftest_grid_barrier(24, 5) == G.HT_ERR_TIMEOUT
    # the context is intact: a full structured ALS call still matches the oracle
    d, n, r = 3, 8, 2
    case = advection_case(d, n, seed=77)
    A = advection_A(case)
    fac = cp_random_factors([n] * d, r, seed=78)
    x0 = OC.CP(np.array([1.0, 0.5]), fac)
    ref, _ = OC.als_sweeps(OC.apply_kron_sum_rk2(x0, A), x0, 2)
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1)
    xo = G.CPTensor(d, [n] * d, r)
    xo.upload(x0.weights, x0.factors)
    x = G.CPTensor(d, [n] * d, r)
    x.upload(x0.weights, x0.factors)
    G.cp_als_sweep_rk2(ctx, xo, G.advection_op(case.c, case.h), case.dt, x, 2)
    torch.cuda.synchronize()
    ctx.check()
    w, f = x.download()
    got = OC.to_full(OC.CP(w, f))
    want = OC.to_full(ref)
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_barrier_argument_errors(G):
    assert G.selftest_grid_barrier(0, -1) == G.HT_ERR_ARG
    assert G.selftest_grid_barrier(65, -1) == G.HT_ERR_ARG
    assert G.selftest_grid_barrier(4, 4) == G.HT_ERR_ARG
