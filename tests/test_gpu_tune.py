"""The autotuner (paper_1803_10270_gb300.tune): it times the FP64 and tensor-core contraction
kernels and the two node-SVD forms on this GPU, and a context built from its cache gives the same
results as one with the library defaults (tuning changes launch shapes and the split between
kernels, not the arithmetic's target)."""
import numpy as np
import pytest

from oracle import ht as OH
from paper_1803_10270_gb300.inputs import advection_case
from tests.helpers import rel_err

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


def test_tune_time_gemm_probe(G):
    for route in (0, 1, 2):   # FP64, tensor-core split, split-FP32
        t = G.tune_time_gemm(64, 64, 64, 2, route=route, reps=3)
        assert 0.0 < t < 1000.0


def test_tuner_values_and_tuned_context(G):
    from paper_1803_10270_gb300 import tune
    res = tune.tune(0, write=False)
    assert res["tc_min_work"] >= 1
    assert set(res["gemm_ctas_per_sm_by_kc"].values()) <= {4, 8, 16, 32}
    assert 32 <= res["svd_cluster_min_cols"] <= 480
    # one step of the 6-D advection workload (n = 16) with the tuned values against the defaults
    # and the oracle, in both precision forms
    case = advection_case(6, 16, seed_offset=0)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    from oracle.problems import advection_A
    ref, _ = OH.step_rk2_poly(u0, advection_A(case), 1e-8, 8)
    tuned = {"tc_min_work": res["tc_min_work"], "gemm_ctas_per_sm": res["gemm_ctas_per_sm_by_kc"]["48"],
             "svd_cluster_min_cols": res["svd_cluster_min_cols"]}
    op = G.advection_op(case.c, case.h)
    for prec, bar in ((G.HT_PREC_FP64, 1e-10), (G.HT_PREC_MIXED, 1e-6)):
        for tuning in (tuned, {}):
            ctx = G.Context(6, [16] * 6, cap=8, max_terms=1, precision=prec, tuning=tuning)
            g = G.HTTensor(6, [16] * 6, 8)
            g.upload(u0.node)
            G.ht_step(ctx, g, op, case.dt, 1e-8, 8)
            ctx.check()
            got = OH.HT(u0.tree, [16] * 6, g.download())
            assert rel_err(got, ref) < bar
            ctx.close()
