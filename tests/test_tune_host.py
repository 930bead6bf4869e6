"""The autotuner's host logic without a GPU: the tensor-core crossover rule and the cache lookup."""
import json

from paper_1803_10270_gb300 import tune


def test_crossover_is_the_smallest_work_from_which_the_tensor_cores_always_win():
    # (work, CUDA-core ms, tensor-core ms, shape): a win at 4096 that a loss at 8192 undoes does not count
    pts = [(512, 0.006, 0.012, None), (4096, 0.020, 0.010, None), (8192, 0.030, 0.040, None),
           (65536, 0.080, 0.050, None), (1 << 20, 0.900, 0.100, None)]
    assert tune.crossover(pts) == 65536
    assert tune.crossover(list(reversed(pts))) == 65536          # order of measurement is irrelevant


def test_crossover_when_the_tensor_cores_never_or_always_win():
    never = [(512, 0.01, 0.02, None), (4096, 0.02, 0.03, None)]
    always = [(512, 0.02, 0.01, None), (4096, 0.03, 0.02, None)]
    assert tune.crossover(never) == 8192                          # twice the largest measured work
    assert tune.crossover(always) == 512
    assert tune.crossover([]) == 1 << 40


def test_cached_values_by_capacity_bucket(monkeypatch, tmp_path):
    cache = tmp_path / "tuning.json"
    cache.write_text(json.dumps({"GB300|152": {"tc_min_work": 84934656, "svd_cluster_min_cols": 64,
                                               "gemm_ctas_per_sm_by_kc": {"48": 8, "96": 16, "192": 16,
                                                                          "100000": 32}}}))
    monkeypatch.setattr(tune, "CACHE", str(cache))
    monkeypatch.setattr(tune, "device_key", lambda device=0: "GB300|152")
    assert tune.cached(0, kc=40) == {"tc_min_work": 84934656, "svd_cluster_min_cols": 64, "gemm_ctas_per_sm": 8}
    assert tune.cached(0, kc=96)["gemm_ctas_per_sm"] == 16
    assert tune.cached(0, kc=448)["gemm_ctas_per_sm"] == 32
    monkeypatch.setattr(tune, "device_key", lambda device=0: "other|1")
    assert tune.cached(0, kc=96) == {}
