"""Host-side logic of bench.py on CPU: replica aggregation over gloo ranks and the reference
arm's rank gating (no GPU involved)."""
import json
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_max, value = bench.aggregate_replicas(100.0 * (rank + 1), steps=50)
    q.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value in res:
        assert ms_max == 200.0                      # the slowest rank sets the job time
        assert abs(value - 2 * 50 / 0.2) < 1e-9      # every rank's steps count


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.aggregate_replicas(250.0, steps=10)
    assert ms == 250.0 and abs(v - 40.0) < 1e-12


def test_reference_arm_only_rank0_works(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def test_oracle_sample_process_runs_with_the_thread_count_set():
    sys.path.insert(0, ROOT)
    import bench
    res, err = bench.oracle_sample_process(0.3, 1)
    assert err is None and res["steps"] >= 1 and res["value"] > 0


def test_reference_arm_line_carries_the_contract_keys(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.setattr(bench, "oracle_sample_process",
                        lambda seconds, threads: ({"steps": 10, "seconds": 2.0, "value": 5.0}, None))
    bench.run_reference(argparse.Namespace(steps=3, warmup=1, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] == 5.0 and line["unit"] == "steps/s"
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 1 and line["higher_is_better"]
    assert line["metric"] == bench.METRIC and line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == 5.0 and cb["cores"] >= 1 and "sample" in cb
    assert isinstance(cb["cpu"], str) and "cores" in cb["cpu"]
    assert line["e2e"] == {"value": 5.0, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_class_roofline_labels_the_split_fp32_contraction():
    """Per-class shares and the dominant class's roofline from a profiler read-out: in a mixed-form
    context the gemm class is the split-FP32 kernel against its FP32-pipe bound, in an FP64
    context the FP64 kernel against the FP64 peak."""
    import types
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    prof = {"gemm": {"ms": 4.0, "launches": 8, "flops": 2e9}, "qr": {"ms": 1.0, "launches": 4, "flops": 1e8},
            "gemm_tc": {"ms": 0.0, "launches": 0, "flops": 0.0}}
    for prec, kernel, peak in ((1, "gemm_f32x2_kernel", bench.F32X2_PEAK_TFLOPS),
                               (0, "gemm_kernel", bench.FP64_PEAK_TFLOPS)):
        ctx = types.SimpleNamespace(cfg=types.SimpleNamespace(precision=prec))
        roof, shares = bench.class_roofline(prof, 2, ctx)
        dom = roof["dominant"]
        assert dom["kernel"] == kernel and dom["peak"] == peak
        assert abs(dom["achieved"] - 2e9 / 4e-3 / 1e12) < 1e-12
        assert abs(shares["gemm"]["share"] - 0.8) < 1e-12 and shares["gemm"]["ms_per_step"] == 2.0
        assert abs(shares["qr"]["counted_tflops"] - 1e8 / 1e-3 / 1e12) < 1e-12
        assert "gemm_tc" not in shares


def test_roofline_traffic_only_from_a_capture_of_the_same_line(tmp_path, monkeypatch):
    """roofline.traffic comes from a counter record of the class's kernel taken on the line's own
    workload; a record of another line, or a stale one, leaves it null.  The qr and svd classes
    name both of their kernels."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel source\n")
    recs = [{"kernel": "qr_r_kernel", "line": "adv6d", "workload": "w1", "when": "d", "sources": {},
             "dram_bytes_per_launch": 1000},
            {"kernel": "qr_coop_kernel", "line": "wide", "workload": "w2", "when": "d",
             "sources": {str(src): "0" * 64}, "dram_bytes_per_launch": 5000}]
    f = tmp_path / "counters.json"
    f.write_text(json.dumps({"records": recs}))
    monkeypatch.setattr(bench, "COUNTERS", str(f))
    prof = {"qr": {"ms": 3.0, "launches": 6, "flops": 3e8}, "gemm": {"ms": 1.0, "launches": 2, "flops": 1e8}}
    roof, _ = bench.class_roofline(prof, 2, None, "adv6d")
    assert roof["dominant"]["kernel"] == "qr_r_kernel/qr_coop_kernel"
    assert roof["dominant"]["traffic"] == 1000 and roof["dominant"]["traffic_record"]["kernel"] == "qr_r_kernel"
    for line in ("kinetic", None):
        roof, _ = bench.class_roofline(prof, 2, None, line)
        assert roof["dominant"]["traffic"] is None and "traffic_record" not in roof["dominant"]
    # the coop record's source hash does not match: stale, so the wide line gets no traffic either
    roof, _ = bench.class_roofline(prof, 2, None, "wide")
    assert roof["dominant"]["traffic"] is None
    assert bench.KERNEL_NAMES["svd"] == "svd_kernel/svd_cluster_kernel"


def test_biorth_form_switch_matches_the_binding(monkeypatch):
    """`--biorth-form` names the binding's ht_config.biorth_form values; cta is the default."""
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1803_10270_gb300 import htgpu as G
    assert bench.BIORTH_FORMS == {"cta": G.BIORTH_FORM_CTA, "cluster": G.BIORTH_FORM_CLUSTER}
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.parse().biorth_form == "cta"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--line", "wide", "--biorth-form", "cluster"])
    assert bench.BIORTH_FORMS[bench.parse().biorth_form] == G.BIORTH_FORM_CLUSTER
