"""Benchmark: explicit time steps of 6-D advection held in HT and CP format on GB300.

Workload: u_t + c.grad u = 0 on [0,2pi)^6, n = 64 points per
dimension, central differences, RK2 with dt = 0.2 h, initial condition
sum_{m=1,2} prod_i exp(sin(x_i + phi_{m,i})) (c, phi seeded).  One step runs the whole hot
path once:
  HT route: ht_step = exact rank-3r RK2-polynomial apply + root-to-leaves HSVD truncation
            (tol 1e-8, r_max 32);
  CP route: cp_als_sweep_rk2 = 5 Gauss-Seidel ALS sweeps (rank 24) towards the exact
            y = p(dt L) x_n (rank 28 r), with y represented by its factor powers.
value = steps/s with all inputs resident in HBM (CUDA events on the launching stream, L2
flushed between timed steps).  e2e = the same through host buffers (pinned host -> device
copy of the state, step, device -> host copy, every step).

--impl reference times the FP64 CPU oracle (the plain restatement of the method) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HT steps/s (apply+truncate) vs FP64 plain form at rel err ≤1e-6; % roofline"
WORKLOAD = ("6-D advection n=64: HT r_max=32 tol=1e-8 + CP rank<=24 with 5 ALS sweeps, "
            "RK2 dt=0.2h; one step = HT apply+HSVD truncate and CP apply+ALS")
D, N, RMAX, TOL, CP_R, SWEEPS = 6, 64, 32, 1e-8, 24, 5
# FP64 peak of GB300 derived from the nominal 1.25 TFLOP/s: 152 SMs x 2070 MHz x 4 FP64
# flop/clk/SM (2 FMA/clk/SM).  An FMA-chain probe measured 1.196 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
# The split-FP32 contraction of the mixed form (gemm_f32x2_kernel) issues 10 FP32 operations per
# FP64 multiply-add (3 FMA, 1 MUL, 6 ADD/SUB: the product, its error, two cross terms, TwoSum and
# the low-part sum) on 128 FP32 lanes per SM: 152 x 2.07 GHz x 128 / 10 multiply-adds per second,
# x 2 flops, in FP64-equivalent flops of the contraction.
F32X2_PEAK_TFLOPS = 152 * 2.070e9 * 128 / 10 * 2 / 1e12
HT_PREC_MIXED = 1   # ht_precision of the C ABI
BIORTH_FORMS = {"cta": 0, "cluster": 1}   # ht_config.biorth_form
KERNEL_NAMES = {"apply": "apply_leaf_kernel/apply_xfer_kernel", "gemm": "gemm_kernel",
                "qr": "qr_r_kernel/qr_coop_kernel", "svd": "svd_kernel/svd_cluster_kernel", "plan": "plan_pre_kernel/rank_select_kernel",
                "cp_small": "cp_hadamard_kernel/cp_normalize_kernel/...",
                "cp_solve": "cp_als_rk2_cluster/cp_als_rk2_persistent"}
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def config_keys(precision: str, l2: str, parallelism: str) -> dict:
    """The workload identity, the same keys in both arms of the benchmark."""
    return {"workload": WORKLOAD, "d": D, "n": N, "ht_r_max": RMAX, "tol": TOL, "cp_rank": CP_R,
            "als_sweeps": SWEEPS, "precision": precision, "l2": l2, "parallelism": parallelism}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="launch every kernel per step instead of a CUDA graph")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--gemm-shape", default="384,147456,384", help="m,n,k of the --line gemm_tc probe")
    p.add_argument("--no-tune", dest="tune", action="store_false",
                   help="skip the autotuner (contexts then use the library defaults or an earlier cache)")
    p.add_argument("--batched", type=int, default=256, help="instances of the ragged batched workload (0: skip)")
    p.add_argument("--no-d12", dest="d12", action="store_false", help="skip the 12-D n=128 line")
    p.add_argument("--line", default="all",
                   choices=["all", "d12", "ab2", "batched", "varcoef", "tt", "cn", "kinetic", "mixed", "wide", "gemm_tc"],
                   help="run one side line alone (for profiling) and print its JSON object")
    p.add_argument("--biorth-form", default="cta", choices=["cta", "cluster"],
                   help="form of the X_t Y_t = I refinement on the kinetic and wide lines (ht_config.biorth_form)")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--record-counters", default=None, metavar="CSV",
                   help="write the ncu counter record of --kernel from this CSV into profiles/counters.json")
    p.add_argument("--kernel", default=None, help="kernel name for --record-counters")
    p.add_argument("--record-workload", default="", help="workload of the capture (--record-counters)")
    p.add_argument("--record-command", default="", help="the ncu command of the capture (--record-counters)")
    p.add_argument("--record-sources", default="", help="comma-separated source files of the kernel")
    p.add_argument("--record-line", default="", help="the bench line whose workload the capture ran "
                                                     "(adv6d, wide, kinetic, batched, gemm_tc, ...)")
    return p.parse_args()


# ------------------------------------------------------------------ oracle legs ----
def oracle_sample(seconds: float) -> dict:
    """Time the CPU oracle's HT + CP step on the same workload for about `seconds`."""
    import numpy as np

    from oracle import cp as OC
    from oracle import ht as OH
    from oracle.problems import advection_A
    from paper_1803_10270_gb300.inputs import advection_case, cp_padding

    case = advection_case(D, N, seed_offset=1)
    A = advection_A(case)
    u = OH.from_cp(np.ones(2), case.ic_factors())
    x = OC.CP(np.ones(2), case.ic_factors())
    pad = cp_padding([N] * D, CP_R - 2, seed=0x5EED + 1, scale=1e-3)
    steps = 0
    t0 = time.perf_counter()
    while True:
        u, _ = OH.step_rk2_poly(u, A, TOL, RMAX)
        x, _ = OC.step_rk2(x, A, CP_R, pad, SWEEPS)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 200:
            break
    return {"steps": steps, "seconds": el, "value": steps / el}


def host_cpu() -> str:
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer / part ids on
    Arm), with the machine type and core count; "unknown" parts where it says nothing."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                k, v = k.strip(), v.strip()
                if k and v and k not in fields:
                    fields[k] = v
    except OSError:
        pass
    name = fields.get("model name") or fields.get("Model") or ""
    if not name and "CPU implementer" in fields:
        name = f"implementer {fields['CPU implementer']} part {fields.get('CPU part', '?')}"
    return f"{name or 'unknown'} ({platform.machine() or 'unknown'}, {os.cpu_count()} cores)"


def oracle_sample_process(seconds: float, threads: int):
    """One oracle sample in a fresh process with its BLAS / OpenMP threads set to `threads`
    (the count the sample may use); (result dict, None) or (None, stderr tail)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--cpu-seconds", str(seconds)],
                       capture_output=True, text=True, env=env, timeout=seconds * 10 + 120)
    if r.returncode != 0:
        return None, r.stderr[-300:]
    return json.loads(r.stdout.strip().splitlines()[-1]), None


def cpu_baseline(seconds: float) -> dict:
    """Run the oracle sample in a fresh single-threaded process (BLAS pinned to 1 thread)."""
    res, err = oracle_sample_process(seconds, 1)
    if res is None:
        return {"value": None, "unit": "steps/s", "cores": 1, "kind": "oracle", "error": err}
    return {"value": res["value"], "unit": "steps/s", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{res['steps']} consecutive steps of the same workload from t=0 "
                      f"(HT + CP routes) in {res['seconds']:.1f} s, FP64 numpy, 1 thread"}


# ------------------------------------------------------------------ clocks ---------
class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        # the timed region starts once the sampler is running (its first line is written)
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < 3.0:
            try:
                if os.path.getsize(self.f.name) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU workload ---
def cp_form_name(G, ctx) -> str:
    """The form cp_als_sweep_rk2 takes for this workload's ranks on ctx."""
    q = G.cp_als_rk2_cluster_ctas(ctx, CP_R, CP_R)
    return f"thread-block cluster of {q} CTAs" if q else "cooperative grid, one CTA per factor column"


class Workload:
    def __init__(self, G, device: int, precision: int):
        import numpy as np
        import torch

        from paper_1803_10270_gb300.inputs import advection_case, cp_padding

        self.G = G
        self.case = advection_case(D, N, seed_offset=1)
        # Kronecker-sum RK2 steps raise ranks by 3: max_terms=1 sizes the workspace for that
        self.ctx = G.Context(D, [N] * D, cap=RMAX, max_terms=1, precision=precision, device=device)
        # the CP route's context (its cp_form selects the cluster or the grid form of the ALS kernel)
        self.cp_ctx = self.ctx
        self.op = G.advection_op(self.case.c, self.case.h)
        self.u = G.HTTensor(D, [N] * D, RMAX)
        self.X = G.CPTensor(D, [N] * D, CP_R)
        self.pad = cp_padding([N] * D, CP_R - 2, seed=0x5EED + 1, scale=1e-3)
        self.np = np
        self.torch = torch
        self.side = torch.cuda.Stream()
        self.ev_fork = torch.cuda.Event()
        self.ev_join = torch.cuda.Event()
        self.reset()

    def reset(self):
        np = self.np
        fac = self.case.ic_factors()
        tr = self.u.tree
        nodes = {}
        for t in range(tr.n_nodes):
            if tr.is_leaf(t):
                nodes[t] = fac[tr.lo[t]]
            elif t == 0:
                nodes[t] = np.eye(2)
            else:
                B = np.zeros((2, 2, 2))
                B[0, 0, 0] = B[1, 1, 1] = 1.0
                nodes[t] = B
        self.u.upload(nodes)
        self.X.upload(np.ones(2), fac)
        self.padded = False

    def _pad_cp(self):
        """First CP step: append the seeded padding columns (weight 1) up to rank 24."""
        np = self.np
        w, f = self.X.download()
        nw = np.linalg.norm
        # normalised columns, norms into the weights (as the oracle's pad does)
        f2, w2 = [], w.copy()
        for F in f:
            nr = nw(F, axis=0)
            f2.append(F / nr)
            w2 = w2 * nr
        self.X.upload(np.concatenate([w2, np.ones(CP_R - 2)]), [np.hstack([F, p]) for F, p in zip(f2, self.pad)])
        self.padded = True

    def step(self, stream=None):
        """HT route on the current stream, CP route on a side stream (independent data),
        forked and joined with events so the pair also captures into one CUDA graph."""
        G, torch = self.G, self.torch
        main = stream if stream is not None else torch.cuda.current_stream()
        self.ev_fork.record(main)
        self.side.wait_event(self.ev_fork)
        G.ht_step(self.ctx, self.u, self.op, self.case.dt, TOL, RMAX, stream=main)
        # CP route: ALS towards y = p(dt L) x_n with x_n as warm start (y never formed)
        G.cp_als_sweep_rk2(self.cp_ctx, self.X, self.op, self.case.dt, self.X, SWEEPS, stream=self.side)
        self.ev_join.record(self.side)
        main.wait_event(self.ev_join)

    def step_route(self, route: str, stream=None):
        """One route alone on the given stream ("ht" or "cp"), for the per-route timings."""
        G = self.G
        if route == "ht":
            G.ht_step(self.ctx, self.u, self.op, self.case.dt, TOL, RMAX, stream=stream)
        else:
            G.cp_als_sweep_rk2(self.cp_ctx, self.X, self.op, self.case.dt, self.X, SWEEPS, stream=stream)

    def first_step(self):
        """Step 1: the rank-2 state defines y; the iterate is that state padded to rank 24."""
        G = self.G
        G.ht_step(self.ctx, self.u, self.op, self.case.dt, TOL, RMAX)
        self._pad_cp()
        X2 = G.CPTensor(D, [N] * D, 2)
        w, f = self.X.download()
        X2.upload(w[:2], [F[:, :2] for F in f])
        G.cp_als_sweep_rk2(self.cp_ctx, X2, self.op, self.case.dt, self.X, SWEEPS)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_1803_10270_gb300 import build as B
    from paper_1803_10270_gb300 import htgpu as G
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    G.load()
    prec = G.HT_PREC_FP64 if args.precision == "fp64" else G.HT_PREC_MIXED
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2
    if args.line != "all":
        warm = max(args.warmup, 3)
        if args.line == "mixed":
            res = run_mixed_lines(G, torch, flush, args)
        elif args.line == "d12":
            res = run_d12(G, torch, flush, args.steps, warm, precision=prec)
        elif args.line == "ab2":
            res = run_ab2_all(G, torch, flush, args.steps, warm)
        elif args.line == "varcoef":
            res = run_varcoef(G, torch, flush, args.steps, warm)
        elif args.line == "tt":
            res = run_tt(G, torch, flush, args.steps, warm)
        elif args.line == "cn":
            res = run_cn(G, torch, flush, args.steps, warm)
        elif args.line == "kinetic":
            res = run_kinetic(G, torch, flush, args.steps, warm, precision=prec,
                              biorth_form=BIORTH_FORMS[args.biorth_form])
        elif args.line == "wide":
            res = run_wide(G, torch, flush, args.steps, warm, precision=prec,
                           biorth_form=BIORTH_FORMS[args.biorth_form])
        elif args.line == "gemm_tc":
            res = run_gemm_probe(G, args)
        else:
            res = run_batched(G, torch, flush, args.batched, args.steps, warm, precision=prec)
        if rank == 0:
            print(json.dumps({"line": args.line, **res}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return
    # ---- autotuner (launch parameters measured on this GPU, cached for every context below)
    tuning = run_tuner(local) if args.tune else None
    W = Workload(G, local, prec)
    stream = torch.cuda.current_stream()

    # warm-up (the first step pads the CP iterate to its target rank)
    W.first_step()
    for _ in range(max(args.warmup - 1, 0)):
        W.step()
    torch.cuda.synchronize()
    W.ctx.check()

    # ---- one step captured as a CUDA graph (ranks live on the device, no host sync inside)
    graph = None
    per_step_launches = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        l0 = W.ctx.launches()
        with torch.cuda.graph(graph):
            W.step()
        per_step_launches = W.ctx.launches() - l0
        torch.cuda.synchronize()
        graph.replay()          # one more warm-up step through the graph
        torch.cuda.synchronize()

    # ---- timed region: device-resident inputs, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = W.ctx.launches()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        if graph is not None:
            graph.replay()
        else:
            W.step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = (W.ctx.launches() - l0) if graph is None else per_step_launches * args.steps
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    W.ctx.check()
    ms_max, value = aggregate_replicas(ms, args.steps)

    # ---- roofline: per-kernel-class CUDA-event time on the launching stream over a second
    #      timed region (same steps, L2 flushed, no graph so each launch can be bracketed)
    # the passes below replay the same stretch of the run as the timed region (the step
    # cost changes as the solution's ranks evolve): restart from t = 0 before each
    def restart():
        W.reset()
        W.first_step()
        for _ in range(max(args.warmup - 1, 0)):
            W.step()
        torch.cuda.synchronize()

    restart()
    roof, shares = profile_pass(W, torch, flush, args.steps)

    # ---- e2e: state from pinned host memory each step, result back to the host
    restart()
    e2e = run_e2e(W, G, torch, args.steps)
    ranks = W.u.ranks()

    # ---- each route alone (same steps from t = 0, graph-captured, L2 flushed): the HT route's
    #      steps/s is the metric's own reading; the combined step above runs both side by side
    routes = {}
    grid_ctx = G.Context(D, [N] * D, cap=RMAX, max_terms=1, precision=prec, device=local, cp_form=G.CP_FORM_GRID)
    for route in ("ht", "cp", "cp_grid"):
        # cp_grid: the CP route in the cooperative grid form (one CTA per factor column), for
        # comparison with the cluster form the step uses
        W.cp_ctx = grid_ctx if route == "cp_grid" else W.ctx
        restart()
        g1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1):
            W.step_route(route[:2], stream=torch.cuda.current_stream())
        evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            evr[i][0].record(stream)
            g1.replay()
            evr[i][1].record(stream)
        torch.cuda.synchronize()
        W.ctx.check()
        W.cp_ctx.check()
        msr = sum(a.elapsed_time(b) for a, b in evr)
        msr_max, vr = aggregate_replicas(msr, args.steps)
        routes[route] = {"value": vr, "unit": "steps/s", "ms_per_step": msr_max / args.steps}
        del g1
    W.cp_ctx = W.ctx
    grid_ctx.close()
    routes["cp"]["form"] = cp_form_name(G, W.ctx)
    routes["cp_grid"]["form"] = "cooperative grid, one CTA per factor column"

    # ---- the paper's two-step scheme (eq. AB2_) on the same HT workload, HT route alone
    ab2 = run_ab2_all(G, torch, flush, args.steps, args.warmup)

    # ---- FP64 against the tensor-core form: the HT route of this workload, the 12-D workload
    #      (100 RK2 steps), the full-size kinetic workload and the ragged batch, each in both forms
    #      from the same initial state; the FP64 halves are the d12 / kinetic / batched lines
    mixed = run_mixed_lines(G, torch, flush, args) if args.d12 else None
    d12 = mixed["d12"]["fp64"] if mixed else None

    # ---- the same HT workload in tensor-train form (linear dimension tree)
    tt = run_tt(G, torch, flush, args.steps, max(args.warmup, 3)) if args.d12 else None

    # ---- the full-size kinetic workload, HEUN2, steps 46-50 (timed in run_mixed_lines)
    kinetic = mixed["kinetic"]["fp64"] if mixed else None

    # ---- implicit Crank-Nicolson step in CP format (ALS), kinetic operator
    cn = run_cn(G, torch, flush, 50, max(args.warmup, 3)) if args.d12 else None

    # ---- variable-coefficient advection (eq. PDE-advR) on the paper's 2-D grid, HEUN2
    varcoef = run_varcoef(G, torch, flush, 100, max(args.warmup, 3)) if args.d12 else None

    # ---- ragged batch of independent instances (ht_batch_step), its own throughput line (timed
    #      in run_mixed_lines when that ran)
    if mixed and "batched" in mixed:
        batched = mixed["batched"]["fp64"]
    else:
        batched = run_batched(G, torch, flush, args.batched, min(args.steps, 20), max(args.warmup, 3)) \
            if args.batched > 0 else None

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic (seeded 6-D advection, n=64)",
            "config": config_keys(args.precision, "flushed between timed steps (256 MB write)",
                                  "replicas" if world > 1 else "single GPU"),
            "run": {"ht_ranks_final": ranks, "streams": "HT route and CP route on two streams (independent data)",
                    "cuda_graph": graph is not None, "cp_form": cp_form_name(G, W.ctx)},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "roofline": roof, "kernel_shares": shares,
        }
        out["routes_alone"] = routes
        out["ab2"] = ab2
        if d12 is not None:
            out["d12"] = d12
        if varcoef is not None:
            out["varcoef"] = varcoef
        if tt is not None:
            out["tt"] = tt
        if cn is not None:
            out["cn"] = cn
        if kinetic is not None:
            out["kinetic"] = kinetic
        if tuning is not None:
            out["tuning"] = tuning
            out["tuning"]["tuned_vs_default"] = tuned_vs_default(G, torch, flush)
        if mixed is not None:
            out["mixed"] = {k: {kk: vv for kk, vv in v.items() if kk != "fp64"} for k, v in mixed.items()}
            for k, v in out["mixed"].items():
                v["fp64_value"] = mixed[k]["fp64"]["value"]
        if batched is not None:
            out["batched"] = batched
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_gemm_probe(G, args) -> dict:
    """One synthetic contraction (op(A) m x k times op(B) k x n, --gemm-shape m,n,k) through the
    tensor-core split kernel and the FP64 kernel: mean times and the tensor kernel's executed MMA
    rate (the small case the profiler captures of gemm_tc_kernel)."""
    m, n, k = (int(x) for x in args.gemm_shape.split(","))
    reps = max(args.steps, 1)
    ttc = G.tune_time_gemm(m, n, k, 1, 1, 4, 16, reps)
    t64 = G.tune_time_gemm(m, n, k, 1, 0, 4, 16, reps)
    tiles = -(-m // 128) * -(-n // 128)
    executed = 10 * 2.0 * 128 * 128 * (32 * -(-k // 32)) * tiles
    pk = measured_peaks().get("bf16_tflops") or 1900.0
    return {"workload": f"contraction {m} x {k} times {k} x {n}, FP64 in and out", "tc_ms": ttc, "fp64_ms": t64,
            "speedup": t64 / ttc, "tc_executed_tflops": executed / (ttc * 1e-3) / 1e12,
            "tc_frac_of_bf16_burst": executed / (ttc * 1e-3) / 1e12 / pk, "slices": 4, "reps": reps}


def run_tuner(device: int) -> dict:
    """The package's autotuner (paper_1803_10270_gb300.tune): measured values, written to its cache."""
    from paper_1803_10270_gb300 import tune
    res = tune.tune(device, write=True)
    return {k: res[k] for k in ("tc_min_work", "gemm_ctas_per_sm_by_kc", "svd_cluster_min_cols", "seconds")}


def tuned_vs_default(G, torch, flush) -> dict:
    """The kinetic line (both forms) and the 12-D line with the library defaults (tuning={}) beside
    the tuned values (the cache the autotuner wrote)."""
    out = {}
    for name, fn, kw in (("kinetic_fp64", run_kinetic, dict(steps=5, warmup=3, precision=0)),
                         ("kinetic_mixed", run_kinetic, dict(steps=5, warmup=3, precision=1, slices=4)),
                         ("d12_fp64", run_d12, dict(steps=50, warmup=3))):
        d = fn(G, torch, flush, tuning={}, profile=False, **kw)["value"]
        t = fn(G, torch, flush, tuning=None, profile=False, **kw)["value"]
        out[name] = {"default": d, "tuned": t, "unit": "steps/s", "speedup": t / d}
    return out


WIDE_WORKLOAD = ("HSVD truncation of a random d=4 HT tensor, n=200, every rank 192, transfer tensors graded "
                 "by 0.9^j (node factors 192 columns wide: cluster SVD; interior matrices 36864 x 192: "
                 "cooperative QR), tol 1e-8")


def run_wide(G, torch, flush, steps: int, warmup: int, precision: int = 0, slices: int = 0,
             biorth_form: int = 0) -> dict:
    """Truncations per second of one wide-factor case (the shape class of the kinetic workload's
    node factors at a size a profiler capture can hold), graph-captured, L2 flushed between."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import normal_arrays
    d, n, w = 4, 200, 192
    u = G.HTTensor(d, [n] * d, w)
    tr = u.tree
    shapes = [(n, w) if tr.is_leaf(t) else ((w, w) if t == 0 else (w, w, w)) for t in range(tr.n_nodes)]
    arrs = normal_arrays(shapes, 0x5EED + 7)
    g = 0.9 ** np.arange(w)
    u.upload({t: (arrs[t] * g.reshape((1,) * (arrs[t].ndim - 1) + (-1,)) if t else arrs[t])
              for t in range(tr.n_nodes)})
    ctx = G.Context(d, [n] * d, cap=w // 3, max_terms=1, precision=precision, mixed_slices=slices,
                    biorth_form=biorth_form)
    out = G.HTTensor(d, [n] * d, w)
    for _ in range(warmup):
        G.ht_truncate(ctx, u, TOL, w, out)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        G.ht_truncate(ctx, u, TOL, w, out, stream=torch.cuda.current_stream())
    per = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    ranks = out.ranks()
    ctx_bi = ctx.biorth_cluster_ctas()
    del graph
    ctx.close()
    return {"workload": WIDE_WORKLOAD, "value": value, "unit": "truncations/s", "ms_per_step": ms_max / steps,
            "steps": steps, "warmup": warmup, "gpu_launches_per_step": per, "ranks_out": ranks,
            "precision": precision_name(precision, slices), "cuda_graph": True,
            "biorth_form": "cluster" if ctx_bi else "cta"}


def run_mixed_lines(G, torch, flush, args) -> dict:
    """Each line in the FP64 and the mixed (tensor-core) form: steps/s, speedup and the relative
    difference of the final states."""
    warm = max(args.warmup, 3)
    out = {"adv6d_ht": mixed_vs_fp64(G, torch, flush, run_d12, steps=args.steps, warmup=warm, d=D, n=N, cap=RMAX,
                                     n_terms=2, seed_offset=1, workload=ADV_HT_WORKLOAD, line="adv6d"),
           "d12": mixed_vs_fp64(G, torch, flush, run_d12, steps=100, warmup=warm),
           "kinetic": mixed_vs_fp64(G, torch, flush, run_kinetic, steps=5, warmup=45)}
    if args.batched > 0:
        out["batched"] = mixed_vs_fp64(G, torch, flush, run_batched, count=args.batched,
                                       steps=min(args.steps, 20), warmup=warm)
    return out


ADV_HT_WORKLOAD = ("6-D advection n=64 HT route alone: r_max 32, tol 1e-8, RK2 dt=0.2h (the headline "
                   "workload's HT half)")


BATCH_WORKLOAD = ("ragged batch: independent 6-D advection instances, n in {32,48,64,96,128}, "
                  "HT r_max in 8..48, seeded velocities, RK2 dt=0.2h, tol 1e-8; "
                  "one step = every instance's HT apply+HSVD truncate, each launch covering all instances")


def ic_nodes(tree, fac, np):
    """Exact rank-R HT form of an R-term separable initial condition (fac[i] is n x R)."""
    R = fac[0].shape[1]
    nodes = {}
    for t in range(tree.n_nodes):
        if tree.is_leaf(t):
            nodes[t] = fac[tree.lo[t]]
        elif t == 0:
            nodes[t] = np.eye(R)
        else:
            B = np.zeros((R, R, R))
            for m in range(R):
                B[m, m, m] = 1.0
            nodes[t] = B
    return nodes


def run_ab2_all(G, torch, flush, steps: int, warmup: int) -> dict:
    """The AB2 line: the exact-sum step (ht_step_ab2) and the two split evaluations of Section 3.2
    (ht_step_ab2_split), each timed; the cancellation study is the relative distance of each split
    result from the exact-sum result after the same steps (on the device, HT inner products)."""
    res, c0, s0 = run_ab2(G, torch, flush, steps, warmup, keep=True)
    res["split"] = {}
    for variant, name in ((0, "argument"), (1, "difference")):
        r, c, sv = run_ab2(G, torch, flush, steps, warmup, variant=variant, keep=True)
        r["rel_dist_from_exact_sum_final"] = ht_rel_diff(G, torch, c0, sv, s0)
        res["split"][name] = r
        c.close()
    c0.close()
    return res


def run_ab2(G, torch, flush, steps: int, warmup: int, variant: int | None = None, keep: bool = False):
    """HT steps/s of the AB2 scheme on the configuration-2 advection workload (ht_step_ab2, or
    ht_step_ab2_split with `variant`): an RK2 start step, then AB2 steps, the timed ones
    graph-captured with L2 flushed between them.  keep: also return the context and the state."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import advection_case
    case = advection_case(D, N, seed_offset=1)
    ctx = G.Context(D, [N] * D, cap=RMAX, max_terms=2)
    u = G.HTTensor(D, [N] * D, RMAX)
    up = G.HTTensor(D, [N] * D, RMAX)
    nodes = ic_nodes(u.tree, case.ic_factors(), np)
    u.upload(nodes)
    up.upload(nodes)
    op = G.advection_op(case.c, case.h)
    def ab2(stream=None):
        if variant is None:
            G.ht_step_ab2(ctx, u, up, op, case.dt, TOL, RMAX, stream=stream)
        else:
            G.ht_step_ab2_split(ctx, u, up, op, case.dt, TOL, RMAX, variant, stream=stream)

    G.ht_step(ctx, u, op, case.dt, TOL, RMAX)       # u_1; u_prev = u_0
    for _ in range(max(warmup - 1, 0)):
        ab2()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        ab2(stream=torch.cuda.current_stream())
    per_step = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    ranks = u.ranks()
    del graph
    res = {"workload": "6-D advection n=64 HT route, AB2 (eq. AB2_) after one RK2 start step, "
                       "r_max 32, tol 1e-8", "value": value, "unit": "steps/s", "ms_per_step": ms_max / steps,
           "steps": steps, "ht_ranks_final": ranks, "cuda_graph": True, "gpu_launches_per_step": per_step,
           "form": "exact sum, one truncation" if variant is None else
                   ("split: w = T(3u - u_prev), v = T(dt L w), T(u + v/2)" if variant == 0 else
                    "split: w = T(u - u_prev), T(u + T(dt L u) + T(dt L w)/2)")}
    if keep:
        return res, ctx, u
    ctx.close()
    return res


D12_WORKLOAD = ("12-D advection n=128: depth-4 tree, seeded separable rank-3 initial condition, "
                "HT r_max 64, tol 1e-8, RK2 dt=0.2h")


TT_WORKLOAD = ("6-D advection n=64 HT route in tensor-train form (the linear dimension tree, "
               "Section 2.2), r_max 32, tol 1e-8, RK2 dt=0.2h, FP64")


def run_d12(G, torch, flush, steps: int, warmup: int, d: int = 12, n: int = 128, cap: int = 64,
            n_terms: int = 3, seed_offset: int = 4, tree: int = 0, workload: str = None, precision: int = 0,
            slices: int = 0, keep: bool = False, profile: bool = True, tuning: dict | None = None,
            line: str = "d12"):
    """HT steps/s of the RK2 step on the 12-D advection workload (n = 128 per dimension, r_max
    64), or another advection workload and tree: the timed steps graph-captured, L2 flushed
    between them; then a profiled stretch of the same length for the per-class roofline.  keep:
    also return the context and the final state (steps warmup + steps, before the profiled
    stretch) for a comparison between precision forms."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import advection_case
    case = advection_case(d, n, n_terms=n_terms, seed_offset=seed_offset)
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1, tree=tree, precision=precision, mixed_slices=slices,
                    tuning=tuning)
    u = G.HTTensor(d, [n] * d, cap, tree=tree)
    u.upload(ic_nodes(u.tree, case.ic_factors(), np))
    op = G.advection_op(case.c, case.h)
    for _ in range(warmup):
        G.ht_step(ctx, u, op, case.dt, TOL, cap)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        G.ht_step(ctx, u, op, case.dt, TOL, cap, stream=torch.cuda.current_stream())
    per_step = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    ranks = u.ranks()
    del graph
    res = {"workload": workload or D12_WORKLOAD, "value": value, "unit": "steps/s", "ms_per_step": ms_max / steps,
           "steps": steps, "warmup": warmup, "gpu_launches_per_step": per_step,
           "ht_ranks_final": ranks, "cuda_graph": True, "precision": precision_name(precision, slices)}
    snap = None
    if keep:
        snap = G.HTTensor(d, [n] * d, cap, tree=tree)
        snap.blob.copy_(u.blob)
        snap.rank_buf.copy_(u.rank_buf)
    if profile:
        pst = min(steps, 10)
        prof = profiled_steps(ctx, torch, flush, lambda: G.ht_step(ctx, u, op, case.dt, TOL, cap), pst)
        res["roofline"], res["kernel_shares"] = class_roofline(prof, pst, ctx, line)
    if keep:
        return res, ctx, snap
    ctx.close()
    return res


VC_WORKLOAD = ("variable-coefficient advection f_t + (C z).grad f = 0 (eq. PDE-advR), N=2 on the paper's "
               "grid: [-60,60)^2 with 600 nodes per variable, seeded C (eigenvalue real parts in [0.5,1]), "
               "f0 = exp(-|z|^2), 4-term operator of Table tab:ordering0, HEUN2 (truncation after each "
               "stage), HT r_max 12, tol 1e-8, dt = 0.2 h / max speed, FP64")


CN_WORKLOAD = ("linearised 6-D kinetic equation (its 5 separable terms), n=16 per variable, "
               "Crank-Nicolson step solved in CP format by ALS (eqs. CNFDE, ALS2, ML, MR): CP rank 6 "
               "(seeded kinetic initial condition), 5 Gauss-Seidel sweeps per step, dt = 5x the explicit "
               "step, FP64")


def run_cn(G, torch, flush, steps: int, warmup: int) -> dict:
    """Implicit steps/s: each step copies x into x_n (the previous level and the initial guess)
    and runs cp_cn_als_step; graph-captured, L2 flushed between steps."""
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    n, sweeps = 16, 5
    kc = kinetic_case(n)
    w0, F0 = kinetic_ic(kc)
    r = len(w0)
    ctx = G.Context(6, [n] * 6, cap=r, max_terms=5)
    kop = G.KineticOp(kc)
    x = G.CPTensor(6, [n] * 6, r)
    xn = G.CPTensor(6, [n] * 6, r)
    x.upload(w0, F0)
    xn.upload(w0, F0)
    dt = 5 * kc.dt

    def step(stream=None):
        xn.blob.copy_(x.blob)
        G.cp_cn_als_step(ctx, xn, kop.op, dt, x, sweeps, stream=stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.check()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        step(stream=torch.cuda.current_stream())
    per_step = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    del graph
    ctx.close()
    return {"workload": CN_WORKLOAD, "value": value, "unit": "steps/s", "ms_per_step": ms_max / steps,
            "steps": steps, "warmup": warmup, "gpu_launches_per_step": per_step, "cp_rank": r, "sweeps": sweeps,
            "cuda_graph": True}


KIN_WORKLOAD = ("linearised 6-D kinetic equation: n=64 per variable, x periodic [0,2pi)^3, v in [-6,6]^3, "
                "nu=1, seeded initial condition M(v)(1 + 0.1 prod sin x_i) + rank-4 perturbation, 5-term operator, "
                "HEUN2 (truncation after each stage), HT r_max 64, tol 1e-6; steps W+1..W+K from t=0 (W warm-up steps)")


def run_kinetic(G, torch, flush, steps: int, warmup: int, precision: int = 0, slices: int = 0,
                keep: bool = False, profile: bool = True, tuning: dict | None = None, biorth_form: int = 0):
    """HT HEUN2 steps/s of the full-size kinetic workload (node ranks grow to about 60 within ten
    steps, so the step cost grows too: the line reports steps warmup+1 .. warmup+steps); then a
    profiled stretch for the per-class roofline; keep as in run_d12."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(64)
    w0, F0 = kinetic_ic(kc)
    ctx = G.Context(6, [64] * 6, cap=64, max_terms=5, precision=precision, mixed_slices=slices, tuning=tuning,
                    biorth_form=biorth_form)
    u = G.HTTensor(6, [64] * 6, 64)
    u.upload(ic_nodes(u.tree, [F * (w0[None, :] if i == 0 else 1.0) for i, F in enumerate(F0)], np))
    kop = G.KineticOp(kc)
    for _ in range(warmup):
        G.ht_step(ctx, u, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2)
    torch.cuda.synchronize()
    ctx.check()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        G.ht_step(ctx, u, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2, stream=torch.cuda.current_stream())
    per_step = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    ranks = u.ranks()
    del graph
    res = {"workload": KIN_WORKLOAD, "value": value, "unit": "steps/s", "ms_per_step": ms_max / steps,
           "steps": steps, "warmup": warmup, "gpu_launches_per_step": per_step, "ht_ranks_final": ranks,
           "cuda_graph": True, "precision": precision_name(precision, slices),
           "biorth_form": "cluster" if ctx.biorth_cluster_ctas() else "cta"}
    snap = None
    if keep:
        snap = G.HTTensor(6, [64] * 6, 64)
        snap.blob.copy_(u.blob)
        snap.rank_buf.copy_(u.rank_buf)
    if profile:
        pst = min(steps, 2)
        prof = profiled_steps(ctx, torch, flush,
                              lambda: G.ht_step(ctx, u, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2), pst)
        res["roofline"], res["kernel_shares"] = class_roofline(prof, pst, ctx, "kinetic")
    if keep:
        return res, ctx, snap
    ctx.close()
    return res


def run_tt(G, torch, flush, steps: int, warmup: int) -> dict:
    """The configuration-2 HT route on the linear (tensor-train) tree."""
    return run_d12(G, torch, flush, steps, warmup, d=D, n=N, cap=RMAX, n_terms=2, seed_offset=1, tree=1,
                   workload=TT_WORKLOAD, line="tt")


def run_varcoef(G, torch, flush, steps: int, warmup: int) -> dict:
    """HT steps/s of HEUN2 with the 4-term variable-coefficient operator on the paper's 2-D grid;
    graph-captured, L2 flushed between steps.  Also the paper's accuracy measure: the relative
    pointwise error at the grid point nearest z* = (0.6988.., 0.6988..) against the
    characteristic solution f0(exp(-tC) z) at the final time (outside the timed region)."""
    import numpy as np
    from scipy.linalg import expm
    from paper_1803_10270_gb300.inputs import varcoef_case
    N, n, cap = 2, 600, 12
    case = varcoef_case(N, n)
    ctx = G.Context(N, [n] * N, cap=cap, max_terms=N * N)
    u = G.HTTensor(N, [n] * N, cap)
    u.upload(ic_nodes(u.tree, case.ic_factors(), np))
    vop = G.VarCoefOp(case)
    for _ in range(warmup):
        G.ht_step(ctx, u, vop.op, case.dt, TOL, cap, scheme=G.HT_SCHEME_HEUN2)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    graph = torch.cuda.CUDAGraph()
    l0 = ctx.launches()
    with torch.cuda.graph(graph):
        G.ht_step(ctx, u, vop.op, case.dt, TOL, cap, scheme=G.HT_SCHEME_HEUN2,
                  stream=torch.cuda.current_stream())
    per_step = ctx.launches() - l0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max, value = aggregate_replicas(ms, steps)
    ranks = u.ranks()
    nodes = u.download()
    del graph
    ctx.close()
    t_end = (warmup + steps) * case.dt
    i = case.star_index()
    a, b = u.tree.c1[0], u.tree.c2[0]          # the two leaves (z_1, z_2) of the 2-D tree
    f_num = float(nodes[a][i, :] @ nodes[0] @ nodes[b][i, :])
    zp = np.array([case.z()[i]] * N)
    y = expm(-t_end * case.C) @ zp
    f_ex = float(np.exp(-(y @ y)))
    return {"workload": VC_WORKLOAD, "value": value, "unit": "steps/s", "ms_per_step": ms_max / steps,
            "steps": steps, "warmup": warmup, "gpu_launches_per_step": per_step, "ht_ranks_final": ranks,
            "t_end": t_end, "pointwise_rel_err_at_z_star": abs(f_num - f_ex) / f_ex, "cuda_graph": True}


def run_batched(G, torch, flush, count: int, steps: int, warmup: int, precision: int = 0, slices: int = 0,
                keep: bool = False, profile: bool = True):
    """Throughput of ht_batch_step on a ragged batch: instance-steps/s over a graph-captured
    step, L2 flushed between timed steps, slowest rank's time for replicas; then a profiled
    stretch (the classes of the first instance's context carry the batch's launches); keep:
    also return the contexts and the final states."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import batched_advection_cases
    cases = batched_advection_cases(count, D)
    ctxs, tens, ops = [], [], []
    ws = 0
    for n, rmax, case in cases:
        c = G.Context(D, [n] * D, cap=rmax, max_terms=1, precision=precision, mixed_slices=slices)
        ws += c.workspace_bytes
        t = G.HTTensor(D, [n] * D, rmax)
        t.upload(ic_nodes(t.tree, case.ic_factors(), np))
        ctxs.append(c)
        tens.append(t)
        ops.append(G.advection_op(case.c, case.h))
    b = G.Batch(ctxs, tens)
    dts = [case.dt for _, _, case in cases]
    tols = [TOL] * count
    rmaxs = [r for _, r, _ in cases]
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        b.step(ops, dts, tols, rmaxs, stream=stream)
    torch.cuda.synchronize()
    l0 = ctxs[0].launches()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.step(ops, dts, tols, rmaxs, stream=torch.cuda.current_stream())
    per_step = ctxs[0].launches() - l0
    graph.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(x) for a, x in ev)
    for c in ctxs:
        c.check()
    ms_max, steps_per_s = aggregate_replicas(ms, steps)
    rk = [max(t.ranks()[1:]) for t in tens]
    ns = [n for n, _, _ in cases]
    del graph
    res = {"workload": BATCH_WORKLOAD, "instances": count, "value": steps_per_s * count,
           "unit": "instance-steps/s", "ms_per_step": ms_max / steps, "steps": steps, "warmup": warmup,
           "gpu_launches_per_step": per_step, "grids": {str(v): ns.count(v) for v in sorted(set(ns))},
           "rank_max_final": max(rk), "rank_mean_final": sum(rk) / len(rk),
           "workspace_gb": ws / 1e9, "l2": "flushed between timed steps (256 MB write)", "cuda_graph": True,
           "precision": precision_name(precision, slices)}
    snaps = None
    if keep:
        snaps = []
        for (n, rmax, _), t in zip(cases, tens):
            sn = G.HTTensor(D, [n] * D, rmax)
            sn.blob.copy_(t.blob)
            sn.rank_buf.copy_(t.rank_buf)
            snaps.append(sn)
    if profile:
        pst = min(steps, 5)
        prof = profiled_steps(ctxs[0], torch, flush, lambda: b.step(ops, dts, tols, rmaxs, stream=stream), pst)
        res["roofline"], res["kernel_shares"] = class_roofline(prof, pst, ctxs[0], "batched")
    b.close()
    if keep:
        return res, ctxs, snaps
    for c in ctxs:
        c.close()
    return res


def precision_name(precision: int, slices: int) -> str:
    return "fp64" if precision == 0 else f"mixed ({slices or 4} BF16 digit planes per operand, FP32 accumulation)"


def mixed_vs_fp64(G, torch, flush, fn, **kw) -> dict:
    """One line in both precision forms from the same initial state and for the same steps:
    steps/s of each, their ratio and the relative difference of the final states (the FP64 GPU
    form is within 1e-10 of the oracle, tests/test_gpu_workloads.py)."""
    r64, c64, s64 = fn(G, torch, flush, precision=0, keep=True, **kw)
    if isinstance(c64, list):     # a batch: free the FP64 workspaces before the mixed run
        for c in c64:
            c.close()
    rmx, cmx, smx = fn(G, torch, flush, precision=1, slices=4, keep=True, **kw)
    if isinstance(cmx, list):     # per instance, each against its FP64 twin
        err = max(ht_rel_diff(G, torch, c, a, b) for c, a, b in zip(cmx, smx, s64))
        for c in cmx:
            c.close()
    else:
        err = ht_rel_diff(G, torch, c64, smx, s64)
        c64.close()
        cmx.close()
    return {"workload": r64["workload"], "fp64": r64, "mixed": rmx, "speedup": rmx["value"] / r64["value"],
            "rel_err_vs_fp64_final": err,
            "steps_compared": r64["steps"] + r64["warmup"]}


def aggregate_replicas(ms_local: float, steps: int):
    """Replicas (one independent copy of the workload per rank, no data-path collective):
    the job time is the slowest rank's, the throughput counts every rank's steps."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    t = torch.tensor([ms_local], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t[0])
    return ms_max, world * steps / (ms_max * 1e-3)


def ht_rel_diff(G, torch, ctx, a, b, tree: int = 0) -> float:
    """|a - b| / |b| on the device: the difference formed exactly (ht_add, ranks adding) and its
    norm taken from the orthogonalised form of the truncation (ht_truncate's norm output, QR based,
    so no cancellation between the two states' O(|u|) parts); |b| from <b, b>."""
    diff = G.HTTensor(a.d, a.n, a.cap + b.cap, tree=tree)
    G.ht_add(ctx, 1.0, a, -1.0, b, diff)
    out = G.HTTensor(a.d, a.n, 1, tree=tree)
    v = torch.zeros(2, dtype=torch.float64, device="cuda")
    G.ht_truncate(ctx, diff, 0.0, 1, out, norm=v[0:1])
    G.ht_inner(ctx, b, b, v[1:2])
    nd, bb = (float(x) for x in v.cpu())
    return nd / math.sqrt(bb) if bb > 0 else float("nan")


def measured_peaks() -> dict:
    """MEASURED_PEAKS.json of the GPU pool (copy bandwidth, cuBLAS bf16 burst and sustained)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def class_roofline(prof: dict, steps: int, ctx=None, line: str | None = None) -> tuple:
    """Per-class shares of one profiled stretch, and the roofline of its dominant class: the
    FP64 classes against the FP64 peak ("alu"), the tensor-core contractions against the
    measured sustained BF16 tensor peak ("tensor", executed MMA flops); in a mixed-form context
    (ctx.cfg.precision) the gemm class is the split-FP32 kernel, against its FP32-pipe bound.
    `traffic` comes from a committed counter record of the class's kernel taken on this line's
    workload (`line`), else it is null: another workload's DRAM bytes say nothing of this one's."""
    split = ctx is not None and ctx.cfg.precision == HT_PREC_MIXED
    total = sum(v["ms"] for v in prof.values()) or 1.0
    shares = {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] / steps,
                  "share": v["ms"] / total,
                  "counted_tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12) if v["ms"] > 0 and v["flops"] > 0 else None}
              for k, v in prof.items() if v["launches"]}
    dom = max(prof, key=lambda k: prof[k]["ms"])
    roof = roofline_of(prof, dom, steps, split, line)
    out = {"dominant": roof}
    if dom != "gemm_tc" and prof.get("gemm_tc", {}).get("launches"):
        out["gemm_tc"] = roofline_of(prof, "gemm_tc", steps, line=line)
    return out, shares


def roofline_of(prof: dict, cls: str, steps: int, split: bool = False, line: str | None = None) -> dict:
    v = prof[cls]
    if cls == "gemm" and split:
        roof = {"kernel": "gemm_f32x2_kernel", "class": cls, "bound": "alu", "unit": "TFLOP/s",
                "peak": F32X2_PEAK_TFLOPS,
                "peak_source": "FP32 pipe (152 SMs x 2.07 GHz x 128 lanes) / 10 FP32 ops per FP64 multiply-add",
                "flops": "FP64-equivalent flops of the contractions (2 m n k)"}
    elif cls == "gemm_tc":
        pk = measured_peaks()
        peak = pk.get("bf16_tflops_sustained") or 1700.0
        roof = {"kernel": "gemm_tc_kernel", "class": cls, "bound": "tensor", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "bf16_tflops_sustained of MEASURED_PEAKS.json" if pk else "fallback 1.7 PFLOP/s",
                "flops": "executed BF16 MMA flops (digit-pair products over whole 128 x 128 tiles)"}
    else:
        roof = {"kernel": KERNEL_NAMES.get(cls, cls), "class": cls, "bound": "alu", "unit": "TFLOP/s",
                "peak": FP64_PEAK_TFLOPS, "peak_source": "FP64 nominal (152 SMs x 2.07 GHz x 4 flop/clk/SM)",
                "flops": "FP64 flops the kernel counts"}
    roof.update({"achieved": None, "frac": None, "traffic": None, "avg_launch_us": None, "steps": steps})
    if v["launches"]:
        per_launch_s = v["ms"] * 1e-3 / v["launches"]
        roof["avg_launch_us"] = per_launch_s * 1e6
        if v["flops"] > 0:
            ach = v["flops"] / v["launches"] / per_launch_s / 1e12
            roof["achieved"] = ach
            roof["frac"] = ach / roof["peak"]
            roof["flops_per_launch"] = v["flops"] / v["launches"]
    attach_traffic(roof, roof["kernel"].split("/"), line)
    return roof


def attach_traffic(roof: dict, kernels, line: str | None) -> None:
    """roof["traffic"] (DRAM bytes per launch) from the first of `kernels` whose committed counter
    record is fresh and was taken on the workload of `line`; null when none is."""
    roof["traffic"] = None
    roof.pop("traffic_record", None)
    for kern in kernels:
        rec = counter_record(kern)
        if rec is None or rec.get("stale") or line is None or rec.get("line") != line:
            continue
        roof["traffic"] = rec.get("dram_bytes_per_launch")
        roof["traffic_record"] = {k: rec[k] for k in ("kernel", "workload", "when") if k in rec}
        return


def profiled_steps(ctx, torch, flush, step, steps: int) -> dict:
    """Per-class CUDA-event times of `steps` launches of step() (no graph, L2 flushed)."""
    ctx.profile(True)
    for _ in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    return prof


COUNTERS = os.path.join(ROOT, "profiles", "counters.json")
# the ncu metrics a counter record keeps (dram bytes give roofline.traffic)
RECORD_METRICS = ("gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
                  "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
                  "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active",
                  "sm__cycles_active.avg", "sm__cycles_elapsed.avg", "launch__grid_size",
                  "launch__registers_per_thread", "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed")
_UNIT = {"byte": 1, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "ns": 1e-3, "us": 1.0, "usecond": 1.0,
         "msecond": 1e3, "ms": 1e3, "nsecond": 1e-3}


def _sha256(path: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def counter_record(kernel: str):
    """The committed ncu counter record of a kernel (profiles/counters.json, written by
    --record-counters), or None.  A record whose kernel sources changed since the capture (their
    SHA-256 differs from the one recorded) is returned with stale = True and no byte count."""
    try:
        with open(COUNTERS) as f:
            recs = json.load(f).get("records", [])
    except (OSError, ValueError):
        return None
    for r in recs:
        if r.get("kernel") != kernel:
            continue
        try:
            fresh = all(_sha256(p) == h for p, h in r.get("sources", {}).items())
        except OSError:
            fresh = False
        if not fresh:
            return {"stale": True, "workload": r.get("workload"), "when": r.get("when")}
        return r
    return None


def parse_ncu_csv(path: str, kernel: str) -> list:
    """Launches of `kernel` in an ncu CSV: the raw page (`ncu -i rep --page raw --csv`, one row per
    launch, a units row under the header) or a --metrics --csv log (one row per metric).  Values
    in bytes / microseconds / plain numbers."""
    import csv
    with open(path, newline="") as f:
        rows = [r for r in csv.reader(f) if r and not r[0].startswith("==")]
    hdr = rows[0]
    out = []
    if "Metric Name" in hdr:
        ik, im, iu, iv, iid = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "ID"))
        per = {}
        for r in rows[1:]:
            if kernel not in r[ik]:
                continue
            v = float(r[iv].replace(",", "")) * _UNIT.get(r[iu].strip().lower(), 1.0)
            per.setdefault(r[iid], {})[r[im]] = v
        return [per[k] for k in sorted(per, key=int)]
    units = rows[1]
    ik = hdr.index("Kernel Name")
    for r in rows[2:]:
        if kernel not in r[ik]:
            continue
        rec = {}
        for m in RECORD_METRICS:
            if m in hdr:
                j = hdr.index(m)
                try:
                    rec[m] = float(r[j].replace(",", "")) * _UNIT.get(units[j].strip().lower(), 1.0)
                except ValueError:
                    pass
        out.append(rec)
    return out


def record_counters(args) -> None:
    """Write (or replace) the counter record of one kernel in profiles/counters.json from an ncu
    CSV, with the SHA-256 of the kernel's source files so a later source change marks it stale."""
    launches = parse_ncu_csv(args.record_counters, args.kernel)
    if not launches:
        raise SystemExit(f"no launch of {args.kernel} in {args.record_counters}")
    last = launches[-1]
    rec = {"kernel": args.kernel, "workload": args.record_workload, "command": args.record_command,
           "line": args.record_line, "when": time.strftime("%Y-%m-%d"), "launches_in_capture": len(launches),
           "metrics": {k: v for k, v in last.items()},
           "sources": {p: _sha256(p) for p in args.record_sources.split(",") if p}}
    if "dram__bytes_read.sum" in last and "dram__bytes_write.sum" in last:
        rec["dram_bytes_per_launch"] = int(round(last["dram__bytes_read.sum"] + last["dram__bytes_write.sum"]))
    try:
        with open(COUNTERS) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        doc = {"about": "ncu counters per kernel (bench.py --record-counters); bench.py reports "
                        "roofline.traffic from dram_bytes_per_launch while every listed source is unchanged",
               "records": []}
    doc["records"] = [r for r in doc["records"] if r.get("kernel") != args.kernel] + [rec]
    with open(COUNTERS, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(json.dumps(rec, indent=1))


def cp_survey_flops_per_launch(r: int = CP_R, d: int = D, n: int = N, sweeps: int = SWEEPS) -> float:
    """The CP-ALS route's algorithmic flops per launch of cp_als_sweep_rk2 as the scope table counts
    them for the explicit y = p(dt L) x (rank R_y = (1 + 2d + d(d-1)/2) r): per mode
    2 d n r^2 (factor Grams) + 2 n R_y r (right-hand side) + r^3 / 3 (Cholesky), d modes a sweep."""
    ry = (1 + 2 * d + d * (d - 1) // 2) * r
    return sweeps * d * (2.0 * d * n * r * r + 2.0 * n * ry * r + r ** 3 / 3.0)


def profile_pass(W, torch, flush, steps: int):
    """Event-time every kernel class over `steps` steps; roofline of the dominant class.  For the
    CP kernel `achieved` uses the scope table's algorithmic flops of the explicit form (75.3 MFLOP
    per launch); the kernel itself never forms y and executes the fewer flops its counter reports
    (`executed_*`)."""
    prof = profiled_steps(W.ctx, torch, flush, W.step, steps)
    rl, shares = class_roofline(prof, steps, W.ctx, line="adv6d")
    roof = rl["dominant"]
    if roof["class"] == "cp_solve":
        # the form cp_als_sweep_rk2 took on this context names the kernel and its counter record
        kern = "cp_als_rk2_cluster" if W.G.cp_als_rk2_cluster_ctas(W.ctx, CP_R, CP_R) else "cp_als_rk2_persistent"
        roof["kernel"] = kern
        attach_traffic(roof, [kern], "adv6d")
    if roof["class"] == "cp_solve" and roof["avg_launch_us"]:
        alg = cp_survey_flops_per_launch()
        roof["executed_flops_per_launch"] = roof.get("flops_per_launch")
        roof["executed_achieved"] = roof["achieved"]
        roof["executed_frac"] = roof["frac"]
        roof["flops_per_launch"] = alg
        roof["flops"] = ("scope-table algorithmic flops of the explicit form: per mode 2 d n r^2 + 2 n R_y r "
                         "+ r^3/3, R_y = 28 r, r = 24, 6 modes x 5 sweeps")
        roof["achieved"] = alg / (roof["avg_launch_us"] * 1e-6) / 1e12
        roof["frac"] = roof["achieved"] / roof["peak"]
    return roof, shares


def run_e2e(W, G, torch, steps: int) -> dict:
    """Per step, through the same public calls: the HT and CP state (one contiguous buffer each,
    at capacity, plus the HT ranks) copied from pinned host memory to the device, the step, and
    the new state copied back to pinned host memory; the host waits for it every step.  The
    copies and the step are captured together in one CUDA graph."""
    hu = torch.empty(W.u.blob.numel(), dtype=torch.float64, pin_memory=True)
    hr = torch.empty(W.u.rank_buf.numel(), dtype=torch.int32, pin_memory=True)
    hx = torch.empty(W.X.blob.numel(), dtype=torch.float64, pin_memory=True)
    hu.copy_(W.u.blob)
    hr.copy_(W.u.rank_buf)
    hx.copy_(W.X.blob)
    torch.cuda.synchronize()

    def one():
        W.u.blob.copy_(hu, non_blocking=True)
        W.u.rank_buf.copy_(hr, non_blocking=True)
        W.X.blob.copy_(hx, non_blocking=True)
        W.step()
        hu.copy_(W.u.blob, non_blocking=True)
        hr.copy_(W.u.rank_buf, non_blocking=True)
        hx.copy_(W.X.blob, non_blocking=True)

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        one()
    graph.replay()
    torch.cuda.synchronize()
    nbytes = hu.numel() * 8 + hr.numel() * 4 + hx.numel() * 8
    t0 = time.perf_counter()
    for _ in range(steps):
        graph.replay()
        torch.cuda.synchronize()
    el = time.perf_counter() - t0
    return {"value": steps / el, "unit": "steps/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": steps, "cuda_graph": True}


def run_reference(args):
    """The oracle on the host cores, on the same config, metric and unit."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    per = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    cores = os.cpu_count() or 1     # every sample may use all host cores (BLAS threads set so)
    for _ in range(args.warmup):
        _, err = oracle_sample_process(per / 4, cores)
        if err is not None:
            raise RuntimeError(f"oracle sample failed: {err}")
    total_steps, total_s = 0, 0.0
    for _ in range(args.steps):
        r, err = oracle_sample_process(per, cores)
        if err is not None:
            raise RuntimeError(f"oracle sample failed: {err}")
        total_steps += r["steps"]
        total_s += r["seconds"]
    v = total_steps / total_s
    out = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded 6-D advection, n=64)",
           "impl": "reference",
           "config": config_keys("fp64", "n/a (host cores; the oracle uses no GPU)", "host cores"),
           "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle", "cpu": host_cpu(),
                            "sample": f"{args.steps} samples of up to {per:.1f} s, each from t=0 in a fresh "
                                      f"process with {cores} BLAS threads, FP64 numpy oracle "
                                      f"({total_steps} steps)"},
           "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.cpu_seconds)))
        return
    if args.record_counters:
        record_counters(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
