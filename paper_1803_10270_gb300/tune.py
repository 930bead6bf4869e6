"""Autotuner for the library's launch parameters on the GPU at hand.

It measures, through the library's own entry points:

* tc_min_work: the work (multiply-adds m n k batch) from which a contraction of the mixed form
  runs faster on the tensor-core split kernel than on the split-FP32 CUDA-core kernel that takes
  the mixed form's smaller contractions.  Square and batched shapes of the truncation's
  contractions are timed through both kernels (ht_tune_time_gemm); the threshold is the smallest
  measured work from which the tensor cores win at that work and every larger one.
* gemm_ctas_per_sm: CTAs per SM of the FP64 contraction launches, chosen by the summed time of
  the same shapes, per capacity bucket of the context (the largest truncation input rank Kc).
* svd_cluster_min_cols: the node-factor width from which the thread-block-cluster SVD beats the
  one-CTA SVD, from ht_truncate timings of random HT tensors whose node factors have that width.

Results go to a JSON cache (``_lib/tuning.json`` beside the built library, keyed by the GPU's name
and SM count); ``Context`` reads it (``cached``) unless given explicit tuning values, and an
absent cache leaves the library defaults.  ``python -m paper_1803_10270_gb300.tune`` runs it.
"""
from __future__ import annotations

import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_lib", "tuning.json")
# capacity buckets (largest truncation input rank Kc) of the per-bucket FP64 CTA count
KC_BUCKETS = (48, 96, 192, 100000)


def device_key(device: int = 0) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|{p.multi_processor_count}"


def _read() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cached(device: int = 0, kc: int | None = None) -> dict:
    """The tuned ht_config values of this GPU ({} when it was never tuned).  With kc (the context's
    largest truncation input rank), the FP64 CTA count of that capacity bucket."""
    try:
        ent = _read().get(device_key(device))
    except Exception:
        return {}
    if not ent:
        return {}
    out = {k: ent[k] for k in ("tc_min_work", "svd_cluster_min_cols") if k in ent}
    per = ent.get("gemm_ctas_per_sm_by_kc", {})
    if per:
        b = next((x for x in KC_BUCKETS if (kc or KC_BUCKETS[0]) <= x), KC_BUCKETS[-1])
        if str(b) in per:
            out["gemm_ctas_per_sm"] = per[str(b)]
    return out


def _shapes(kc_max: int):
    """(m, n, k, batch) shapes of a truncation at capacity kc_max: a transfer absorption
    (k1 x k2 k times k1 x k1), its batched form, a leaf projection and a node factor product."""
    out = []
    for r in (8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384):
        if r > kc_max:
            break
        out.append((r, r * r, r, 1))            # R_t1 B_t: k1 x (k2 k)
        out.append((r, r, r, r))                # batched mode product
        out.append((128, r, r, 1))              # leaf projection, n = 128
        out.append((r, r, r, 1))                # node factor R_t E_t
    return out


def crossover(pts) -> int:
    """The tensor-core threshold from timed points (work, CUDA-core ms, tensor-core ms, shape): the
    smallest measured work from which the tensor cores are faster at that work and every larger
    one; twice the largest measured work when they never are (1 << 40 without points)."""
    pts = sorted(pts, key=lambda p: p[0])
    for i, p in enumerate(pts):
        if all(q[2] < q[1] for q in pts[i:]):
            return int(p[0])
    return int(pts[-1][0] * 2) if pts else 1 << 40


def _time(G, m, n, k, b, route, slices, ctas, reps):
    """Mean ms of one contraction: one launch first, then up to `reps` more within about 20 ms."""
    t1 = G.tune_time_gemm(m, n, k, b, route, slices, ctas, 1)
    r = max(1, min(reps, int(20.0 / max(t1, 1e-3))))
    return G.tune_time_gemm(m, n, k, b, route, slices, ctas, r) if r > 1 else t1


def tune(device: int = 0, slices: int = 4, reps: int = 10, write: bool = True, verbose: bool = False) -> dict:
    import torch
    from paper_1803_10270_gb300 import htgpu as G
    torch.cuda.set_device(device)
    G.load()
    t0 = time.time()
    # ---- FP64 CTAs per SM, per capacity bucket
    ctas_opts = (4, 8, 16, 32)
    by_kc = {}
    timings = {}
    for kc in KC_BUCKETS:
        shapes = _shapes(min(kc, 384))
        tot = {}
        for c in ctas_opts:
            tot[c] = sum(_time(G, m, n, k, b, 0, slices, c, reps) for (m, n, k, b) in shapes)
        best = min(tot, key=tot.get)
        by_kc[str(kc)] = best
        timings[f"fp64_ctas_kc{kc}"] = {str(c): tot[c] for c in ctas_opts}
    # ---- tensor-core crossover against the split-FP32 kernel (at the CUDA-core launches' tuned
    # CTA count of the largest bucket)
    c_big = by_kc[str(KC_BUCKETS[-1])]
    pts = []
    for (m, n, k, b) in _shapes(384):
        t64 = _time(G, m, n, k, b, 2, slices, c_big, reps)
        ttc = _time(G, m, n, k, b, 1, slices, 4, reps)
        pts.append((m * n * k * b, t64, ttc, (m, n, k, b)))
    pts.sort(key=lambda p: p[0])
    tc_min = crossover(pts)
    timings["gemm_crossover"] = [{"work": w, "shape": list(sh), "f32x2_ms": a, "tc_ms": c} for (w, a, c, sh) in pts]
    # ---- cluster SVD switch width
    svd_min, svd_t = _tune_svd_switch(G, torch, device)
    timings["svd_switch"] = svd_t
    res = {"tc_min_work": int(tc_min), "gemm_ctas_per_sm_by_kc": by_kc, "svd_cluster_min_cols": int(svd_min),
           "slices": slices, "when": time.strftime("%Y-%m-%d %H:%M:%S"), "seconds": time.time() - t0,
           "timings": timings}
    if verbose:
        print(json.dumps({k: v for k, v in res.items() if k != "timings"}, indent=1))
    if write:
        doc = _read()
        doc[device_key(device)] = res
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(doc, f, indent=1)
    return res


def _tune_svd_switch(G, torch, device: int):
    """Smallest node-factor width (of those measured) from which truncations with the cluster SVD
    are faster than with the one-CTA SVD, over random d = 4 HT tensors of that rank."""
    import numpy as np
    from paper_1803_10270_gb300.inputs import normal_arrays
    widths = (64, 96, 128, 160, 192)
    res = {}
    for w in widths:
        d, n = 4, w + 8
        tr = G.tree_info(d, 0)
        shapes = []
        for t in range(tr.n_nodes):
            if tr.is_leaf(t):
                shapes.append((n, w))
            elif t == 0:
                shapes.append((w, w))
            else:
                shapes.append((w, w, w))
        arrs = normal_arrays(shapes, 5 + w)
        nodes = {t: arrs[t] * (0.9 ** np.arange(arrs[t].shape[-1])).reshape((1,) * (arrs[t].ndim - 1) + (-1,))
                 if t else arrs[t] for t in range(tr.n_nodes)}
        times = {}
        for label, mc in (("cluster", 32), ("one_cta", 480)):
            ctx = G.Context(d, [n] * d, cap=(w + 2) // 3, max_terms=1, device=device,
                            tuning={"svd_cluster_min_cols": mc})
            u = G.HTTensor(d, [n] * d, w)
            u.upload(nodes)
            out = G.HTTensor(d, [n] * d, w)
            G.ht_truncate(ctx, u, 1e-8, w, out)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                G.ht_truncate(ctx, u, 1e-8, w, out)
            e1.record()
            torch.cuda.synchronize()
            ctx.check()
            times[label] = e0.elapsed_time(e1) / 3
            ctx.close()
        res[str(w)] = times
    win = [w for w in widths if res[str(w)]["cluster"] < res[str(w)]["one_cta"]]
    best = 128
    for i, w in enumerate(widths):
        if all(x in win for x in widths[i:]):
            best = w
            break
    return best, res


if __name__ == "__main__":
    import sys
    dev = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    tune(dev, verbose=True)
