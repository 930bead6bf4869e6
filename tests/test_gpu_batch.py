"""Batched steps (ht_batch_step): every instance of a batch equals ht_step on that instance
alone, bit for bit (the same kernels on the same descriptors, one launch covering all
instances; these batches are small enough that the QR launches split large matrices as a lone
step does), and so the FP64 oracle's step (Section 3.2) within the FP64 bound.  Instances
differ in grid size, rank capacity, velocity and cap, as in a ragged batch of advection
problems."""
import math

import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A, kinetic_terms
from paper_1803_10270_gb300.inputs import advection_case, kinetic_case
from tests.helpers import random_ht, rel_err

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


def upload(G, u: OH.HT, cap):
    t = G.HTTensor(u.tree.d, u.n, cap)
    t.upload(u.node)
    return t


def same_tensor(a, b):
    ra, rb = a.ranks(), b.ranks()
    assert ra == rb
    da, db = a.download(), b.download()
    for t in range(len(da)):
        assert np.array_equal(da[t], db[t]), f"node {t}"


# (n, cap) per instance: ragged grids and capacities
RAGGED = [(8, 4), (12, 8), (16, 6), (10, 5), (6, 8)]


def advection_instances(G, d, seeds):
    out = []
    for (n, cap), seed in zip(RAGGED, seeds):
        case = advection_case(d, n, seed=seed)
        u0 = OH.from_cp(np.ones(2), case.ic_factors())
        out.append((case, u0, cap))
    return out


def test_batch_rk2poly_matches_single_and_oracle(G):
    d = 6
    inst = advection_instances(G, d, [101, 202, 303, 404, 505])
    singles, batched, ctx_s, ctx_b, ops, refs = [], [], [], [], [], []
    for case, u0, cap in inst:
        ctx_s.append(G.Context(d, [case.n] * d, cap=cap, max_terms=1))
        ctx_b.append(G.Context(d, [case.n] * d, cap=cap, max_terms=1))
        singles.append(upload(G, u0, cap))
        batched.append(upload(G, u0, cap))
        ops.append(G.advection_op(case.c, case.h))
        refs.append(u0)
    batch = G.Batch(ctx_b, batched)
    dts = [c.dt for c, _, _ in inst]
    tols = [1e-8] * len(inst)
    rmaxs = [cap for _, _, cap in inst]
    for step in range(3):
        for i, (case, _, cap) in enumerate(inst):
            G.ht_step(ctx_s[i], singles[i], ops[i], case.dt, 1e-8, cap)
            refs[i], _ = OH.step_rk2_poly(refs[i], advection_A(case), 1e-8, cap)
        batch.step(ops, dts, tols, rmaxs)
        sync()
        for i in range(len(inst)):
            ctx_b[i].check()
            same_tensor(batched[i], singles[i])
            e = rel_err(OH.HT(refs[i].tree, list(refs[i].n), batched[i].download()), refs[i])
            assert e < TOL64, f"instance {i} step {step}: {e:.3e}"
    batch.close()


def test_batch_heun2_kinetic_matches_single(G):
    d = 6
    sizes = [(5, 6), (6, 6), (4, 4)]
    ctx_s, ctx_b, singles, batched, ops, kops, refs, kcs = [], [], [], [], [], [], [], []
    for j, (n, cap) in enumerate(sizes):
        kc = kinetic_case(n)
        kcs.append(kc)
        u0 = random_ht(d, n, 2, seed=41 + j, scale_decay=0.3)
        kop = G.KineticOp(kc)
        kops.append(kop)
        ops.append(kop.op)
        ctx_s.append(G.Context(d, [n] * d, cap=cap, max_terms=5))
        ctx_b.append(G.Context(d, [n] * d, cap=cap, max_terms=5))
        singles.append(upload(G, u0, cap))
        batched.append(upload(G, u0, cap))
        refs.append(u0)
    batch = G.Batch(ctx_b, batched)
    for step in range(2):
        for i, (n, cap) in enumerate(sizes):
            G.ht_step(ctx_s[i], singles[i], ops[i], kcs[i].dt, 1e-6, cap, scheme=G.HT_SCHEME_HEUN2)
            alphas, factors = kinetic_terms(kcs[i])
            refs[i], _ = OH.step_heun2(refs[i], alphas, factors, kcs[i].dt, 1e-6, cap)
        batch.step(ops, [kc.dt for kc in kcs], [1e-6] * 3, [cap for _, cap in sizes], scheme=G.HT_SCHEME_HEUN2)
        sync()
        for i in range(len(sizes)):
            same_tensor(batched[i], singles[i])
            e = rel_err(OH.HT(refs[i].tree, list(refs[i].n), batched[i].download()), refs[i])
            assert e < TOL64, f"instance {i} step {step}: {e:.3e}"
    batch.close()


def test_batch_graph_replay_matches_eager(G):
    import torch
    d = 6
    inst = advection_instances(G, d, [7, 8, 9, 10])
    ctx_e = [G.Context(d, [c.n] * d, cap=cap, max_terms=1) for c, _, cap in inst]
    ctx_g = [G.Context(d, [c.n] * d, cap=cap, max_terms=1) for c, _, cap in inst]
    ue = [upload(G, u0, cap) for _, u0, cap in inst]
    ug = [upload(G, u0, cap) for _, u0, cap in inst]
    ops = [G.advection_op(c.c, c.h) for c, _, _ in inst]
    dts = [c.dt for c, _, _ in inst]
    tols = [1e-8] * len(inst)
    rmaxs = [cap for _, _, cap in inst]
    be = G.Batch(ctx_e, ue)
    bg = G.Batch(ctx_g, ug)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bg.step(ops, dts, tols, rmaxs, stream=s)        # uploads the operators before capture
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            bg.step(ops, dts, tols, rmaxs, stream=s)
    for _ in range(4):
        be.step(ops, dts, tols, rmaxs)
    for _ in range(3):
        graph.replay()
    sync()
    for a, b in zip(ue, ug):
        same_tensor(a, b)
    be.close()
    bg.close()


def test_batch_argument_errors(G):
    d = 4
    case = advection_case(d, 6, seed=3)
    u0 = OH.from_cp(np.ones(2), case.ic_factors())
    c1 = G.Context(d, [6] * d, cap=4, max_terms=1)
    c2 = G.Context(5, [6] * 5, cap=4, max_terms=1)
    t1 = upload(G, u0, 4)
    t1b = upload(G, u0, 4)
    with pytest.raises(G.HTError):
        G.Batch([c1, c1], [t1, t1b])             # one workspace per instance
    u5 = OH.from_cp(np.ones(2), advection_case(5, 6, seed=3).ic_factors())
    with pytest.raises(G.HTError):
        G.Batch([c1, c2], [t1, upload(G, u5, 4)])   # same d for every instance
    b = G.Batch([c1], [t1])
    op = G.advection_op(case.c, case.h)
    with pytest.raises(G.HTError):
        b.step([op], [case.dt], [1e-8], [5])       # rmax above the tensor's capacity
    with pytest.raises(G.HTError):
        G.Batch([c1], [t1b])                        # c1 is bound to b
    b.close()
    b2 = G.Batch([c1], [t1b])                       # released by close
    b2.close()
