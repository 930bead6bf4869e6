"""GPU parity at the shapes of the other configurations and at edge cases (FP64 form)."""
import math

import numpy as np
import pytest

from oracle import ht as OH
from oracle.problems import advection_A
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import advection_case, cp_random_factors
from tests.helpers import min_gap, random_ht, rel_err

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


def to_gpu(G, u, cap):
    t = G.HTTensor(u.tree.d, u.n, cap)
    t.upload(u.node)
    return t


def from_gpu(t, tree):
    return OH.HT(tree, list(t.n), t.download())


def test_twelve_dim_depth4_tree_steps(G):
    """12-D advection (the shape of the 12-D configuration: depth-4 tree, separable rank-3
    initial condition), n = 6, r_max 6, 3 RK2 steps against the oracle."""
    d, n = 12, 6
    case = advection_case(d, n, n_terms=3, seed_offset=4)
    A = advection_A(case)
    tree = build_tree(d)
    assert max(tree.depth) == 4
    u = OH.from_cp(np.ones(3), case.ic_factors())
    ctx = G.Context(d, [n] * d, cap=6, max_terms=1)
    g = to_gpu(G, u, 6)
    op = G.advection_op(case.c, case.h)
    for step in range(3):
        u, rep = OH.step_rk2_poly(u, A, 1e-6, 6)
        G.ht_step(ctx, g, op, case.dt, 1e-6, 6)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64


def test_two_dim_steps_and_rank_cap_one(G):
    d, n = 2, 24
    case = advection_case(d, n, seed=3)
    A = advection_A(case)
    u = random_ht(d, n, 4, seed=2, scale_decay=0.3)
    for rmax in (1, 4):
        uo = u
        ctx = G.Context(d, [n] * d, cap=4, max_terms=1)
        g = to_gpu(G, u, 4)
        op = G.advection_op(case.c, case.h)
        for step in range(3):
            uo, rep = OH.step_rk2_poly(uo, A, 1e-9, rmax)
            G.ht_step(ctx, g, op, case.dt, 1e-9, rmax)
            sync()
            assert g.ranks() == rep.ranks
            assert rel_err(from_gpu(g, uo.tree), uo) < TOL64


def test_zero_tensor_and_zero_tolerance(G):
    import torch
    d, n = 4, 5
    z = random_ht(d, n, 2, seed=4)
    for t in z.node:
        z.node[t] = np.zeros_like(z.node[t])
    ctx = G.Context(d, [n] * d, cap=6, max_terms=1)
    g = to_gpu(G, z, 6)
    out = G.HTTensor(d, [n] * d, 6)
    G.ht_truncate(ctx, g, 1e-8, 6, out)
    sync()
    ctx.check()
    assert out.ranks()[1:] == [1] * (2 * d - 2)
    assert all(np.abs(a).max() == 0.0 for a in out.download().values())
    # tol 0 keeps every nonzero direction up to the cap
    u = random_ht(d, n, 3, seed=5, scale_decay=0.5)
    ref, rep = OH.truncate(u, 0.0, 6)
    g2 = to_gpu(G, u, 6)
    G.ht_truncate(ctx, g2, 0.0, 6, out)
    sync()
    assert out.ranks() == rep.ranks
    assert rel_err(from_gpu(out, u.tree), ref) < TOL64
    assert rel_err(ref, u) < 1e-12        # nothing was cut


def test_adv6d_n64_full_size_mass_bound(G):
    """n=64, d=6 (64^6 grid points): the apply conserves the discrete mass exactly, the HSVD
    changes it by at most sqrt(N) |v - T(v)| <= sqrt(N) tol |v|; checked over 5 steps."""
    import torch
    case = advection_case(6, 64, seed_offset=1)
    u = OH.from_cp(np.ones(2), case.ic_factors())
    ctx = G.Context(6, [64] * 6, cap=32, max_terms=1)
    g = to_gpu(G, u, 32)
    op = G.advection_op(case.c, case.h)
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.ht_mass(ctx, g, m)
    sync()
    m0 = float(m[0])
    assert abs(m0 - OH.mass(u)) < 1e-12 * abs(m0)
    nrm = OH.norm(u)
    for _ in range(5):
        G.ht_step(ctx, g, op, case.dt, 1e-8, 32)
        G.ht_mass(ctx, g, m)
        sync()
        m1 = float(m[0])
        assert abs(m1 - m0) <= math.sqrt(64.0 ** 6) * 1e-8 * nrm * 1.01
        m0 = m1


def test_kinetic6d_shape_heun2(G):
    """Linearised 6-D kinetic equation (x periodic, v in [-6, 6]) with its initial condition
    M(v)(1 + 0.1 prod sin x_i) plus a seeded rank-4 perturbation, n = 12, HEUN2 with a
    truncation after each stage, r_max 12, tol 1e-6: three steps against the oracle."""
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(12)
    w, F = kinetic_ic(kc)
    u = OH.from_cp(w, F)
    alphas, factors = kinetic_terms(kc)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [12] * 6, cap=12, max_terms=5)
    g = to_gpu(G, u, 12)
    for step in range(3):
        u, reps = OH.step_heun2(u, alphas, factors, kc.dt, 1e-6, 12)
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 12, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        assert g.ranks() == reps[1].ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"


def test_twelve_dim_full_size_steps(G):
    """The 12-D workload at full size (n = 128 per dimension, 128^12 grid points, r_max 64,
    tol 1e-8, separable rank-3 initial condition): the oracle's HT-format step needs no full
    grid, so five RK2 steps are compared with it directly, ranks and entries; the discrete mass
    moves by at most sqrt(N) tol |v| per step."""
    import torch
    d, n, cap = 12, 128, 64
    case = advection_case(d, n, n_terms=3, seed_offset=4)
    A = advection_A(case)
    u = OH.from_cp(np.ones(3), case.ic_factors())
    ctx = G.Context(d, [n] * d, cap=cap, max_terms=1)
    g = to_gpu(G, u, cap)
    op = G.advection_op(case.c, case.h)
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.ht_mass(ctx, g, m)
    sync()
    m0 = float(m[0])
    assert abs(m0 - OH.mass(u)) < 1e-12 * abs(m0)
    for step in range(5):
        nrm = OH.norm(u)
        u, rep = OH.step_rk2_poly(u, A, 1e-8, cap)
        G.ht_step(ctx, g, op, case.dt, 1e-8, cap)
        G.ht_mass(ctx, g, m)
        sync()
        ctx.check()
        assert g.ranks() == rep.ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"
        m1 = float(m[0])
        assert abs(m1 - m0) <= math.sqrt(float(n) ** d) * 1e-8 * nrm * 1.01
        m0 = m1


def test_truncate_tall_node_matrices_rank_deficient(G):
    """ht_truncate of a d=4 HT with every rank 24: the interior node matrices (576 x 24) are
    reduced in row blocks plus a banded combine step.  A duplicated leaf column and a zero
    transfer slice make node matrices rank deficient.  Ranks and T(u) against the oracle."""
    d, n, r = 4, 30, 24
    u = random_ht(d, n, r, seed=11, scale_decay=0.7)
    tree = u.tree
    leaf = next(t for t in range(tree.n_nodes) if tree.is_leaf(t))
    inner = next(t for t in range(1, tree.n_nodes) if not tree.is_leaf(t))
    u.node[leaf][:, 1] = u.node[leaf][:, 0]
    u.node[inner][:, :, 5] = 0.0
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1)
    for rel_tol in (1e-6, 1e-10, 1e-13):
        ref, rep = OH.truncate(u, rel_tol, r)
        g = to_gpu(G, u, r)
        out = G.HTTensor(d, [n] * d, r)
        G.ht_truncate(ctx, g, rel_tol, r, out)
        sync()
        ctx.check()
        assert out.ranks() == rep.ranks, f"tol {rel_tol}"
        assert rel_err(from_gpu(out, tree), ref) < TOL64, f"tol {rel_tol}"


@pytest.mark.parametrize("n,r,decay,deficient,ctx_cap",
                         [(150, 131, 0.85, True, 131), (144, 140, 0.8, False, 140), (380, 370, 0.95, False, 124)])
def test_truncate_wide_node_factors(G, n, r, decay, deficient, ctx_cap):
    """ht_truncate of d=4 HT tensors of rank 131 (odd: a dummy player in every Jacobi round), 140
    and 370: every node factor is that many columns wide, so the node SVDs run in the cluster form
    (columns spread over the shared memory of one thread-block cluster; 370 columns come near its
    480-column limit, the width of the kinetic workload's node factors).  Graded transfer tensors
    make the root's children cut to ranks near 40 (132 at rank 370) at tol 1e-8; the other nodes
    keep every direction.  The deficient case duplicates a leaf column and zeroes a transfer
    slice (zero singular values in the wide factors).  The rank-370 input fits a context of
    capacity 124 (truncation inputs up to 3 x 124 = 372).  Ranks and T(u) against the oracle
    (about 100 s of oracle time at rank 370)."""
    d = 4
    u = random_ht(d, n, r, seed=21, scale_decay=decay)
    if deficient:
        tree = u.tree
        leaf = next(t for t in range(tree.n_nodes) if tree.is_leaf(t))
        inner = next(t for t in range(1, tree.n_nodes) if not tree.is_leaf(t))
        u.node[leaf][:, 1] = u.node[leaf][:, 0]
        u.node[inner][:, :, 7] = 0.0
    ref, rep = OH.truncate(u, 1e-8, r)
    assert max(rep.ranks[1:]) == r and min(rep.ranks[1:]) < r
    ctx = G.Context(d, [n] * d, cap=ctx_cap, max_terms=1)
    g = to_gpu(G, u, r)
    out = G.HTTensor(d, [n] * d, r)
    G.ht_truncate(ctx, g, 1e-8, r, out)
    sync()
    ctx.check()
    assert out.ranks() == rep.ranks
    assert rel_err(from_gpu(out, u.tree), ref) < TOL64
    ctx.close()


def test_profiler_counts_the_cooperative_qr_flops(G):
    """The event profiler's QR class counts the Householder flops of every matrix it reduces,
    those of the cooperative form too: in the truncation of a d=4 HT tensor of rank 96 the two
    interior node matrices (96^2 x 96, over 2^16 entries and twice as tall as wide) go to the
    cooperative kernel, so the class must count at least their 2 sum_j (m - j)(2 + 4 (k - j - 1))
    flops (about 339 M; the leaves' 100 x 96 matrices add about 5 M)."""
    d, n, r = 4, 100, 96
    u = random_ht(d, n, r, seed=5, scale_decay=0.9)
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1)
    g = to_gpu(G, u, r)
    out = G.HTTensor(d, [n] * d, r)
    ctx.profile(True)
    G.ht_truncate(ctx, g, 1e-8, r, out)
    sync()
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.check()
    m, k = r * r, r
    interior = sum((m - j) * (2.0 + 4.0 * (k - j - 1)) for j in range(k))
    assert prof["qr"]["launches"] > 0
    assert prof["qr"]["flops"] >= 2 * interior, (prof["qr"]["flops"], 2 * interior)
    ctx.close()


def test_biorth_cluster_form_matches_the_one_cta_form_bitwise(G):
    """The cluster form of the X_t Y_t = I refinement (each node's four products dealt out over
    the CTAs of a thread-block cluster) sums every element in the order of the one-CTA form:
    ht_truncate of a d=4 tensor of rank 131 (k^2 and K k above the cluster's threads) returns
    the same ranks and the same bits with either form, and matches the oracle."""
    d, n, r = 4, 150, 131
    u = random_ht(d, n, r, seed=21, scale_decay=0.85)
    ref, rep = OH.truncate(u, 1e-8, r)
    outs = []
    for form in (G.BIORTH_FORM_CLUSTER, G.BIORTH_FORM_CTA):
        ctx = G.Context(d, [n] * d, cap=r, max_terms=1, biorth_form=form)
        assert (ctx.biorth_cluster_ctas() in (8, 16)) == (form == G.BIORTH_FORM_CLUSTER)
        out = G.HTTensor(d, [n] * d, r)
        G.ht_truncate(ctx, to_gpu(G, u, r), 1e-8, r, out)
        sync()
        ctx.check()
        outs.append((out.ranks(), from_gpu(out, u.tree)))
        ctx.close()
    (ra, a), (rb, b) = outs
    assert ra == rb == rep.ranks
    for t in range(u.tree.n_nodes):
        assert np.array_equal(a.node[t], b.node[t]), t
    assert rel_err(a, ref) < TOL64


def test_untruncated_graded_spectrum_reproduces_u(G):
    """A truncation that keeps every direction returns u to rounding, even when node spectra
    span ten decades (transfer tensors graded by 0.7^j, rank 24): the projectors Y_t X_t of the
    R-factor form are refined to X_t Y_t = I, so no 1/s_k amplification of SVD rounding remains
    (without the refinement this case moved u by 2.5e-7)."""
    d, n, r = 4, 30, 24
    u = random_ht(d, n, r, seed=11, scale_decay=0.7)
    ref, rep = OH.truncate(u, 1e-13, r)
    assert rep.ranks[1:] == [r] * (2 * d - 2)
    ctx = G.Context(d, [n] * d, cap=r, max_terms=1)
    g = to_gpu(G, u, r)
    out = G.HTTensor(d, [n] * d, r)
    G.ht_truncate(ctx, g, 1e-13, r, out)
    sync()
    ctx.check()
    assert out.ranks() == rep.ranks
    assert rel_err(from_gpu(out, u.tree), u) < 1e-13


def test_kinetic6d_n64_full_size_two_heun2_steps(G):
    """The kinetic workload at full size: n = 64 per variable (64^6 grid points), HT r_max 64,
    five operator terms (a 31 GB context), its seeded initial condition (rank 6), HEUN2 with
    tol 1e-6: two steps against the oracle's HT-format steps (node ranks reach 42; the stage sums
    put 3960 x 252 matrices through the QR and 252-column node factors through the SVD)."""
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(64)
    w, F = kinetic_ic(kc)
    u = OH.from_cp(w, F)
    alphas, factors = kinetic_terms(kc)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [64] * 6, cap=64, max_terms=5)
    g = to_gpu(G, u, 64)
    for step in range(2):
        u, reps = OH.step_heun2(u, alphas, factors, kc.dt, 1e-6, 64)
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2)
        sync()
        ctx.check()
        assert g.ranks() == reps[1].ranks, f"step {step}"
        assert rel_err(from_gpu(g, u.tree), u) < TOL64, f"step {step}"
    ctx.close()


def test_kinetic6d_n64_late_window_one_step(G):
    """The kinetic workload at full size after 45 HEUN2 steps on the GPU (node ranks near 61, node
    factors 300-370 columns wide: the cluster SVD near its limit, the cooperative QR on the stage
    sums): one more step from that state on the GPU and in the oracle, ranks and tensors compared
    (the bench's kinetic window is steps 46-50)."""
    from oracle.problems import kinetic_terms
    from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic
    kc = kinetic_case(64)
    w, F = kinetic_ic(kc)
    u0 = OH.from_cp(w, F)
    alphas, factors = kinetic_terms(kc)
    kop = G.KineticOp(kc)
    ctx = G.Context(6, [64] * 6, cap=64, max_terms=5)
    g = to_gpu(G, u0, 64)
    for _ in range(45):
        G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2)
    sync()
    ctx.check()
    state = from_gpu(g, u0.tree)
    assert max(g.ranks()[1:]) >= 55
    ref, reps = OH.step_heun2(state, alphas, factors, kc.dt, 1e-6, 64)
    G.ht_step(ctx, g, kop.op, kc.dt, 1e-6, 64, scheme=G.HT_SCHEME_HEUN2)
    sync()
    ctx.check()
    assert g.ranks() == reps[1].ranks
    assert rel_err(from_gpu(g, u0.tree), ref) < TOL64
    ctx.close()
