"""The kinetic step pinned by its x-Fourier-mode closed form, independent of the operator's
term list.

The periodic central difference is circulant in x: on exp(i k x) it multiplies by
i sin(k h) / h.  For an x-band-limited f (the kinetic initial condition carries x-modes |k| <= 2
only) every x-mode K = (k1, k2, k3) therefore evolves on its own v-grid problem,
    L_K g = -i (v1 s(k1) + v2 s(k2) + v3 s(k3)) g - nu g + nu M(v) sum_v h_v^3 g,   s(k) = sin(k h)/h,
(the transport of the linearised kinetic equation, Section 4.2, eq. BGK_LIN, and the collision
term with rho = sum_v h_v^3 f), and one untruncated HEUN2 step is p(dt L_K) g with
p(z) = 1 + z + z^2/2 on each mode.  Nothing here uses the oracle's kinetic term list, so a wrong
sign, a transport factor on the wrong dimension or a lost term in it fails the comparison.
"""
import functools

import numpy as np

from oracle import ht as OH
from oracle.problems import kinetic_terms
from paper_1803_10270_gb300.inputs import kinetic_case, kinetic_ic


@functools.lru_cache(maxsize=1)
def full_size_step():
    """(case, CP weights, CP factors, u0, u1): one untruncated HEUN2 step of the oracle at the
    kinetic workload's full size (n = 64, dt the explicit step), shared by the tests below."""
    kc = kinetic_case(64)
    w, F = kinetic_ic(kc)
    alphas, factors = kinetic_terms(kc)
    u0 = OH.from_cp(w, F)
    u1, _ = OH.step_heun2(u0, alphas, factors, kc.dt, 0.0, 10 ** 6)
    return kc, w, F, u0, u1


def mode_closed_form_step(kc, w, F, dt, kmax=2):
    """Full-grid f after one step of p(dt L) on the band-limited CP f = sum_t w_t prod_j F_j[:, t]."""
    n, hx, hv, nu = kc.n, kc.hx, kc.hv, kc.nu
    x, v, m = kc.xgrid(), kc.vgrid(), kc.maxwellian()
    ks = np.arange(-kmax, kmax + 1)
    phase = np.exp(1j * np.outer(ks, x))                  # e^{i k x}, (modes, n)
    # x-DFT coefficients of each x-factor; band-limited to |k| <= kmax (checked)
    coef = []
    for j in range(3):
        c = np.conj(phase) @ F[j] / n                     # (modes, rank)
        assert np.allclose(phase.T @ c, F[j], atol=1e-13 * max(1.0, np.abs(F[j]).max()))
        coef.append(c)
    M = np.einsum("a,b,c->abc", m, m, m)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    s = np.sin(ks * hx) / hx
    out = np.zeros((n,) * 6)
    Ex = [phase[:, :, None, None] * np.ones((1, 1, n, n)),
          phase[:, None, :, None] * np.ones((1, n, 1, n)),
          phase[:, None, None, :] * np.ones((1, n, n, 1))]
    for a, k1 in enumerate(ks):
        for b, k2 in enumerate(ks):
            for c, k3 in enumerate(ks):
                amp = w * coef[0][a] * coef[1][b] * coef[2][c]          # (rank,)
                if np.abs(amp).max() == 0.0:
                    continue
                g = np.einsum("t,it,jt,kt->ijk", amp, F[3], F[4], F[5])  # complex v array
                sym = -1j * (V1 * s[a] + V2 * s[b] + V3 * s[c])

                def L(h):
                    return sym * h - nu * h + nu * M * (hv ** 3 * h.sum())
                Lg = L(g)
                gn = g + dt * Lg + 0.5 * dt * dt * L(Lg)
                ex = np.exp(1j * (k1 * x[:, None, None] + k2 * x[None, :, None] + k3 * x[None, None, :]))
                out += np.real(np.einsum("abc,ijk->abcijk", ex, gn))
    return out


def test_heun2_step_matches_x_fourier_mode_closed_form():
    """The oracle's untruncated HT HEUN2 step of the kinetic operator (n = 12, the seeded kinetic
    initial condition, dt = 5x the explicit step) equals the x-mode-wise closed form on the full
    grid to rounding."""
    kc = kinetic_case(12)
    w, F = kinetic_ic(kc)
    dt = 5 * kc.dt
    alphas, factors = kinetic_terms(kc)
    u = OH.from_cp(w, F)
    u1, _ = OH.step_heun2(u, alphas, factors, dt, 0.0, 10 ** 6)
    # the full grid as U_{t1} B_root U_{t2}^T (x dimensions fastest, as in eq. HTD), without the
    # Kronecker product of the two root-child bases
    c1, c2 = u1.tree.children[0]
    full = OH.node_basis(u1, c1) @ u1.node[0] @ OH.node_basis(u1, c2).T
    got = full.reshape((kc.n,) * 6, order="F")
    ref = mode_closed_form_step(kc, w, F, dt)
    f0 = OH.to_full(u)
    assert np.abs(ref - f0).max() > 1e-3 * np.abs(f0).max()       # the step moves f
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def contract(u, vecs):
    """sum over the grid of u * prod_i vecs[i] (complex vectors), leaves to root (eq. HTD)."""
    tr = u.tree
    val = {}
    for t in sorted(range(tr.n_nodes), key=lambda t: -tr.depth[t]):
        X = u.node[t]
        if tr.is_leaf(t):
            val[t] = vecs[tr.lo[t]] @ X
        else:
            a, b = tr.children[t]
            if t == 0:
                return complex(val[a] @ X @ val[b])
            val[t] = np.einsum("a,b,abc->c", val[a], val[b], X)
    raise RuntimeError("unreachable")


def test_full_size_heun2_step_matches_mode_closed_form_on_samples():
    """The same closed form at the kinetic workload's full size (n = 64: no full grid): after
    one untruncated HEUN2 step of the oracle (node ranks up to 222), the x-Fourier coefficient
    f^(K; v) at sampled x-modes K and v-grid points equals p(dt L_K) applied to the mode's
    v-array, to rounding."""
    kc, w, F, _, u1 = full_size_step()
    dt = kc.dt
    n, hx, hv, nu = kc.n, kc.hx, kc.hv, kc.nu
    x, v, m = kc.xgrid(), kc.vgrid(), kc.maxwellian()
    M = np.einsum("a,b,c->abc", m, m, m)
    V1, V2, V3 = np.meshgrid(v, v, v, indexing="ij")
    rng = np.random.default_rng(12)
    modes = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (2, 2, -1), (-1, 1, 1), (1, -2, 0)]
    pts = [(32, 32, 32), (0, 63, 17)] + [tuple(rng.integers(0, n, 3)) for _ in range(10)]
    scale = 0.0
    for K in modes:
        coef = [np.exp(-1j * K[j] * x) @ F[j] / n for j in range(3)]
        g = np.einsum("t,it,jt,kt->ijk", w * coef[0] * coef[1] * coef[2], F[3], F[4], F[5])
        s = [np.sin(k * hx) / hx for k in K]
        sym = -1j * (V1 * s[0] + V2 * s[1] + V3 * s[2])

        def L(h):
            return sym * h - nu * h + nu * M * (hv ** 3 * h.sum())
        Lg = L(g)
        ref = g + dt * Lg + 0.5 * dt * dt * L(Lg)
        scale = max(scale, np.abs(ref).max())
        for p in pts:
            vecs = [np.exp(-1j * K[j] * x) / n for j in range(3)]
            vecs += [np.eye(n)[p[j]] for j in range(3)]
            got = contract(u1, vecs)
            assert abs(got - ref[p]) <= 1e-12 * scale, (K, p)


def moment_vectors(kc):
    """Per dimension the vectors whose product is each moment functional: the x-average of the
    density, the momentum components and the second moment |v|^2 (Section 4.2, eqs. rho0, u0,
    T0 unnormalised)."""
    n, v = kc.n, kc.vgrid()
    a = np.full(n, kc.hx / (2 * np.pi))
    b = np.full(n, kc.hv)
    out = {"rho": [a, a, a, b, b, b]}
    for d in range(3):
        vv = [b, b, b]
        vv[d] = kc.hv * v
        out[f"p{d}"] = [a, a, a] + vv
        vv = [b, b, b]
        vv[d] = kc.hv * v * v
        out[f"e{d}"] = [a, a, a] + vv
    return out


def moments(u, kc):
    m = {k: contract(u, vecs).real for k, vecs in moment_vectors(kc).items()}
    m["e"] = m.pop("e0") + m.pop("e1") + m.pop("e2")
    return m


def test_explicit_steps_relax_the_moments_at_rate_nu():
    """Exponential relaxation at rate nu (Section 4.2), in the discrete form the explicit step
    must reproduce: the kinetic operator keeps the density (l L = 0) and relaxes the momentum
    and E - 3 c2 rho at rate nu (l L = -nu l; c2 = sum_j h v_j^2 m_j), so one untruncated HEUN2
    step, p(dt L) with p(z) = 1 + z + z^2/2, keeps rho and multiplies those by p(-nu dt), to
    rounding.  Full size n = 64, moments by contraction on the format."""
    kc, _, _, u0, u1 = full_size_step()
    dt = kc.dt
    g = 1.0 - kc.nu * dt + 0.5 * (kc.nu * dt) ** 2
    c2 = kc.hv * float(np.sum(kc.vgrid() ** 2 * kc.maxwellian()))
    m0 = moments(u0, kc)
    assert max(abs(m0[f"p{d}"]) for d in range(3)) > 1e-4 * m0["rho"]
    m1 = moments(u1, kc)
    assert abs(m1["rho"] - m0["rho"]) <= 1e-13 * m0["rho"]
    for d in range(3):
        assert abs(m1[f"p{d}"] - g * m0[f"p{d}"]) <= 1e-13 * m0["rho"], d
    assert abs((m1["e"] - 3 * c2 * m1["rho"]) - g * (m0["e"] - 3 * c2 * m0["rho"])) <= 1e-13 * m0["e"]
