"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the CPU oracle.

This module holds only input generation: random draws, grids and the pointwise
values of initial conditions and operator coefficients.  None of the method's
arithmetic (operator application, orthogonalisation, truncation, ALS) lives here,
so the oracle and the CUDA path can both import it without sharing method code.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): the state advances by
0x9E3779B97F4A7C15 and each output is the state passed through two xor-shift-multiply
rounds.  Larger random arrays (random HT / CP tensors for tests) use numpy's PCG64
generator seeded from the same integer seed.

Workloads follow the paper's two problem classes:
- linear advection u_t + c . grad u = 0 on the periodic box [0, 2*pi)^d with a
  sum of separable products exp(sin(x_i + phi_{m,i})) as initial condition
  (Section 4.1 studies advection in six dimensions with a separable initial state);
- the linearised kinetic (BGK-type) equation f_t + v . grad_x f = -nu (f - M(v) rho)
  (Section 4.2, eq. BGK_LIN and Table tab:ordering give the separable operator);
- variable-coefficient advection f_t + sum_j (C z)_j df/dz_j = 0 (Section 4.1, eq. PDE-advR,
  Table tab:ordering0) with the initial condition exp(-|z|^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1
SEED_BASE = 0x5EED


class SplitMix64:
    """splitmix64 stream; uniform() in [0,1) from the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def normal(self) -> float:
        # Box-Muller on two uniforms (first one shifted away from 0).
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class AdvectionCase:
    """Seeded constant-coefficient periodic advection problem.

    Grid: x_j = j*h, h = 2*pi/n (node-centred, periodic).  Velocity c_i ~ U[-1,1].
    Initial condition u0 = sum_m prod_i exp(sin(x_i + phi_{m,i})), phi ~ U[0, 2*pi).
    Draw order: c_1..c_d, then phi term by term, dimension by dimension.
    """

    d: int
    n: int
    n_terms: int
    seed: int
    c: np.ndarray = field(repr=False)
    phi: np.ndarray = field(repr=False)

    @property
    def h(self) -> float:
        return 2.0 * math.pi / self.n

    @property
    def dt(self) -> float:
        return 0.2 * self.h

    def x(self) -> np.ndarray:
        return np.arange(self.n, dtype=np.float64) * self.h

    def ic_factors(self) -> list[np.ndarray]:
        """Per dimension an n x n_terms array: column m holds exp(sin(x + phi_{m,i}))."""
        x = self.x()
        return [np.stack([np.exp(np.sin(x + self.phi[m, i])) for m in range(self.n_terms)], axis=1)
                for i in range(self.d)]


def advection_case(d: int, n: int, n_terms: int = 2, seed: int | None = None, seed_offset: int = 0) -> AdvectionCase:
    if seed is None:
        seed = SEED_BASE + seed_offset
    g = SplitMix64(seed)
    c = np.array([g.uniform_range(-1.0, 1.0) for _ in range(d)])
    phi = np.array([[g.uniform_range(0.0, 2.0 * math.pi) for _ in range(d)] for _ in range(n_terms)])
    return AdvectionCase(d=d, n=n, n_terms=n_terms, seed=seed, c=c, phi=phi)


BATCH_GRIDS = (32, 48, 64, 96, 128)


def batched_advection_cases(count: int, d: int = 6, seed_offset: int = 3):
    """A ragged batch of independent advection problems: per instance (n, r_max, case) with n
    drawn from BATCH_GRIDS and r_max from 8..48 (one splitmix64 stream, seed 0x5EED + seed_offset,
    two draws per instance), and the velocity and phases of instance i from its own seed
    0x5EED + 1000 + i."""
    g = SplitMix64(SEED_BASE + seed_offset)
    out = []
    for i in range(count):
        n = BATCH_GRIDS[int(g.uniform_range(0.0, float(len(BATCH_GRIDS)))) % len(BATCH_GRIDS)]
        rmax = 8 + int(g.uniform_range(0.0, 41.0)) % 41
        out.append((n, rmax, advection_case(d, n, seed=SEED_BASE + 1000 + i)))
    return out


def normal_array(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """N(0, scale^2) array from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)


def normal_arrays(shapes, seed: int, scale: float = 1.0) -> list[np.ndarray]:
    rng = np.random.Generator(np.random.PCG64(seed))
    return [scale * rng.standard_normal(s) for s in shapes]


def cp_random_factors(ns, rank: int, seed: int) -> list[np.ndarray]:
    """Random CP factors, one n_i x rank array per dimension."""
    return normal_arrays([(n, rank) for n in ns], seed)


def cp_padding(ns, n_new: int, seed: int, scale: float) -> list[np.ndarray]:
    """Seeded N(0,1)*scale columns used to pad a CP iterate up to its target rank."""
    g = SplitMix64(seed)
    return [np.array([[scale * g.normal() for _ in range(n_new)] for _ in range(n)]).reshape(n, n_new)
            for n in ns]


# ---------------------------------------------------------------------------
# linearised kinetic equation (x periodic [0,2pi)^3, v in [-6,6]^3)
# ---------------------------------------------------------------------------
@dataclass
class KineticCase:
    """Grids and coefficient vectors for f_t + v.grad_x f = -nu (f - M(v) rho).

    x grid: x_j = j*h_x, h_x = 2*pi/n.  v grid (cell centred): v_j = -6 + (j+1/2)*12/n.
    m: 1-D Maxwellian exp(-v^2/2) normalised so that sum_j h_v m_j = 1.
    w: quadrature weights h_v (rho(x) = sum_v w^3 f).
    """

    n: int
    nu: float
    seed: int

    @property
    def hx(self) -> float:
        return 2.0 * math.pi / self.n

    @property
    def hv(self) -> float:
        return 12.0 / self.n

    def xgrid(self) -> np.ndarray:
        return np.arange(self.n, dtype=np.float64) * self.hx

    def vgrid(self) -> np.ndarray:
        return -6.0 + (np.arange(self.n, dtype=np.float64) + 0.5) * self.hv

    def maxwellian(self) -> np.ndarray:
        g = np.exp(-0.5 * self.vgrid() ** 2)
        return g / (self.hv * g.sum())

    def weights(self) -> np.ndarray:
        return np.full(self.n, self.hv)

    @property
    def dt(self) -> float:
        return 0.2 * self.hx / 6.0


def kinetic_ic(kc: "KineticCase", seed: int | None = None, n_pert: int = 4, amp: float = 1e-2):
    """CP form (weights, factors) of the kinetic initial condition on (x1,x2,x3,v1,v2,v3):
    f0 = M(v) (1 + 0.1 prod_i sin(x_i)) plus a seeded rank-n_pert perturbation whose x-factors
    are band-limited (Fourier modes |k| <= 2) and whose v-factors are m(v) times a polynomial of
    degree <= 2 (splitmix64 coefficients in [-1, 1]); each perturbation term is scaled to
    max-norm amp.  M = m^(x3) with the case's discretely normalised Maxwellian m."""
    g = SplitMix64(kc.seed + 7 if seed is None else seed)
    x, v, m = kc.xgrid(), kc.vgrid(), kc.maxwellian()
    ones = np.ones_like(x)
    weights = [1.0, 0.1]
    factors = [[ones, ones, ones, m, m, m], [np.sin(x), np.sin(x), np.sin(x), m, m, m]]
    for _ in range(n_pert):
        fs = []
        for _i in range(3):
            f = np.zeros_like(x)
            for k in range(3):
                a, b = g.uniform_range(-1.0, 1.0), g.uniform_range(-1.0, 1.0)
                f = f + a * np.cos(k * x) + b * np.sin(k * x)
            fs.append(f)
        for _i in range(3):
            c0, c1, c2 = (g.uniform_range(-1.0, 1.0) for _ in range(3))
            fs.append(m * (c0 + c1 * v + c2 * v * v))
        scale = float(np.prod([np.abs(f).max() for f in fs]))
        weights.append(amp / scale if scale > 0 else 0.0)
        factors.append(fs)
    F = [np.stack([t[i] for t in factors], axis=1) for i in range(6)]
    return np.array(weights), F


def kinetic_case(n: int, nu: float = 1.0, seed: int | None = None, seed_offset: int = 2) -> KineticCase:
    if seed is None:
        seed = SEED_BASE + seed_offset
    return KineticCase(n=n, nu=nu, seed=seed)


# the paper's evaluation point z* = (h, ..., h) of the pointwise error (Section 4.1)
Z_STAR = 0.698835274542439


@dataclass
class VarCoefCase:
    """Seeded variable-coefficient advection problem f_t + sum_j (C z)_j df/dz_j = 0 on the
    periodic box [-zmax, zmax)^N (Section 4.1, eq. PDE-advR; the paper uses zmax = 60).

    Grid: z_j = -zmax + j h, h = 2 zmax / n.  C = S + K with S = diag(s_i), s_i ~ U[0.5, 1],
    and K skew, K_jk = (a_jk - a_kj) / 2 with a_jk ~ U[-1, 1] (draw order: s_1..s_N, then a row
    by row): every eigenvalue of C has real part in [0.5, 1] (for a unit eigenvector x,
    x^* K x is imaginary), so exp(-tC) contracts as in the paper's experiment.  Initial
    condition exp(-|z|^2), separable of rank 1.  dt = cfl h / (zmax max_j sum_k |C_jk|), the
    largest transport speed on the box.
    """

    N: int
    n: int
    zmax: float
    seed: int
    cfl: float
    C: np.ndarray = field(repr=False)

    @property
    def h(self) -> float:
        return 2.0 * self.zmax / self.n

    @property
    def dt(self) -> float:
        vmax = self.zmax * float(np.abs(self.C).sum(axis=1).max())
        return self.cfl * self.h / vmax

    def z(self) -> np.ndarray:
        return -self.zmax + np.arange(self.n, dtype=np.float64) * self.h

    def ic_factors(self) -> list[np.ndarray]:
        """Per dimension an n x 1 array exp(-z^2)."""
        return [np.exp(-self.z() ** 2)[:, None] for _ in range(self.N)]

    def star_index(self) -> int:
        """Grid index nearest to the paper's evaluation coordinate h = 0.698835274542439."""
        return int(np.argmin(np.abs(self.z() - Z_STAR)))


def varcoef_case(N: int, n: int, zmax: float = 60.0, cfl: float = 0.2, seed: int | None = None,
                 seed_offset: int = 5) -> VarCoefCase:
    if seed is None:
        seed = SEED_BASE + seed_offset
    g = SplitMix64(seed)
    s = [g.uniform_range(0.5, 1.0) for _ in range(N)]
    a = np.array([[g.uniform_range(-1.0, 1.0) for _ in range(N)] for _ in range(N)])
    C = np.diag(s) + 0.5 * (a - a.T)
    return VarCoefCase(N=N, n=n, zmax=zmax, seed=seed, cfl=cfl, C=C)
