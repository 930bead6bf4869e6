"""Crank-Nicolson step solved by CP alternating least squares, for the oracle (FP64, numpy).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU legs use it.

Section 3.3 (eqs. CNFDE, BLs, rRr1, ALS2, ML, MR, eq:77).  With L = sum_q alpha_q prod_k L_k^q
the Crank-Nicolson operators are separable:
    A = I - dt/2 L = sum_{e=0}^{rL} eta_e  prod_k E_k^e,   B = I + dt/2 L = sum_e zeta_e prod_k E_k^e,
E^0 the identity (eta_0 = zeta_0 = 1), E^e the e-th term of L, eta_e = -dt/2 alpha_e and
zeta_e = +dt/2 alpha_e.  One step minimises |A x - B x_n| over the factors of a CP tensor x of
fixed rank r, one dimension q at a time (Gauss-Seidel, q = 1..d, repeated `sweeps` times).
With the other factors fixed, the normal equations of dimension q (eq. ALS2) are, on the grid
basis (the 1-D integrals of eq:77 become grid products S^{ez} = (E_q^e)^T E_q^z),
    sum_{e,z} eta_e eta_z  S^{ez} V Gamma^{ezT} = sum_{e,z} eta_e zeta_z  S^{ez} Xn_q diag(lam_n) Gn^{ezT},
    Gamma^{ez} = hadamard_{k != q} (E_k^e X_k)^T (E_k^z X_k)        (r x r, eq. ML),
    Gn^{ez}    = hadamard_{k != q} (E_k^e X_k)^T (E_k^z Xn_k)       (r x r_n, eq. MR),
i.e. M vec(V) = vec(R) with M = sum eta_e eta_z Gamma^{ez} kron S^{ez} ((n r) x (n r), SPD;
vec column major, index i + n l), solved by Cholesky; V is the new factor X_q.  The weights of
the initial guess are folded into its first factor, so x carries unit weights.  Convergence
measure of a sweep: max over q of |X_q^new - X_q^old|^2 (the paper's increment criterion).

Parity: pinned by tests -- a mode solve equals brute-force least squares over the full grid
(library lstsq on the unfolded A); pure relaxation L = -nu I gives the closed form
(1 - nu dt/2)/(1 + nu dt/2) x_n; a spatially uniform Maxwellian is a fixed point of the
kinetic operator; the residual never increases from one mode solve to the next; an x-uniform
state relaxes to the rank-2 closed form g f0 + (1 - g) rho M; the exact full-grid step with
these eta / zeta keeps the density and multiplies the momentum and E - 3 c2 rho by g; from the
Maxwellian the density, velocity and temperature (Section 4.2, eqs. rho0, u0, T0) stay constant.
"""
from __future__ import annotations

import numpy as np

from .cp import CP


def cn_terms(alphas: list, factors: list, dt: float, d: int):
    """(eta, zeta, E): E[e][k] the 1-D factor of term e on dimension k (None = identity).
    A = I - dt/2 L and B = I + dt/2 L as separable sums with the identity as term 0
    (Section 3.3, eqs. CNFDE and BLs)."""
    eta = [1.0] + [-0.5 * dt * a for a in alphas]
    zeta = [1.0] + [0.5 * dt * a for a in alphas]
    E = [[None] * d] + [list(f) for f in factors]
    return eta, zeta, E


def _ap(F, X):
    """F X for a 1-D factor F of eq. BLs (None = the identity), Section 3.3."""
    return X if F is None else F @ X


def mode_system(X: list, xn: CP, eta, zeta, E, q: int):
    """M ((n r) x (n r)) and R (n x r) of the normal equations of dimension q (Section 3.3,
    eqs. ALS2, ML, MR, with eq:77's integrals as grid products)."""
    d = len(X)
    n, r = X[q].shape
    T = len(eta)
    Y = [[_ap(E[e][k], X[k]) for k in range(d)] for e in range(T)]
    Yn = [[_ap(E[e][k], xn.factors[k]) for k in range(d)] for e in range(T)]
    M = np.zeros((n * r, n * r))
    R = np.zeros((n, r))
    XnW = xn.factors[q] * xn.weights[None, :]
    for e in range(T):
        Ee = np.eye(n) if E[e][q] is None else E[e][q]
        for z in range(T):
            Ez = np.eye(n) if E[z][q] is None else E[z][q]
            Gam = np.ones((r, r))
            Gn = np.ones((r, xn.rank))
            for k in range(d):
                if k != q:
                    Gam = Gam * (Y[e][k].T @ Y[z][k])
                    Gn = Gn * (Y[e][k].T @ Yn[z][k])
            S = Ee.T @ Ez
            M += eta[e] * eta[z] * np.kron(Gam, S)
            R += eta[e] * zeta[z] * (S @ XnW @ Gn.T)
    return M, R


def mode_solve(X: list, xn: CP, eta, zeta, E, q: int) -> np.ndarray:
    """The new factor of dimension q: M vec(V) = vec(R) of eq. ALS2 solved by Cholesky
    (Section 3.3)."""
    M, R = mode_system(X, xn, eta, zeta, E, q)
    n, r = X[q].shape
    Lc = np.linalg.cholesky(M)
    y = np.linalg.solve(Lc, R.reshape(-1, order="F"))
    v = np.linalg.solve(Lc.T, y)
    return v.reshape(n, r, order="F")


def cn_als_step(xn: CP, x0: CP, alphas: list, factors: list, dt: float, sweeps: int, variant: str = "gs"):
    """x_{n+1} of rank x0.rank from the initial guess x0; returns (x, eps per sweep).

    variant "gs": Gauss-Seidel, each mode solved with the modes before it already updated.
    variant "jacobi_damped": the parallel ALS of Appendix B (Algorithm 1): every mode solved from
    the same iterate X^int, then X_q <- X_q^int + (V_q - X_q^int) / 4 for all q.  eps is the
    largest |V_q - X_q^old|^2 of the sweep in both variants."""
    d = xn.d
    eta, zeta, E = cn_terms(alphas, factors, dt, d)
    X = [f.copy() for f in x0.factors]
    X[0] = X[0] * x0.weights[None, :]
    eps = []
    for _ in range(sweeps):
        e_max = 0.0
        if variant == "gs":
            for q in range(d):
                V = mode_solve(X, xn, eta, zeta, E, q)
                e_max = max(e_max, float(np.sum((V - X[q]) ** 2)))
                X[q] = V
        elif variant == "jacobi_damped":
            Vs = [mode_solve(X, xn, eta, zeta, E, q) for q in range(d)]
            for q in range(d):
                e_max = max(e_max, float(np.sum((Vs[q] - X[q]) ** 2)))
                X[q] = X[q] + 0.25 * (Vs[q] - X[q])
        else:
            raise ValueError(variant)
        eps.append(e_max)
    return CP(np.ones(x0.rank), X), eps


def cn_residual(x: CP, xn: CP, alphas: list, factors: list, dt: float) -> float:
    """|A x - B x_n| on the full grid (small grids only): the functional the ALS step of
    Section 3.3 minimises (eqs. CNFDE, BLs)."""
    from .cp import to_full
    d = x.d
    eta, zeta, E = cn_terms(alphas, factors, dt, d)

    def apply_full(u, coefs):
        out = np.zeros_like(u)
        for c, Ee in zip(coefs, E):
            v = u
            for k, F in enumerate(Ee):
                if F is not None:
                    v = np.moveaxis(np.tensordot(F, v, axes=([1], [k])), 0, k)
            out += c * v
        return out

    return float(np.linalg.norm(apply_full(to_full(x), eta) - apply_full(to_full(xn), zeta)))
