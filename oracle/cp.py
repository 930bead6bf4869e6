"""Canonical (CP) tensors and alternating least squares for the oracle (FP64).

CP format (Section 2.1, eq. functional-SSE): u = sum_l lambda_l prod_k X_k[:, l]; on
the grid each X_k is n_k x r (the coefficient vectors beta of eq. gfun with the grid
basis).  The ALS mode update (eqs. als, SSYSTEM, A^{ln}_{jhp}, f_{jh}^n) minimises
|y - x| over the factor of one dimension k with the others fixed.  On an orthonormal
grid basis the mass matrix (phi_h, phi_s) is a multiple of the identity, so the
normal equations become

  X_k Gamma_k = Y_k diag(mu) H_k,
  Gamma_k = hadamard_{j != k} X_j^T X_j   (r x r, the A_j of eq. SSYSTEM),
  H_k     = hadamard_{j != k} Y_j^T X_j   (R_y x r, the right-hand side g_j),

solved with a Cholesky factorisation of Gamma_k.

Sweep order: Gauss-Seidel over k = 1..d (Section 3.1, the ALS as block Gauss-Seidel).
Variant 'jacobi_damped' follows Appendix B, Algorithm 1: every mode is solved from the
same iterate, the increment is damped by 1/4, and the convergence measure of
Algorithm 5 is max_k |X_k^new - X_k^int| / |X_k^int|.

Parity: pinned by tests -- a mode update equals the brute-force least-squares solution
over the unfolded full grid (library lstsq); the residual never increases under
Gauss-Seidel; an exact rank-r target with exact initial factors is a fixed point;
a rank-1 target is recovered by the rank-1 iteration (higher-order power method); the
damped-Jacobi sweep is a quarter step from one iterate; a singular Gamma_k takes the
shift and keeps the fit; `residual` equals |to_full(y) - to_full(x)|_F formed on the grid;
`apply_kron_sum_rk2` equals the fully discrete Fourier closed form; `pad` with zero
padding keeps the tensor; `step_rk2`'s rank-24 fit at n = 64 stays within that residual
(the advection-mode tests).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CP:
    """sum_l weights[l] prod_k factors[k][:, l] (Section 2.1, eq. functional-SSE)."""
    weights: np.ndarray        # (r,)
    factors: list              # d arrays n_k x r

    @property
    def rank(self) -> int:
        return self.weights.shape[0]

    @property
    def d(self) -> int:
        return len(self.factors)

    def copy(self) -> "CP":
        return CP(self.weights.copy(), [f.copy() for f in self.factors])


def to_full(x: CP) -> np.ndarray:
    """The grid values of eq. functional-SSE, term by term (small grids only)."""
    shape = tuple(f.shape[0] for f in x.factors)
    out = np.zeros(shape)
    for l in range(x.rank):
        term = np.array(x.weights[l])
        for f in x.factors:
            term = np.multiply.outer(term, f[:, l])
        out += term
    return out


def normalize(x: CP) -> CP:
    """Unit factor columns, norms collected in the weights (the lambda_l of eq.
    functional-SSE, Section 2.1)."""
    w = x.weights.copy()
    fs = []
    for f in x.factors:
        nr = np.linalg.norm(f, axis=0)
        safe = np.where(nr > 0, nr, 1.0)
        fs.append(f / safe[None, :])
        w = w * np.where(nr > 0, nr, 1.0)
    return CP(w, fs)


def apply_kron_sum_rk2(x: CP, A: list) -> CP:
    """y = p(S) x, S = sum_i A_i, p(z) = 1 + z + z^2/2, exactly in CP form.

    p(S) = I + sum_i A_i + 1/2 sum_i A_i^2 + sum_{i<j} A_i A_j, so every rank-1 term of x
    becomes 1 + 2d + d(d-1)/2 rank-1 terms (eq. Lz applied term by term).  Column order:
    term type major, original rank index minor.
    """
    d = x.d
    types = [()] + [(i,) for i in range(d)] + [(i, i) for i in range(d)] + \
            [(i, j) for i in range(d) for j in range(i + 1, d)]
    ws, fs = [], [[] for _ in range(d)]
    for ty in types:
        coef = 0.5 if (len(ty) == 2 and ty[0] == ty[1]) else 1.0
        ws.append(coef * x.weights)
        for k in range(d):
            Xk = x.factors[k]
            p = ty.count(k)
            for _ in range(p):
                Xk = A[k] @ Xk
            fs[k].append(Xk)
    return CP(np.concatenate(ws), [np.hstack(f) for f in fs])


def _mode_solve(y: CP, x_factors: list, k: int):
    """Unnormalised minimiser X_k of |y - sum_l prod_j X_j[:, l]| (others fixed): the
    normal equations of eqs. SSYSTEM and A^{ln}_{jhp} on the grid basis (Section 2.1)."""
    d = len(x_factors)
    r = x_factors[0].shape[1]
    Gam = np.ones((r, r))
    H = np.ones((y.rank, r))
    for j in range(d):
        if j == k:
            continue
        Gam *= x_factors[j].T @ x_factors[j]
        H *= y.factors[j].T @ x_factors[j]
    rhs = y.factors[k] @ (y.weights[:, None] * H)          # n_k x r
    try:
        L = np.linalg.cholesky(Gam)                          # Gam = L L^T
    except np.linalg.LinAlgError:
        # Section 2.1: poorly conditioned ALS matrices are regularised; shift only on failure
        L = np.linalg.cholesky(Gam + (1e-14 * np.trace(Gam) / r) * np.eye(r))
    Z = np.linalg.solve(L, rhs.T)                            # forward substitution
    return np.linalg.solve(L.T, Z).T                         # back substitution


def als_sweeps(y: CP, x0: CP, sweeps: int, variant: str = "gs"):
    """ALS rank reduction of y starting from x0 (Section 2.1, eq. als; Gauss-Seidel order of
    Section 3.1; damped Jacobi of Appendix B, Algorithm 1).  Returns (x, eps_conv per sweep).

    Gauss-Seidel ('gs'): for k = 1..d, normalise the other factors, solve the mode-k
    normal equations, then split the solution into unit columns and weights.
    'jacobi_damped': all modes from the same (unnormalised) iterate, damped 1/4.
    """
    d = y.d
    x = normalize(x0)
    eps_hist = []
    if variant == "gs":
        for _ in range(sweeps):
            eps = 0.0
            for k in range(d):
                scaled_old = x.factors[k] * x.weights[None, :]
                Xt = _mode_solve(y, x.factors, k)
                dn = np.linalg.norm(Xt - scaled_old)
                den = np.linalg.norm(scaled_old)
                eps = max(eps, dn / den if den > 0 else dn)
                nr = np.linalg.norm(Xt, axis=0)
                safe = np.where(nr > 0, nr, 1.0)
                x.factors[k] = Xt / safe[None, :]
                x.weights = nr
            eps_hist.append(eps)
        return x, eps_hist
    if variant == "jacobi_damped":
        # unnormalised iterate: weights folded into the first factor (Algorithm 1 keeps beta only)
        fac = [f.copy() for f in x.factors]
        fac[0] = fac[0] * x.weights[None, :]
        for _ in range(sweeps):
            new = [_mode_solve(y, fac, k) for k in range(d)]
            eps = max(np.linalg.norm(new[k] - fac[k]) / np.linalg.norm(fac[k]) for k in range(d))
            fac = [fac[k] + (new[k] - fac[k]) / 4.0 for k in range(d)]
            eps_hist.append(eps)
        return normalize(CP(np.ones(fac[0].shape[1]), fac)), eps_hist
    raise ValueError(variant)


def pad(x: CP, r_target: int, padding: list) -> CP:
    """Append r_target - r columns (given seeded arrays, weight 1) to every factor: the
    initialisation the ALS rank reduction needs at every step (Section 4.1)."""
    r = x.rank
    if r >= r_target:
        return x.copy()
    m = r_target - r
    xn = normalize(x)
    return CP(np.concatenate([xn.weights, np.ones(m)]),
              [np.hstack([f, p[:, :m]]) for f, p in zip(xn.factors, padding)])


def residual(y: CP, x: CP) -> float:
    """|y - x| via factor Grams (no full grid): the error the ALS of Section 2.1 minimises."""
    def gram(a: CP, b: CP):
        G = np.outer(a.weights, b.weights)
        for fa, fb in zip(a.factors, b.factors):
            G = G * (fa.T @ fb)
        return G.sum()
    v = gram(y, y) - 2 * gram(y, x) + gram(x, x)
    return float(np.sqrt(max(v, 0.0)))


def step_rk2(x: CP, A: list, r_target: int, padding: list, sweeps: int, variant: str = "gs"):
    """One CP step: y = p(dt L) x exactly, then ALS rank reduction of y from the warm
    start x padded to r_target columns (Section 3.2 with ALS as the rank reduction)."""
    y = apply_kron_sum_rk2(x, A)
    rt = min(r_target, y.rank)
    x0 = pad(x, rt, padding) if x.rank < rt else x.copy()
    return als_sweeps(y, x0, sweeps, variant)
