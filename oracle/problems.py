"""Operator matrices of the two model problems for the oracle (dense, plain numpy).

- Advection u_t + c . grad u = 0 (Section 4.1 with constant coefficients): L = sum_i L_i,
  L_i = -c_i D on dimension i, D the periodic central difference.  ``advection_A``
  returns the step matrices dt*L_i used by the RK2 polynomial form.
- Linearised kinetic equation f_t + v . grad_x f = -nu (f - M(v) rho) (Section 4.2,
  eq. BGK_LIN; Table tab:ordering lists its separable terms): dimensions
  (x1, x2, x3, v1, v2, v3) and five terms
    q = 1..3: alpha = -1,   D on x_i, diag(v) on v_i;
    q = 4:    alpha = -nu,  identity;
    q = 5:    alpha = +nu,  (m w^T) on each v dimension (rho = sum_v w^3 f, M = m^{x3}).

- Variable-coefficient advection f_t + sum_j (sum_k C_jk z_k) df/dz_j = 0 (Section 4.1, eq.
  PDE-advR; Table tab:ordering0 orders its N^2 separable terms): term q = (j-1) N + k has
  alpha_q = -C_jk, the derivative D on dimension j and multiplication by z on dimension k
  (for k = j the single factor diag(z) D on dimension j), identity elsewhere.

Parity: pinned by tests (dense Kronecker operator on tiny grids; exact conservation of
the weighted mass; the Maxwellian is a fixed point of the collision terms; the paper's
term tables as golden files; the advection operator on exp(-|z|^2) against its closed form
2 (z^T C z) exp(-|z|^2) within the central-difference error).
"""
from __future__ import annotations

import numpy as np

from .ht import central_diff_matrix


def advection_A(case) -> list:
    """dt L_i = -dt c_i D on dimension i: the Kronecker-sum terms of eq. Lz for constant-
    coefficient advection (Section 4.1)."""
    D = central_diff_matrix(case.n, case.h)
    return [case.dt * (-case.c[i]) * D for i in range(case.d)]


def kinetic_terms(kc):
    """(alphas, factors) of the kinetic operator on (x1,x2,x3,v1,v2,v3); None = identity
    (Section 4.2, eq. BGK_LIN; terms of Table tab:ordering)."""
    n = kc.n
    D = central_diff_matrix(n, kc.hx)
    V = np.diag(kc.vgrid())
    P1 = np.outer(kc.maxwellian(), kc.weights())
    alphas, factors = [], []
    for i in range(3):
        f = [None] * 6
        f[i] = D
        f[3 + i] = V
        alphas.append(-1.0)
        factors.append(f)
    alphas.append(-kc.nu)
    factors.append([None] * 6)
    alphas.append(kc.nu)
    factors.append([None, None, None, P1, P1, P1])
    return alphas, factors


def varcoef_terms(case):
    """(alphas, factors) of -sum_j (C z)_j d/dz_j in the order of Table tab:ordering0:
    q = (j-1) N + k (1-based j, k) carries -C_jk; None = identity."""
    N, n = case.N, case.n
    D = central_diff_matrix(n, case.h)
    Z = np.diag(case.z())
    alphas, factors = [], []
    for j in range(N):
        for k in range(N):
            f = [None] * N
            if k == j:
                f[j] = Z @ D
            else:
                f[j] = D
                f[k] = Z
            alphas.append(-float(case.C[j, k]))
            factors.append(f)
    return alphas, factors
