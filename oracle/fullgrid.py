"""Full-grid FD stepper for small grids (oracle for the apply step).

Discretisation (the configurations' reading of Section 3.2 with eq. PDE0 and the
advection problem eq. PDE-advR at constant coefficients):
- periodic node-centred grid x_j = j h, h = 2 pi / n;
- (D u)_j = (u_{j+1} - u_{j-1}) / (2h) along one axis, indices mod n;
- L = - sum_i c_i D_i  (u_t + c . grad u = 0);
- one explicit two-stage second-order Runge-Kutta step on the linear ODE u' = L u,
  which for every such scheme is u <- u + dt L u + dt^2/2 L(L u).

Parity: pinned by tests against the fully discrete Fourier closed form
u_n = F^{-1}[ R(dt lambda(k))^n F u_0 ], lambda(k) = -i sum_j c_j sin(k_j h)/h,
R(z) = 1 + z + z^2/2; and by exact mass conservation.
"""
from __future__ import annotations

import numpy as np


def central_diff(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """(u_{j+1} - u_{j-1}) / (2h) along `axis`, periodic (the FD reading of eq. PDE0)."""
    return (np.roll(u, -1, axis=axis) - np.roll(u, 1, axis=axis)) / (2.0 * h)


def apply_L(u: np.ndarray, c, h) -> np.ndarray:
    """L u = -sum_i c_i D_i u, the constant-coefficient case of eq. PDE-advR (Section 4.1)."""
    out = np.zeros_like(u)
    for i in range(u.ndim):
        hi = h[i] if np.ndim(h) else h
        out -= c[i] * central_diff(u, i, hi)
    return out


def rk2_step(u: np.ndarray, c, h, dt: float) -> np.ndarray:
    """u + dt L u + dt^2/2 L(L u): a two-stage second-order explicit step of u' = L u
    (Section 3.2)."""
    Lu = apply_L(u, c, h)
    return u + dt * Lu + 0.5 * dt * dt * apply_L(Lu, c, h)


def rk2_steps(u: np.ndarray, c, h, dt: float, steps: int) -> np.ndarray:
    """`steps` repetitions of rk2_step (Section 3.2)."""
    for _ in range(steps):
        u = rk2_step(u, c, h, dt)
    return u


def ab2_step(u: np.ndarray, u_prev: np.ndarray, c, h, dt: float) -> np.ndarray:
    """The two-step Adams-Bashforth scheme of eq. AB2_: u + dt (3/2 L u - 1/2 L u_prev)."""
    return u + dt * (1.5 * apply_L(u, c, h) - 0.5 * apply_L(u_prev, c, h))


def cp_to_full(weights, factors) -> np.ndarray:
    """sum_l w_l prod_k X_k[:, l] on the full grid (eq. functional-SSE)."""
    shape = tuple(f.shape[0] for f in factors)
    out = np.zeros(shape)
    for l in range(factors[0].shape[1]):
        term = np.array(weights[l], dtype=np.float64)
        for f in factors:
            term = np.multiply.outer(term, f[:, l])
        out += term
    return out
