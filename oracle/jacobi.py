"""One-sided (Hestenes) Jacobi SVD, written out for the oracle.

The hierarchical SVD the paper cites (Section 2.2, rank reduction by HSVD) needs the
leading singular vectors of every node matricisation.  This routine computes the
SVD of an m x k matrix A (m >= k after the caller's QR) by orthogonalising its
columns with plane rotations:

  for a column pair (p, q): alpha = |a_p|^2, beta = |a_q|^2, gamma = a_p . a_q;
  if |gamma| > tol * sqrt(alpha beta) (tol = eps * max(m, 8), the rounding level of a
  length-m dot product) and both columns are above the rounding floor eps * |A|_F (a
  column below it carries no information, and rotating it only reshuffles rounding noise,
  which would keep the sweeps from terminating on rank-deficient matrices):
  zeta = (beta - alpha) / (2 gamma),
  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = c t,
  [a_p, a_q] <- [c a_p - s a_q, s a_p + c a_q]  (same rotation on V).

Pairs are visited in the round-robin (Brent-Luk) order: each round rotates k/2
disjoint pairs, k-1 rounds make a sweep, sweeps repeat until no pair rotates.
On exit sigma_j = |a_j|, U = A V diag(1/sigma), sorted by decreasing sigma.

Parity: pinned by tests (numpy/LAPACK singular values, reconstruction, orthogonality,
matrices with known singular values).
"""
from __future__ import annotations

import numpy as np


def _round_robin(k: int):
    """Brent-Luk tournament: list of rounds, each a pair of index arrays (p, q) (the pair order
    of the node SVDs of the HSVD, Section 2.2)."""
    m = k + (k % 2)
    players = list(range(m))
    rounds = []
    for _ in range(m - 1):
        ps, qs = [], []
        for i in range(m // 2):
            a, b = players[i], players[m - 1 - i]
            if a < k and b < k:
                ps.append(min(a, b))
                qs.append(max(a, b))
        rounds.append((np.array(ps, dtype=np.int64), np.array(qs, dtype=np.int64)))
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_svd(A: np.ndarray, tol: float | None = None, max_sweeps: int = 60):
    """Return (U, s, V) with A = U diag(s) V^T, s descending; A is m x k with m >= k (a node
    SVD of the HSVD, Section 2.2)."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, k = A.shape
    if tol is None:
        tol = np.finfo(np.float64).eps * max(m, 8)
    if m < k:
        raise ValueError("jacobi_svd expects m >= k (QR-reduce wide matrices first)")
    V = np.eye(k)
    floor2 = (np.finfo(np.float64).eps ** 2) * float(np.sum(A * A))
    if k > 1:
        rounds = _round_robin(k)
        for _ in range(max_sweeps):
            rotated = False
            for p, q in rounds:
                if p.size == 0:
                    continue
                ap, aq = A[:, p], A[:, q]
                alpha = np.einsum("ij,ij->j", ap, ap)
                beta = np.einsum("ij,ij->j", aq, aq)
                gamma = np.einsum("ij,ij->j", ap, aq)
                act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
                act &= gamma != 0.0
                act &= (alpha > floor2) & (beta > floor2)
                if not act.any():
                    continue
                rotated = True
                p, q = p[act], q[act]
                alpha, beta, gamma = alpha[act], beta[act], gamma[act]
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
            if not rotated:
                break
    s = np.sqrt(np.einsum("ij,ij->j", A, A))
    order = np.argsort(-s, kind="stable")
    s = s[order]
    A = A[:, order]
    V = V[:, order]
    U = np.zeros_like(A)
    nz = s > 0
    U[:, nz] = A[:, nz] / s[nz]
    return U, s, V


def svd_left(F: np.ndarray):
    """Left singular vectors and values of a (possibly wide) matrix F (k x m) (Section 2.2).

    F^T = Q R (QR as a library step) reduces the problem to R^T (k x k'), whose SVD
    R^T = U S W^T gives F = U S (Q W)^T.  Returns (U, s) with U k x k (padded with an
    orthonormal completion when k' < k) and s of length k (zeros appended).
    """
    k, m = F.shape
    if m > k:
        Q, R = np.linalg.qr(F.T, mode="reduced")   # R: k x k
        M = R.T
    else:
        M = F
    kk = M.shape[1]
    if kk < k:
        M = np.hstack([M, np.zeros((k, k - kk))])
    # SVD of M (k x k): one-sided Jacobi on M^T gives M^T = Z S U^T.
    Z, s, U = jacobi_svd(M.T)
    return U, s
