"""Hierarchical Tucker (HT) tensors for the oracle: FP64, plain numpy, no blocking.

Representation (Section 2.2, eqs. HTD / coreT): on the balanced dimension tree of
``oracle.tree`` every node t has a rank k_t.
- leaf t = {i}:      U_t, an n_i x k_t matrix (tensor components T^{i});
- interior t=(t1,t2): transfer tensor B_t with shape (k_t1, k_t2, k_t);
- root:              B_root with shape (k_t1, k_t2)   (the paper's A^{1}).
The node basis is U_t = (U_t2 kron U_t1) B_t with B_t reshaped (k_t1 k_t2) x k_t in
Fortran order, so row index = multi-index of the node's dimensions, first fastest.
The full tensor is U_root reshaped to (n_0, ..., n_{d-1}).

Operations (the paper lists addition, orthogonalisation, rank reduction, scalar
products and linear transforms as the HT toolkit it relies on, Section 2.2; the
explicit step of Section 3.2, eq. AB2_, needs addition, operator application and
rank reduction):
- ``apply_kron_sum_rk2``   v = p(dt L) u, p(z) = 1 + z + z^2/2, for L = sum_i L_i (eq. Lz
                            with one factor per term differing from the identity);
- ``apply_separable``      v = sum_q alpha_q (kron_i A_i^q) u for a general separable
                            operator (eq. Lz);
- ``add``                  a u + b w (ranks add, block-diagonal transfers; Section 3.2);
- ``orthogonalize``        leaves by QR, transfer tensors bottom-up;
- ``truncate``             root-to-leaves hierarchical SVD (HSVD, Section 2.2 and 3.2);
- ``norm``, ``inner``, ``mass``.

Parity: pinned by tests -- to_full vs brute-force CP evaluation; apply vs the
Fourier closed form of the fully discrete scheme; truncate vs Eckart-Young (d = 2),
exact recovery of separable inputs, brute-force projector products built from full
matricisation SVDs, the HSVD error bounds and idempotence; add, inner, norm and mass
vs the same operations on the full grid; step_rk2_poly, step_ab2 and step_heun2 vs the
full-grid steppers and the Fourier / kinetic x-mode closed forms; step_ab2_split,
untruncated, vs the full-grid AB2 step and, truncated, within the propagated HSVD bound.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .jacobi import svd_left
from .tree import Tree, build_tree


@dataclass
class HT:
    """Nodes of an HT tensor on a dimension tree (Section 2.2, eqs. HTD / coreT)."""
    tree: Tree
    n: list
    node: dict = field(default_factory=dict)   # t -> ndarray

    def copy(self) -> "HT":
        return HT(self.tree, list(self.n), {t: a.copy() for t, a in self.node.items()})

    def rank(self, t: int) -> int:
        tr = self.tree
        if t == 0:
            return 1
        if tr.is_leaf(t):
            return self.node[t].shape[1]
        return self.node[t].shape[2]

    def ranks(self) -> list:
        return [self.rank(t) for t in range(self.tree.n_nodes)]


# ---------------------------------------------------------------------------
# construction and full evaluation
# ---------------------------------------------------------------------------
def from_cp(weights, factors, tree: Tree | None = None) -> HT:
    """Exact HT form of a CP tensor sum_l w_l prod_i X_i[:, l].

    A CP tensor is the fully diagonal case of the hierarchical Schmidt form (footnote to
    eq. HTD): leaves are the factor matrices, interior transfer tensors are the diagonal
    B[a,b,c] = delta_abc and the root is diag(w).
    """
    d = len(factors)
    tree = tree or build_tree(d)
    r = factors[0].shape[1]
    ht = HT(tree, [f.shape[0] for f in factors])
    for t in range(tree.n_nodes):
        if tree.is_leaf(t):
            ht.node[t] = np.array(factors[tree.lo[t]], dtype=np.float64)
        elif t == 0:
            ht.node[t] = np.diag(np.asarray(weights, dtype=np.float64))
        else:
            B = np.zeros((r, r, r))
            for a in range(r):
                B[a, a, a] = 1.0
            ht.node[t] = B
    return ht


def node_basis(ht: HT, t: int) -> np.ndarray:
    """U_t = (U_t2 kron U_t1) B_t  (eq. HTD, recursively)."""
    tr = ht.tree
    if tr.is_leaf(t):
        return ht.node[t]
    c1, c2 = tr.children[t]
    U1 = node_basis(ht, c1)
    U2 = node_basis(ht, c2)
    B = ht.node[t]
    k1, k2 = B.shape[0], B.shape[1]
    k = 1 if t == 0 else B.shape[2]
    return np.kron(U2, U1) @ B.reshape(k1 * k2, k, order="F")


def to_full(ht: HT) -> np.ndarray:
    """The grid values: the root basis of eq. HTD reshaped to the grid (small grids only)."""
    return node_basis(ht, 0).reshape(tuple(ht.n), order="F")


def matricize(full: np.ndarray, dims: list) -> np.ndarray:
    """Node matricisation: rows = dims (first fastest), columns = the rest (the t-unfolding
    whose singular values the HSVD of Section 2.2 takes)."""
    rest = [i for i in range(full.ndim) if i not in dims]
    nr = int(np.prod([full.shape[i] for i in dims]))
    return full.transpose(dims + rest).reshape(nr, -1, order="F")


# ---------------------------------------------------------------------------
# 1-D operators
# ---------------------------------------------------------------------------
def central_diff_matrix(n: int, h: float) -> np.ndarray:
    """(D u)_j = (u_{j+1} - u_{j-1}) / (2h), periodic: the 1-D derivative factor of eq. Lz
    on the grid."""
    D = np.zeros((n, n))
    for j in range(n):
        D[j, (j + 1) % n] += 1.0 / (2.0 * h)
        D[j, (j - 1) % n] -= 1.0 / (2.0 * h)
    return D


# ---------------------------------------------------------------------------
# operator application (eq. Lz; explicit step, Section 3.2)
# ---------------------------------------------------------------------------
_BINOM = [[1], [1, 1], [1, 2, 1]]
_POLY = [1.0, 1.0, 0.5]   # p(z) = 1 + z + z^2/2


def apply_kron_sum_poly(ht: HT, A: list, coeffs) -> HT:
    """v = q(S) u with S = sum_i A_i (A_i acts on dimension i only) and
    q(z) = sum_{j <= D} coeffs[j] z^j, D = len(coeffs) - 1 <= 2.

    A[i] is the n_i x n_i matrix dt*L_i.  With S_t = sum_{i in t} A_i the node basis of v is
    [U_t, S_t U_t, .., S_t^D U_t]; since S_t = S_t1 + S_t2 with commuting summands,
    S_t^j U_t = sum_{j1+j2=j} C(j,j1) (S_t2^{j2} U_t2 kron S_t1^{j1} U_t1) B_t, so
      leaf:     U'_i = [U_i, A_i U_i, .., A_i^D U_i]                      (n_i x (D+1)k)
      interior: B'[(j1,a),(j2,b),(j,c)] = C(j,j1) [j = j1+j2] B[a,b,c]
      root:     B'[(j1,a),(j2,b)] = coeffs[j1+j2] C(j1+j2,j1) [j1+j2 <= D] B[a,b]
    with block index (j, c) -> j*k + c.  This is the structured sum of Section 3.2 (sums of HT
    tensors have block structure), taken exactly with no truncation.
    """
    D = len(coeffs) - 1
    if not 0 <= D <= 2:
        raise ValueError("degree 0..2")
    nb = D + 1
    tr = ht.tree
    out = HT(tr, list(ht.n))
    for t in range(tr.n_nodes):
        X = ht.node[t]
        if tr.is_leaf(t):
            Ai = A[tr.lo[t]]
            cols = [X]
            for _ in range(D):
                cols.append(Ai @ cols[-1])
            out.node[t] = np.hstack(cols)
        elif t == 0:
            k1, k2 = X.shape
            Bn = np.zeros((nb * k1, nb * k2))
            for j1 in range(nb):
                for j2 in range(nb - j1):
                    j = j1 + j2
                    Bn[j1 * k1:(j1 + 1) * k1, j2 * k2:(j2 + 1) * k2] = coeffs[j] * _BINOM[j][j1] * X
            out.node[t] = Bn
        else:
            k1, k2, k = X.shape
            Bn = np.zeros((nb * k1, nb * k2, nb * k))
            for j1 in range(nb):
                for j2 in range(nb - j1):
                    j = j1 + j2
                    Bn[j1 * k1:(j1 + 1) * k1, j2 * k2:(j2 + 1) * k2, j * k:(j + 1) * k] = _BINOM[j][j1] * X
            out.node[t] = Bn
    return out


def apply_kron_sum_rk2(ht: HT, A: list) -> HT:
    """v = p(S) u with p(z) = 1 + z + z^2/2 (every two-stage order-2 Runge-Kutta method on a
    linear ODE, Section 3.2): apply_kron_sum_poly with coefficients (1, 1, 1/2), rank 3k."""
    return apply_kron_sum_poly(ht, A, _POLY)


def apply_separable(ht: HT, alphas: list, factors: list) -> HT:
    """v = sum_q alpha_q (kron_i A_i^q) u  (eq. Lz), exact, rank r_L * k.

    factors[q][i] is the n_i x n_i matrix A_i^q (None = identity).  The sum of the r_L
    rank-k HT tensors (kron_i A_i^q) u has leaves [A_i^q U_i]_q, block-diagonal interior
    transfers B'[(q,a),(q,b),(q,c)] = B[a,b,c] and root blocks alpha_q B_root.
    """
    tr = ht.tree
    R = len(alphas)
    out = HT(tr, list(ht.n))
    for t in range(tr.n_nodes):
        X = ht.node[t]
        if tr.is_leaf(t):
            i = tr.lo[t]
            blocks = [X if factors[q][i] is None else factors[q][i] @ X for q in range(R)]
            out.node[t] = np.hstack(blocks)
        elif t == 0:
            k1, k2 = X.shape
            Bn = np.zeros((R * k1, R * k2))
            for q in range(R):
                Bn[q * k1:(q + 1) * k1, q * k2:(q + 1) * k2] = alphas[q] * X
            out.node[t] = Bn
        else:
            k1, k2, k = X.shape
            Bn = np.zeros((R * k1, R * k2, R * k))
            for q in range(R):
                Bn[q * k1:(q + 1) * k1, q * k2:(q + 1) * k2, q * k:(q + 1) * k] = X
            out.node[t] = Bn
    return out


def add(a: float, u: HT, b: float, w: HT) -> HT:
    """a u + b w; ranks add, transfer tensors are block diagonal (Section 3.2)."""
    tr = u.tree
    out = HT(tr, list(u.n))
    for t in range(tr.n_nodes):
        X, Y = u.node[t], w.node[t]
        if tr.is_leaf(t):
            out.node[t] = np.hstack([X, Y])
        elif t == 0:
            Bn = np.zeros((X.shape[0] + Y.shape[0], X.shape[1] + Y.shape[1]))
            Bn[:X.shape[0], :X.shape[1]] = a * X
            Bn[X.shape[0]:, X.shape[1]:] = b * Y
            out.node[t] = Bn
        else:
            s = [X.shape[i] + Y.shape[i] for i in range(3)]
            Bn = np.zeros(s)
            Bn[:X.shape[0], :X.shape[1], :X.shape[2]] = X
            Bn[X.shape[0]:, X.shape[1]:, X.shape[2]:] = Y
            out.node[t] = Bn
    return out


# ---------------------------------------------------------------------------
# mode products on transfer tensors
# ---------------------------------------------------------------------------
def mode_mult(B: np.ndarray, M: np.ndarray, mode: int) -> np.ndarray:
    """B x_mode M: contracts axis `mode` of B with the columns of M (new = M @ old); the
    mode product of the HT toolkit (Section 2.2)."""
    return np.moveaxis(np.tensordot(M, B, axes=(1, mode)), 0, mode)


# ---------------------------------------------------------------------------
# orthogonalisation (bottom-up) and HSVD truncation (root to leaves)
# ---------------------------------------------------------------------------
def orthogonalize(ht: HT) -> HT:
    """Orthonormal node bases for every non-root node (orthogonalisation, Section 2.2).

    Leaves: U = Q R (QR as a library step).  Interior nodes bottom-up: absorb the
    children's R factors, B <- B x1 R_t1 x2 R_t2, then QR of the (k1 k2) x k
    matricisation gives the new B (= Q) and R_t for the parent.  Root: B <- R1 B R2^T.
    """
    tr = ht.tree
    out = HT(tr, list(ht.n))
    Rf = {}
    order = sorted(range(tr.n_nodes), key=lambda t: -tr.depth[t])
    for t in order:
        X = ht.node[t]
        if tr.is_leaf(t):
            Q, R = np.linalg.qr(X, mode="reduced")
            out.node[t] = Q
            Rf[t] = R
        else:
            c1, c2 = tr.children[t]
            if t == 0:
                out.node[t] = Rf[c1] @ X @ Rf[c2].T
            else:
                C = mode_mult(mode_mult(X, Rf[c1], 0), Rf[c2], 1)
                k1, k2, k = C.shape
                Q, R = np.linalg.qr(C.reshape(k1 * k2, k, order="F"), mode="reduced")
                out.node[t] = Q.reshape(k1, k2, Q.shape[1], order="F")
                Rf[t] = R
    return out


def node_svds(orth: HT) -> dict:
    """Singular values and left singular vectors of every node matricisation (the node SVDs
    of the HSVD, Section 2.2).

    For an orthogonalised HT the t-matricisation of u is U_t F_t^... with U_t
    orthonormal, so its left singular pairs are those of the node factor F_t
    (F_t F_t^T is the reduced Gramian).  Root children: F_t1 = B, F_t2 = B^T.
    Interior t with factor F_t: F_t1 = [B_t x3 F_t^T]_(1), F_t2 = [B_t x3 F_t^T]_(2).
    Each F is replaced by W S (its left singular pairs) before use below, which keeps
    F F^T unchanged.  Returns t -> (W_t, s_t) for every non-root node.
    """
    tr = ht_tree = orth.tree
    out = {}
    F = {}
    c1, c2 = tr.children[0]
    B = orth.node[0]
    F[c1] = B
    F[c2] = B.T
    for level in tr.levels()[1:]:
        for t in level:
            W, s = svd_left(F[t])
            out[t] = (W, s)
            if not tr.is_leaf(t):
                Ft = W * s[None, :]
                a, b = tr.children[t]
                D = mode_mult(orth.node[t], Ft.T, 2)       # (k1, k2, k)
                k1, k2, k = D.shape
                F[a] = D.reshape(k1, k2 * k, order="F")
                F[b] = D.transpose(1, 0, 2).reshape(k2, k1 * k, order="F")
    return out


@dataclass
class TruncReport:
    """What the HSVD truncation (Section 2.2) chose and discarded, per node."""
    ranks: list
    sigma: dict          # t -> singular values of the node matricisation
    discarded: dict      # t -> sqrt(sum of discarded sigma^2)
    norm: float
    threshold: float


def choose_rank(s: np.ndarray, thr: float, rmax: int) -> int:
    """Smallest k >= 1 with sum_{j >= k} s_j^2 <= thr^2, then min(k, rmax).

    The paper computes the rank 'adaptively up to r_max' (Section 4.1) without a formula;
    this is the relative-tolerance reading with the HSVD split of the error budget.
    """
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
    k = len(s)
    for kk in range(1, len(s) + 1):
        if tail[kk] <= thr * thr:
            k = kk
            break
    return max(1, min(k, rmax))


def truncate(ht: HT, rel_tol: float, rmax: int):
    """Root-to-leaves HSVD truncation T(u) (Section 2.2 / 3.2, HSVD rank reduction).

    1. orthogonalise; 2. left singular pairs of every node matricisation (from the
    untruncated tensor); 3. rank k_t: smallest k with discarded energy
    <= (rel_tol |u|)^2 / (2d-3), capped at rmax; the two root children share one rank,
    chosen from the first child; 4. project: leaves U <- U W_k, interior
    B <- B x1 W_t1^T x2 W_t2^T x3 W_t^T, root B <- W_t1^T B W_t2.
    Returns (truncated HT, TruncReport).
    """
    tr = ht.tree
    d = tr.d
    orth = orthogonalize(ht)
    nrm = float(np.linalg.norm(orth.node[0]))
    svds = node_svds(orth)
    n_edges = max(2 * d - 3, 1)
    thr = rel_tol * nrm / math.sqrt(n_edges)
    c1, c2 = tr.children[0]
    ranks = [1] * tr.n_nodes
    disc = {}
    for t in range(1, tr.n_nodes):
        src = c1 if t == c2 else t
        W, s = svds[src]
        k = choose_rank(s, thr, rmax)
        k = min(k, svds[t][0].shape[1])
        ranks[t] = k
    for t in range(1, tr.n_nodes):
        s = svds[t][1]
        disc[t] = float(np.sqrt(np.sum(s[ranks[t]:] ** 2)))
    out = HT(tr, list(ht.n))
    Wk = {t: svds[t][0][:, :ranks[t]] for t in range(1, tr.n_nodes)}
    for t in range(tr.n_nodes):
        X = orth.node[t]
        if tr.is_leaf(t):
            out.node[t] = X @ Wk[t]
        elif t == 0:
            out.node[t] = Wk[c1].T @ X @ Wk[c2]
        else:
            a, b = tr.children[t]
            Y = mode_mult(X, Wk[a].T, 0)
            Y = mode_mult(Y, Wk[b].T, 1)
            out.node[t] = mode_mult(Y, Wk[t].T, 2)
    rep = TruncReport(ranks=ranks, sigma={t: svds[t][1] for t in svds}, discarded=disc,
                      norm=nrm, threshold=thr)
    return out, rep


# ---------------------------------------------------------------------------
# scalar quantities
# ---------------------------------------------------------------------------
def _contract_vectors(ht: HT, vecs: list) -> float:
    """sum over the grid of u * prod_i vecs[i] (leaf contraction up the tree of eq. HTD)."""
    tr = ht.tree
    val = {}
    for t in sorted(range(tr.n_nodes), key=lambda t: -tr.depth[t]):
        X = ht.node[t]
        if tr.is_leaf(t):
            val[t] = vecs[tr.lo[t]] @ X
        else:
            a, b = tr.children[t]
            if t == 0:
                return float(val[a] @ X @ val[b])
            val[t] = np.einsum("a,b,abc->c", val[a], val[b], X)
    raise RuntimeError("unreachable")


def mass(ht: HT) -> float:
    """sum of all grid values (the discrete mass up to the cell volume; Section 4.2 checks
    the density moment)."""
    return _contract_vectors(ht, [np.ones(n) for n in ht.n])


def inner(u: HT, w: HT) -> float:
    """<u, w> over the grid via leaf Grams contracted up the tree (scalar product of the HT
    toolkit, Section 2.2)."""
    tr = u.tree
    G = {}
    for t in sorted(range(tr.n_nodes), key=lambda t: -tr.depth[t]):
        X, Y = u.node[t], w.node[t]
        if tr.is_leaf(t):
            G[t] = X.T @ Y
        else:
            a, b = tr.children[t]
            if t == 0:
                return float(np.einsum("ab,ac,bd,cd->", X, G[a], G[b], Y))
            G[t] = np.einsum("abk,ac,bd,cdl->kl", X, G[a], G[b], Y)
    raise RuntimeError("unreachable")


def norm(u: HT) -> float:
    """sqrt(<u, u>) (Section 2.2)."""
    return math.sqrt(max(inner(u, u), 0.0))


# ---------------------------------------------------------------------------
# explicit steps (Section 3.2: apply, add, rank-reduce)
# ---------------------------------------------------------------------------
def step_rk2_poly(u: HT, A: list, rel_tol: float, rmax: int):
    """One step u <- T(p(dt L) u) for a Kronecker-sum operator (single truncation): apply
    and rank reduction of Section 3.2."""
    return truncate(apply_kron_sum_rk2(u, A), rel_tol, rmax)


def step_ab2(u: HT, u_prev: HT, A: list, rel_tol: float, rmax: int):
    """The paper's explicit two-step scheme (eq. AB2_, Section 3.2) for a Kronecker-sum operator:
    u_next = T(u + dt (3/2 L u - 1/2 L u_prev)) = T((1 + 3/2 S) u + (-1/2 S) u_prev) with
    S = dt L, the sum formed exactly (ranks add, block-diagonal transfers) and truncated once."""
    v = add(1.0, apply_kron_sum_poly(u, A, (1.0, 1.5)), 1.0, apply_kron_sum_poly(u_prev, A, (0.0, -0.5)))
    return truncate(v, rel_tol, rmax)


def step_ab2_split(u: HT, u_prev: HT, A: list, rel_tol: float, rmax: int, variant: str = "argument"):
    """eq. AB2_ evaluated as a sequence of simple tensor operations, each followed by a rank
    reduction (Section 3.2, the paragraph after eq. AB2_), with S = dt L (A[i] = dt L_i):

    'argument':   w = T(3 u - u_prev);  v = T(S w);  u_next = T(u + v/2)
                  (the argument of L reduced first, then L w reduced again);
    'difference': w = T(u - u_prev);  a = T(S u);  b = T(S w);  u_next = T(u + a + b/2)
                  (the passage's literal w_{n+1} = f_{n+1} - f_n; dt/2 L (3u - u_prev) = S u + S w / 2).

    Every T is the HSVD truncation with the same tolerance and cap.  Returns (u_next, reports)."""
    if variant == "argument":
        w, r1 = truncate(add(3.0, u, -1.0, u_prev), rel_tol, rmax)
        v, r2 = truncate(apply_kron_sum_poly(w, A, (0.0, 1.0)), rel_tol, rmax)
        un, r3 = truncate(add(1.0, u, 0.5, v), rel_tol, rmax)
        return un, (r1, r2, r3)
    if variant == "difference":
        w, r1 = truncate(add(1.0, u, -1.0, u_prev), rel_tol, rmax)
        a, r2 = truncate(apply_kron_sum_poly(u, A, (0.0, 1.0)), rel_tol, rmax)
        b, r3 = truncate(apply_kron_sum_poly(w, A, (0.0, 1.0)), rel_tol, rmax)
        un, r4 = truncate(add(1.0, u, 1.0, add(1.0, a, 0.5, b)), rel_tol, rmax)
        return un, (r1, r2, r3, r4)
    raise ValueError(variant)


def step_heun2(u: HT, alphas: list, factors: list, dt: float, rel_tol: float, rmax: int):
    """Heun's two-stage RK2 with a truncation after each stage (general separable L):

    u* = T(u + dt L u);  u_next = T(u/2 + (u* + dt L u*)/2).
    Splitting the step into sub-operations each followed by rank reduction is the
    memory-saving variant discussed in Section 3.2.
    """
    I_alpha = [1.0] + [dt * a for a in alphas]
    I_fac = [[None] * len(u.n)] + list(factors)
    ustar, rep1 = truncate(apply_separable(u, I_alpha, I_fac), rel_tol, rmax)
    v = add(0.5, u, 0.5, apply_separable(ustar, I_alpha, I_fac))
    unext, rep2 = truncate(v, rel_tol, rmax)
    return unext, (rep1, rep2)
