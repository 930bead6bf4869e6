"""Test helpers: oracle-side comparisons of HT / CP tensors and random inputs."""
import math

import numpy as np

from oracle import ht as OH
from oracle.tree import build_tree
from paper_1803_10270_gb300.inputs import normal_arrays


def random_ht(d, ns, rank, seed, scale_decay=None, kind="balanced"):
    """Random HT with every non-root rank = rank (leaves min(n, rank) not enforced), on the
    balanced or the linear (tensor-train) tree."""
    tree = build_tree(d, kind)
    ns = [ns] * d if np.isscalar(ns) else list(ns)
    rk = {t: (1 if t == 0 else rank) for t in range(tree.n_nodes)}
    shapes = []
    for t in range(tree.n_nodes):
        if tree.is_leaf(t):
            shapes.append((ns[tree.lo[t]], rk[t]))
        else:
            a, b = tree.children[t]
            shapes.append((rk[a], rk[b]) if t == 0 else (rk[a], rk[b], rk[t]))
    arrs = normal_arrays(shapes, seed)
    u = OH.HT(tree, ns)
    for t in range(tree.n_nodes):
        u.node[t] = arrs[t]
        if scale_decay is not None and not tree.is_leaf(t):
            # graded transfer tensors: make singular values decay
            k = arrs[t].shape[-1]
            g = scale_decay ** np.arange(k)
            u.node[t] = arrs[t] * g.reshape((1,) * (arrs[t].ndim - 1) + (k,))
    return u


def ht_diff_norm(a: OH.HT, b: OH.HT) -> float:
    """|a - b| through an orthogonalised HT difference (no full grid, no Gram cancellation)."""
    diff = OH.add(1.0, a, -1.0, b)
    o = OH.orthogonalize(diff)
    return float(np.linalg.norm(o.node[0]))


def ht_norm(a: OH.HT) -> float:
    return float(np.linalg.norm(OH.orthogonalize(a).node[0]))


def rel_err(a: OH.HT, b: OH.HT) -> float:
    return ht_diff_norm(a, b) / max(ht_norm(b), 1e-300)


def min_gap(rep, ranks):
    """Smallest ratio s_k / s_{k+1} at the chosen cuts (inf when nothing is cut)."""
    g = math.inf
    for t, s in rep.sigma.items():
        k = ranks[t]
        if k < len(s) and s[k] > 0:
            g = min(g, s[k - 1] / s[k])
    return g
