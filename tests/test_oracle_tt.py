"""The tensor-train format as HT on the linear dimension tree (Section 2.2): oracle pins.

On the linear tree ({a} | [a+1, b) at every node) the node matricisations are the TT
unfoldings, so the oracle's node singular values must equal those of the full tensor's
unfoldings (brute force on tiny tensors), and the HSVD truncation obeys the quasi-optimality
bound |u - T(u)|^2 <= sum over nodes of the discarded squared singular values."""
import numpy as np
import pytest

from oracle import ht as OH
from oracle.tree import build_tree
from tests.helpers import random_ht


def test_linear_tree_shape():
    for d in (2, 3, 5, 8):
        t = build_tree(d, "linear")
        assert t.n_nodes == 2 * d - 1
        assert max(t.depth) == d - 1
        # interior node [i, d) has children {i} (a leaf) and [i+1, d)
        node = 0
        for i in range(d - 1):
            assert (t.lo[node], t.hi[node]) == (i, d)
            c1, c2 = t.children[node]
            assert t.is_leaf(c1) and (t.lo[c1], t.hi[c1]) == (i, i + 1)
            assert (t.lo[c2], t.hi[c2]) == (i + 1, d)
            node = c2
        assert t.is_leaf(node)


def unfolding_sv(full, dims):
    d = full.ndim
    rest = [i for i in range(d) if i not in dims]
    M = np.transpose(full, list(dims) + rest).reshape(int(np.prod([full.shape[i] for i in dims])), -1)
    return np.linalg.svd(M, compute_uv=False)


@pytest.mark.parametrize("kind", ["linear", "balanced"])
def test_node_singular_values_equal_unfolding_singular_values(kind):
    d, n, r = 5, 4, 3
    u = random_ht(d, n, r, seed=21, scale_decay=0.6, kind=kind)
    full = OH.to_full(u)
    sv = OH.node_svds(OH.orthogonalize(u))
    for t in range(1, u.tree.n_nodes):
        s_brute = unfolding_sv(full, u.tree.dims(t))
        s = np.asarray(sv[t][1])          # (W_t, s_t)
        k = min(len(s), len(s_brute))
        assert np.allclose(s[:k], s_brute[:k], rtol=1e-10, atol=1e-12 * s_brute[0]), t
        assert np.all(s_brute[k:] <= 1e-12 * s_brute[0])


@pytest.mark.parametrize("rmax", [1, 2, 3])
def test_tt_truncation_quasi_optimality(rmax):
    d, n, r = 5, 4, 3
    u = random_ht(d, n, r, seed=22, scale_decay=0.5, kind="linear")
    full = OH.to_full(u)
    tu, rep = OH.truncate(u, 0.0, rmax)
    err2 = float(np.sum((OH.to_full(tu) - full) ** 2))
    bound = 0.0
    for t in range(1, u.tree.n_nodes):
        if t == u.tree.children[0][1]:
            continue                      # the root children share one spectrum: count it once
        s = unfolding_sv(full, u.tree.dims(t))
        bound += float(np.sum(s[rep.ranks[t]:] ** 2))
    assert err2 <= bound * (1 + 1e-10) + 1e-24
    assert all(k <= rmax for k in rep.ranks[1:])
