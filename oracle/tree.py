"""Dimension trees (Section 2.2, eq. HTD).

Balanced: the paper splits the six variables {1..6} as {1,2,3}|{4,5,6} and then {1}|{2,3},
{4}|{5,6} (eq. HTD / coreT).  Generalised: the index range [a, b) splits at
a + floor((b - a)/2).  Linear: [a, b) splits at a + 1 ({a} | [a+1, b)), the degenerate tree on
which HT is the tensor-train format (Section 2.2).  Nodes are numbered breadth first from the
root (node 0).

Parity: pinned by tests (the d = 6 split reproduces the paper's grouping; 2d-1 nodes; on the
linear tree the node singular values equal those of the TT unfoldings of the full tensor).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class Tree:
    """A dimension tree (Section 2.2, eq. HTD): node ranges [lo, hi), children, depths."""
    d: int
    lo: list        # first dimension of each node
    hi: list        # one past the last dimension
    children: list  # (c1, c2) or None for a leaf
    parent: list
    depth: list

    @property
    def n_nodes(self) -> int:
        return len(self.lo)

    def is_leaf(self, t: int) -> bool:
        return self.children[t] is None

    def leaf_of_dim(self, i: int) -> int:
        for t in range(self.n_nodes):
            if self.is_leaf(t) and self.lo[t] == i:
                return t
        raise KeyError(i)

    def dims(self, t: int) -> list:
        return list(range(self.lo[t], self.hi[t]))

    def levels(self) -> list:
        """Nodes grouped by depth, root first."""
        m = max(self.depth)
        return [[t for t in range(self.n_nodes) if self.depth[t] == k] for k in range(m + 1)]


def build_tree(d: int, kind: str = "balanced") -> Tree:
    """The balanced tree of eq. HTD / coreT, or the linear tree of the tensor-train format
    (Section 2.2), numbered breadth first."""
    if d < 2:
        raise ValueError("HT needs d >= 2")
    if kind not in ("balanced", "linear"):
        raise ValueError(kind)
    lo, hi, children, parent, depth = [0], [d], [None], [-1], [0]
    t = 0
    while t < len(lo):
        a, b = lo[t], hi[t]
        if b - a > 1:
            m = a + 1 if kind == "linear" else a + (b - a) // 2
            c1 = len(lo)
            lo += [a, m]
            hi += [m, b]
            children += [None, None]
            parent += [t, t]
            depth += [depth[t] + 1] * 2
            children[t] = (c1, c1 + 1)
        t += 1
    return Tree(d=d, lo=lo, hi=hi, children=children, parent=parent, depth=depth)
