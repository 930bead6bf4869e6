"""Pins of the oracle against values the paper prints (fixtures under tests/golden/)."""
import os

import numpy as np

from oracle.ht import central_diff_matrix
from oracle.problems import kinetic_terms
from paper_1803_10270_gb300.inputs import kinetic_case

HERE = os.path.dirname(os.path.abspath(__file__))


def read_terms():
    rows = []
    with open(os.path.join(HERE, "golden", "kinetic_operator_terms.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_kinetic_operator_contains_the_paper_terms():
    """Every term of Table tab:ordering (transport -v_i d/dx_i and the relaxation -nu I) is a
    term of the oracle's kinetic operator, with the same coefficient and 1-D factors.  The
    oracle adds one more term, +nu P (P = I_x x (m w^T)^{x3}), the Maxwellian source of the
    linearised relaxation -nu (f - M(v) rho)."""
    kc = kinetic_case(6)
    alphas, factors = kinetic_terms(kc)
    D = central_diff_matrix(kc.n, kc.hx)
    V = np.diag(kc.vgrid())
    rows = read_terms()
    assert len(rows) == 4
    used = set()
    for row in rows:
        alpha = -kc.nu if row[1] == "-nu" else float(row[1])
        want = []
        for tok in row[2:]:
            if tok == "1":
                want.append(None)
            elif tok.startswith("dx"):
                want.append(D)
            else:
                want.append(V)
        hit = None
        for q, (a, fs) in enumerate(zip(alphas, factors)):
            if q in used or abs(a - alpha) > 1e-15:
                continue
            same = all((w is None and f is None) or (w is not None and f is not None and np.array_equal(w, f))
                       for w, f in zip(want, fs))
            if same:
                hit = q
                break
        assert hit is not None, f"paper term {row[0]} missing"
        used.add(hit)
    extra = [q for q in range(len(alphas)) if q not in used]
    assert len(extra) == 1 and abs(alphas[extra[0]] - kc.nu) < 1e-15
