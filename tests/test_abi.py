"""CPU-side checks of the C-ABI library: it builds, loads, exports every declared symbol,
and its host-side argument checks answer without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_10270_gb300 import build as B
    B.build()
    from paper_1803_10270_gb300 import htgpu as G
    return G.load()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z][a-z0-9_]*)\s*\(", txt, re.M):
            if m.group(1) not in ("if", "while", "for", "sizeof", "return"):
                names.append(m.group(1))
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    from paper_1803_10270_gb300 import htgpu as G
    declared = _declared_functions()
    assert "ht_step" in declared and "cp_als_sweep" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(G.exported_names())


def test_tree_info_matches_oracle(lib):
    from oracle.tree import build_tree
    from paper_1803_10270_gb300 import htgpu as G
    for d, kind in [(d, k) for d in (2, 3, 6, 7, 12, 16) for k in ("balanced", "linear")]:
        ti = G.tree_info(d, 0 if kind == "balanced" else 1)
        to = build_tree(d, kind)
        assert ti.lo == to.lo and ti.hi == to.hi
        for t in range(to.n_nodes):
            ch = to.children[t]
            assert (ti.c1[t], ti.c2[t]) == ((-1, -1) if ch is None else ch)
            assert ti.depth[t] == to.depth[t]


def test_host_side_argument_errors(lib):
    from paper_1803_10270_gb300 import htgpu as G
    arrs = [(C.c_int * 31)() for _ in range(6)]
    assert lib.ht_tree_info(1, 0, *arrs) == G.HT_ERR_ARG
    assert lib.ht_tree_info(4, 2, *arrs) == G.HT_ERR_ARG
    assert lib.ht_tree_info(17, 0, *arrs) == G.HT_ERR_ARG
    cfg = G.ht_config()
    cfg.d = 1
    assert lib.ht_workspace_bytes(C.byref(cfg)) == 0
    cfg.d = 6
    for i in range(6):
        cfg.n[i] = 16
    cfg.cap = 8
    cfg.max_terms = 6
    cfg.precision = 0
    assert lib.ht_workspace_bytes(C.byref(cfg)) > 0
    cfg.precision = 7
    assert lib.ht_workspace_bytes(C.byref(cfg)) == 0
    out = C.c_void_p()
    assert lib.ht_ctx_create(C.byref(out), C.byref(cfg)) == G.HT_ERR_ARG
    assert lib.ht_step(None, None, None, 0.1, 1e-8, 4, 0, None) == G.HT_ERR_ARG
    assert lib.cp_als_sweep(None, None, None, 1, 0, None, None) == G.HT_ERR_ARG
    assert lib.ht_status_string(G.HT_ERR_CAPACITY) == b"HT_ERR_CAPACITY"
