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
    cfg.precision = 0
    cfg.biorth_form = 2
    assert lib.ht_workspace_bytes(C.byref(cfg)) == 0
    cfg.biorth_form = 1
    assert lib.ht_workspace_bytes(C.byref(cfg)) > 0
    cfg.precision = 7
    out = C.c_void_p()
    assert lib.ht_ctx_create(C.byref(out), C.byref(cfg)) == G.HT_ERR_ARG
    assert lib.ht_step(None, None, None, 0.1, 1e-8, 4, 0, None) == G.HT_ERR_ARG
    assert lib.cp_als_sweep(None, None, None, 1, 0, None, None) == G.HT_ERR_ARG
    assert lib.ht_status_string(G.HT_ERR_CAPACITY) == b"HT_ERR_CAPACITY"


def test_every_entry_point_checks_its_arguments_before_the_gpu(lib):
    """Each entry point answers null or malformed arguments with its status code, from host
    checks made before any CUDA call (so this runs without a GPU); the destroy calls and the
    launch counter accept a null handle."""
    from paper_1803_10270_gb300 import htgpu as G
    ARG, CAPY = G.HT_ERR_ARG, G.HT_ERR_CAPACITY
    assert lib.ht_apply(None, None, None, 0.1, 0, None, None) == ARG
    assert lib.ht_truncate(None, None, 1e-8, 4, None, None, 0, None, None) == ARG
    assert lib.ht_step_ab2(None, None, None, None, 0.1, 1e-8, 4, None) == ARG
    assert lib.ht_from_cp(None, None, None, None) == ARG
    assert lib.ht_mass(None, None, None, None) == ARG
    assert lib.ht_inner(None, None, None, None, None) == ARG
    assert lib.cp_apply_rk2(None, None, None, 0.1, None, None) == ARG
    assert lib.cp_als_sweep_rk2(None, None, None, 0.1, None, 5, 0, None, None) == ARG
    assert lib.cp_cn_als_step(None, None, None, 0.1, None, 5, 0, None, None) == ARG
    assert lib.ht_ctx_profile(None, 1) == ARG
    assert lib.ht_ctx_profile_read(None, None, None, None) == ARG
    assert lib.ht_ctx_check(None, None) == ARG
    assert lib.ht_ctx_launches(None) == 0
    assert lib.ht_biorth_cluster_ctas(None, None) == ARG
    lib.ht_ctx_destroy(None)
    lib.ht_batch_destroy(None)
    out = C.c_void_p()
    assert lib.ht_batch_create(None, 1, None, None) == ARG
    assert lib.ht_batch_create(C.byref(out), 0, None, None) == ARG and not out.value
    assert lib.ht_batch_step(None, None, None, None, None, 0, None) == ARG
    # the allocation-free sweep takes no context: its size checks are all on the host
    dummy = (C.c_double * 1)()
    addr = C.cast(dummy, C.c_void_p).value

    def cp(d, n, rank, cap):
        t = G.cp_tensor()
        t.d, t.rank, t.cap, t.weight = d, rank, cap, addr
        for k in range(d):
            t.n[k] = n
            t.factor[k] = addr
        return t
    call = lambda y, x, sweeps=5, variant=0: lib.cp_als_sweep_noalloc(C.byref(y), C.byref(x), sweeps, variant,
                                                                      None, None, None)
    assert lib.cp_als_sweep_noalloc(None, None, 5, 0, None, None, None) == ARG
    assert call(cp(6, 16, 4, 4), cp(6, 16, 2, 2), sweeps=65) == ARG
    assert call(cp(6, 16, 4, 4), cp(6, 16, 2, 2), variant=7) == ARG
    assert call(cp(1, 16, 4, 4), cp(1, 16, 2, 2)) == ARG                 # d < 2
    assert call(cp(6, 16, 4, 4), cp(5, 16, 2, 2)) == ARG                 # d mismatch
    assert call(cp(6, 16, 4, 4), cp(6, 17, 2, 2)) == ARG                 # n mismatch
    assert call(cp(6, 16, 4, 4), cp(6, 16, 3, 2)) == CAPY                # rank > cap
    assert call(cp(9, 16, 4, 4), cp(9, 16, 2, 2)) == CAPY                # d > 8
    assert call(cp(6, 257, 4, 4), cp(6, 257, 2, 2)) == CAPY              # n > 256
    assert call(cp(6, 16, 4, 4), cp(6, 16, 33, 33)) == CAPY              # x rank > 32
    assert call(cp(6, 16, 1025, 1025), cp(6, 16, 2, 2)) == CAPY          # y rank > 1024
    y, x = cp(6, 16, 4, 4), cp(6, 16, 2, 2)
    x.factor[3] = None
    assert call(y, x) == ARG                                             # missing factor


def test_product_path_fails_loudly_without_a_gpu_or_library(lib):
    """No CPU fallback: without a GPU, creating a context raises the library's HT_ERR_CUDA, and a
    library that was not built raises instead of substituting anything."""
    import torch
    from paper_1803_10270_gb300 import htgpu as G
    with pytest.raises(RuntimeError, match="not built"):
        G.load(os.path.join(ROOT, "no_such_dir", "libhtgpu.so"))
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: contexts are created normally")
    with pytest.raises(G.HTError, match="HT_ERR_CUDA"):
        G.Context(6, [16] * 6, cap=8, max_terms=1)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of the header's structs have the header's field offsets and
    sizes: a C program compiled against include/htgpu.h prints them (gcc, no GPU)."""
    import shutil
    import subprocess
    from paper_1803_10270_gb300 import htgpu as G
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    structs = [("ht_config", G.ht_config), ("cp_tensor", G.cp_tensor), ("ht_factor", G.ht_factor), ("ht_op", G.ht_op)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "htgpu.h"', "int main(void) {"]
    for name, py in structs:
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, py in structs:
        assert got[(name, "sizeof")] == C.sizeof(py), name
        for f, _ in py._fields_:
            assert got[(name, f)] == getattr(py, f).offset, (name, f)
