"""Thin Python binding of the htgpu C ABI (include/htgpu.h).

Argument marshalling only: torch supplies device memory and the CUDA stream, every
step of the computation runs in the library's kernels.  Loading fails loudly when the
compiled library is missing; there is no CPU fallback.

Names follow the C entry points: ht_apply, ht_truncate, ht_step, ht_from_cp, ht_mass,
ht_inner, cp_apply_rk2, cp_als_sweep.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HT_MAXD = 16
HT_MAXNODES = 2 * HT_MAXD - 1
HT_MAXTERMS = 16
HT_MAXBLOCKTERMS = 10
HT_MAXSTENCIL = 9

HT_OK, HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA, HT_ERR_NONFINITE, HT_ERR_TIMEOUT, HT_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
HT_PREC_FP64, HT_PREC_MIXED = 0, 1
CP_FORM_AUTO, CP_FORM_GRID = 0, 1   # ht_config.cp_form
BIORTH_FORM_CTA, BIORTH_FORM_CLUSTER = 0, 1   # ht_config.biorth_form
HT_F_IDENTITY, HT_F_STENCIL, HT_F_DIAG, HT_F_RANK1, HT_F_DIAG_STENCIL = 0, 1, 2, 3, 4
HT_APPLY_L, HT_APPLY_EULER, HT_APPLY_RK2POLY = 0, 1, 2
HT_SCHEME_RK2POLY, HT_SCHEME_HEUN2 = 0, 1
HT_TREE_BALANCED, HT_TREE_LINEAR = 0, 1
CP_ALS_GS, CP_ALS_JACOBI_DAMPED = 0, 1

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libhtgpu.so")


class ht_tensor(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int * HT_MAXD), ("cap", C.c_int),
                ("node", C.c_void_p * HT_MAXNODES), ("rank", C.c_void_p)]


class cp_tensor(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int * HT_MAXD), ("rank", C.c_int), ("cap", C.c_int),
                ("factor", C.c_void_p * HT_MAXD), ("weight", C.c_void_p)]


class ht_factor(C.Structure):
    _fields_ = [("kind", C.c_int), ("half_width", C.c_int), ("stencil", C.c_double * HT_MAXSTENCIL),
                ("v", C.c_void_p), ("w", C.c_void_p)]


class ht_op(C.Structure):
    _fields_ = [("d", C.c_int), ("n_terms", C.c_int), ("kron_sum", C.c_int),
                ("alpha", C.c_double * HT_MAXTERMS), ("f", (ht_factor * HT_MAXD) * HT_MAXTERMS)]


class ht_config(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int * HT_MAXD), ("cap", C.c_int), ("max_terms", C.c_int),
                ("precision", C.c_int), ("device", C.c_int), ("tree", C.c_int), ("mixed_slices", C.c_int),
                ("tc_min_work", C.c_longlong), ("gemm_ctas_per_sm", C.c_int), ("svd_cluster_min_cols", C.c_int),
                ("cp_form", C.c_int), ("biorth_form", C.c_int)]


_EXPORTS = {
    "ht_workspace_bytes": (C.c_size_t, [C.POINTER(ht_config)]),
    "ht_ctx_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(ht_config)]),
    "ht_ctx_destroy": (None, [C.c_void_p]),
    "ht_ctx_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ht_ctx_launches": (C.c_longlong, [C.c_void_p]),
    "ht_biorth_cluster_ctas": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "ht_status_string": (C.c_char_p, [C.c_int]),
    "ht_ctx_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "ht_ctx_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double)]),
    "ht_tree_info": (C.c_int, [C.c_int, C.c_int] + [C.POINTER(C.c_int)] * 6),
    "ht_apply": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.POINTER(ht_op), C.c_double, C.c_int,
                           C.POINTER(ht_tensor), C.c_void_p]),
    "ht_truncate": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.c_double, C.c_int, C.POINTER(ht_tensor),
                              C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "ht_step": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.POINTER(ht_op), C.c_double, C.c_double,
                          C.c_int, C.c_int, C.c_void_p]),
    "ht_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "ht_batch_destroy": (None, [C.c_void_p]),
    "ht_batch_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_int), C.c_int, C.c_void_p]),
    "ht_step_ab2": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.POINTER(ht_tensor), C.POINTER(ht_op), C.c_double,
                              C.c_double, C.c_int, C.c_void_p]),
    "ht_from_cp": (C.c_int, [C.c_void_p, C.POINTER(cp_tensor), C.POINTER(ht_tensor), C.c_void_p]),
    "ht_add": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(ht_tensor), C.c_double, C.POINTER(ht_tensor),
                         C.POINTER(ht_tensor), C.c_void_p]),
    "ht_step_ab2_split": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.POINTER(ht_tensor), C.POINTER(ht_op),
                                    C.c_double, C.c_double, C.c_int, C.c_int, C.c_void_p]),
    "ht_mass": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.c_void_p, C.c_void_p]),
    "ht_inner": (C.c_int, [C.c_void_p, C.POINTER(ht_tensor), C.POINTER(ht_tensor), C.c_void_p, C.c_void_p]),
    "cp_apply_rk2": (C.c_int, [C.c_void_p, C.POINTER(cp_tensor), C.POINTER(ht_op), C.c_double,
                               C.POINTER(cp_tensor), C.c_void_p]),
    "cp_als_sweep": (C.c_int, [C.c_void_p, C.POINTER(cp_tensor), C.POINTER(cp_tensor), C.c_int, C.c_int,
                               C.c_void_p, C.c_void_p]),
    "cp_als_sweep_rk2": (C.c_int, [C.c_void_p, C.POINTER(cp_tensor), C.POINTER(ht_op), C.c_double,
                                   C.POINTER(cp_tensor), C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "cp_als_rk2_cluster_ctas": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "cp_als_sweep_noalloc": (C.c_int, [C.POINTER(cp_tensor), C.POINTER(cp_tensor), C.c_int, C.c_int,
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    "ht_selftest_grid_barrier": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "ht_selftest_fastmath": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "ht_tune_time_gemm": (C.c_int, [C.c_int] * 8 + [C.POINTER(C.c_double)]),
    "ht_selftest_gemm_mixed": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                         C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                         C.c_void_p, C.c_int, C.c_longlong, C.c_longlong, C.c_longlong,
                                         C.c_int, C.c_void_p]),
    "cp_cn_als_step": (C.c_int, [C.c_void_p, C.POINTER(cp_tensor), C.POINTER(ht_op), C.c_double,
                                 C.POINTER(cp_tensor), C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
}

_lib = None


def exported_names() -> list:
    return list(_EXPORTS)


def load(path: str | None = None):
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"htgpu library not built: {p} (run __graft_entry__.build())")
    lib = C.CDLL(p)
    for name, (res, args) in _EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


class HTError(RuntimeError):
    def __init__(self, status: int, what: str):
        name = load().ht_status_string(status).decode()
        super().__init__(f"{what}: {name} ({status})")
        self.status = status


def _check(st: int, what: str):
    if st != HT_OK:
        raise HTError(st, what)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------- tree
@dataclass
class TreeInfo:
    d: int
    lo: list
    hi: list
    c1: list
    c2: list
    parent: list
    depth: list

    @property
    def n_nodes(self):
        return 2 * self.d - 1

    def is_leaf(self, t):
        return self.c1[t] < 0


def tree_info(d: int, tree: int = 0) -> TreeInfo:
    lib = load()
    arrs = [(C.c_int * HT_MAXNODES)() for _ in range(6)]
    _check(lib.ht_tree_info(d, tree, *arrs), "ht_tree_info")
    nn = 2 * d - 1
    return TreeInfo(d, *[list(a)[:nn] for a in arrs])


# ----------------------------------------------------------------------------- ctx
class Context:
    """Owns an ht_ctx (workspace on the device)."""

    def __init__(self, d: int, n, cap: int, max_terms: int = 6, precision: int = HT_PREC_FP64,
                 device: int = 0, tree: int = 0, mixed_slices: int = 0, tuning: dict | None = None,
                 cp_form: int = 0, biorth_form: int = 0):
        """tuning: values for the ht_config tuning fields (tc_min_work, gemm_ctas_per_sm,
        svd_cluster_min_cols); None takes the tuning cache of this device when one exists
        (paper_1803_10270_gb300.tune), {} the library defaults.  cp_form: CP_FORM_AUTO (the
        cluster form of cp_als_sweep_rk2 where it fits) or CP_FORM_GRID.  biorth_form:
        BIORTH_FORM_CTA (one CTA per node) or BIORTH_FORM_CLUSTER (a thread-block cluster per
        node in contexts of truncation rank 160 and above); the two give the same bits."""
        lib = load()
        cfg = ht_config()
        cfg.d = d
        for i, v in enumerate(n):
            cfg.n[i] = int(v)
        cfg.cap = cap
        cfg.max_terms = max_terms
        cfg.precision = precision
        cfg.device = device
        cfg.tree = tree
        cfg.mixed_slices = mixed_slices
        cfg.cp_form = cp_form
        cfg.biorth_form = biorth_form
        if tuning is None:
            from paper_1803_10270_gb300 import tune as _tune
            tuning = _tune.cached(device, max(3, max_terms + 2) * cap)
        for k in ("tc_min_work", "gemm_ctas_per_sm", "svd_cluster_min_cols"):
            if k in tuning:
                setattr(cfg, k, int(tuning[k]))
        self.tuning = dict(tuning)
        self.cfg = cfg
        self.d, self.n, self.cap, self.device = d, list(n), cap, device
        self.ptr = C.c_void_p()
        _check(lib.ht_ctx_create(C.byref(self.ptr), C.byref(cfg)), "ht_ctx_create")

    @property
    def workspace_bytes(self) -> int:
        return int(load().ht_workspace_bytes(C.byref(self.cfg)))

    def launches(self) -> int:
        return int(load().ht_ctx_launches(self.ptr))

    def biorth_cluster_ctas(self) -> int:
        """CTAs per node of the cluster form of the X_t Y_t = I refinement, 0 for one CTA per node."""
        out = C.c_int(0)
        _check(load().ht_biorth_cluster_ctas(self.ptr, C.byref(out)), "ht_biorth_cluster_ctas")
        return int(out.value)

    KERNEL_CLASSES = ["apply", "gemm", "qr", "svd", "plan", "cp_small", "cp_solve", "gemm_tc"]

    def profile(self, on: bool):
        _check(load().ht_ctx_profile(self.ptr, 1 if on else 0), "ht_ctx_profile")

    def profile_read(self) -> dict:
        n = len(self.KERNEL_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_longlong * n)()
        fl = (C.c_double * n)()
        _check(load().ht_ctx_profile_read(self.ptr, ms, cnt, fl), "ht_ctx_profile_read")
        return {k: {"ms": ms[i], "launches": cnt[i], "flops": fl[i]} for i, k in enumerate(self.KERNEL_CLASSES)}

    def check(self, stream=None):
        _check(load().ht_ctx_check(self.ptr, _stream_ptr(stream)), "device error word")

    def close(self):
        if self.ptr:
            load().ht_ctx_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- tensors
class HTTensor:
    """Device buffers of an HT tensor (capacity `cap`) plus its ht_tensor struct."""

    def __init__(self, d: int, n, cap: int, device="cuda", tree: int = 0):
        import torch
        self.d, self.n, self.cap = d, list(n), cap
        self.tree = tree_info(d, tree)
        # one device allocation (`blob`) holds every node buffer at 256-byte aligned offsets, so
        # the whole state moves between host and device in one copy
        sizes = []
        for t in range(self.tree.n_nodes):
            if self.tree.is_leaf(t):
                sizes.append(self.n[self.tree.lo[t]] * cap)
            elif t == 0:
                sizes.append(cap * cap)
            else:
                sizes.append(cap ** 3)
        offs, off = [], 0
        for sz in sizes:
            offs.append(off)
            off += (sz + 31) // 32 * 32
        self.blob = torch.zeros(off, dtype=torch.float64, device=device)
        self.bufs = [self.blob[o:o + sz] for o, sz in zip(offs, sizes)]
        self.rank_buf = torch.ones(HT_MAXNODES, dtype=torch.int32, device=device)
        s = ht_tensor()
        s.d = d
        for i, v in enumerate(self.n):
            s.n[i] = v
        s.cap = cap
        for t, b in enumerate(self.bufs):
            s.node[t] = b.data_ptr()
        s.rank = self.rank_buf.data_ptr()
        self.struct = s

    def ranks(self) -> list:
        return [int(v) for v in self.rank_buf[: self.tree.n_nodes].cpu()]

    def upload(self, nodes: dict):
        """nodes: t -> numpy array in the oracle's shapes (leaf n x k, interior (k1,k2,k), root (k1,k2))."""
        import torch
        rk = np.ones(HT_MAXNODES, dtype=np.int32)
        for t, a in nodes.items():
            a = np.asarray(a, dtype=np.float64)
            flat = a.reshape(-1, order="F")
            if flat.size > self.bufs[t].numel():
                raise ValueError(f"node {t} exceeds capacity")
            self.bufs[t][: flat.size].copy_(torch.from_numpy(flat))
            if t != 0:
                rk[t] = a.shape[1] if self.tree.is_leaf(t) else a.shape[2]
        self.rank_buf.copy_(torch.from_numpy(rk))

    def download(self) -> dict:
        rk = self.ranks()
        out = {}
        tr = self.tree
        for t in range(tr.n_nodes):
            buf = self.bufs[t].cpu().numpy()
            if tr.is_leaf(t):
                shape = (self.n[tr.lo[t]], rk[t])
            else:
                k1, k2 = rk[tr.c1[t]], rk[tr.c2[t]]
                shape = (k1, k2) if t == 0 else (k1, k2, rk[t])
            out[t] = buf[: int(np.prod(shape))].reshape(shape, order="F").copy()
        return out


class CPTensor:
    """Device buffers of a CP tensor (column capacity `cap`)."""

    def __init__(self, d: int, n, cap: int, device="cuda"):
        import torch
        self.d, self.n, self.cap = d, list(n), cap
        # factors and weights in one device allocation (`blob`), 256-byte aligned views
        sizes = [v * cap for v in self.n] + [cap]
        offs, off = [], 0
        for sz in sizes:
            offs.append(off)
            off += (sz + 31) // 32 * 32
        self.blob = torch.zeros(off, dtype=torch.float64, device=device)
        views = [self.blob[o:o + sz] for o, sz in zip(offs, sizes)]
        self.factors, self.weight = views[:-1], views[-1]
        s = cp_tensor()
        s.d = d
        for i, v in enumerate(self.n):
            s.n[i] = v
        s.rank = 0
        s.cap = cap
        for i, f in enumerate(self.factors):
            s.factor[i] = f.data_ptr()
        s.weight = self.weight.data_ptr()
        self.struct = s

    @property
    def rank(self) -> int:
        return int(self.struct.rank)

    def upload(self, weights, factors):
        import torch
        r = len(weights)
        if r > self.cap:
            raise ValueError("rank exceeds capacity")
        self.weight[:r].copy_(torch.from_numpy(np.asarray(weights, dtype=np.float64)))
        for i, f in enumerate(factors):
            self.factors[i][: f.size].copy_(torch.from_numpy(np.asarray(f, dtype=np.float64).reshape(-1, order="F")))
        self.struct.rank = r

    def download(self):
        r = self.rank
        w = self.weight[:r].cpu().numpy().copy()
        fs = [self.factors[i][: self.n[i] * r].cpu().numpy().reshape(self.n[i], r, order="F").copy()
              for i in range(self.d)]
        return w, fs


# ----------------------------------------------------------------------------- operators
def stencil_factor(coefs) -> ht_factor:
    f = ht_factor()
    f.kind = HT_F_STENCIL
    w = (len(coefs) - 1) // 2
    f.half_width = w
    for j, c in enumerate(coefs):
        f.stencil[j] = float(c)
    return f


def advection_op(c, h) -> ht_op:
    """L = -sum_i c_i D_i, D the periodic central difference (u_{j+1} - u_{j-1}) / (2h)."""
    d = len(c)
    op = ht_op()
    op.d = d
    op.n_terms = d
    op.kron_sum = 1
    hs = [h] * d if np.isscalar(h) else list(h)
    for i in range(d):
        op.alpha[i] = -float(c[i])
        for j in range(d):
            op.f[i][j] = stencil_factor([-0.5 / hs[i], 0.0, 0.5 / hs[i]]) if j == i else ht_factor()
    return op


class KineticOp:
    """-v.grad_x f - nu f + nu M(v) rho on (x1,x2,x3,v1,v2,v3); keeps its device vectors alive."""

    def __init__(self, kc, device="cuda"):
        import torch
        self.vg = torch.tensor(kc.vgrid(), dtype=torch.float64, device=device)
        self.m = torch.tensor(kc.maxwellian(), dtype=torch.float64, device=device)
        self.w = torch.tensor(kc.weights(), dtype=torch.float64, device=device)
        op = ht_op()
        op.d = 6
        op.n_terms = 5
        op.kron_sum = 0
        hx = kc.hx
        for i in range(3):
            op.alpha[i] = -1.0
            for j in range(6):
                op.f[i][j] = ht_factor()
            op.f[i][i] = stencil_factor([-0.5 / hx, 0.0, 0.5 / hx])
            fd = ht_factor()
            fd.kind = HT_F_DIAG
            fd.v = self.vg.data_ptr()
            op.f[i][3 + i] = fd
        op.alpha[3] = -kc.nu
        for j in range(6):
            op.f[3][j] = ht_factor()
        op.alpha[4] = kc.nu
        for j in range(6):
            f = ht_factor()
            if j >= 3:
                f.kind = HT_F_RANK1
                f.v = self.m.data_ptr()
                f.w = self.w.data_ptr()
            op.f[4][j] = f
        self.op = op


class VarCoefOp:
    """-sum_j (C z)_j d/dz_j on (z_1..z_N) in the term order of Table tab:ordering0 (term
    q = j N + k carries -C_jk: the derivative on z_j and z on z_k, or z d/dz_j when k = j);
    keeps its device vector z alive."""

    def __init__(self, case, device="cuda"):
        import torch
        self.z = torch.tensor(case.z(), dtype=torch.float64, device=device)
        N = case.N
        D = [-0.5 / case.h, 0.0, 0.5 / case.h]
        op = ht_op()
        op.d = N
        op.n_terms = N * N
        op.kron_sum = 0
        for j in range(N):
            for k in range(N):
                q = j * N + k
                op.alpha[q] = -float(case.C[j, k])
                for i in range(N):
                    op.f[q][i] = ht_factor()
                if k == j:
                    f = stencil_factor(D)
                    f.kind = HT_F_DIAG_STENCIL
                    f.v = self.z.data_ptr()
                    op.f[q][j] = f
                else:
                    op.f[q][j] = stencil_factor(D)
                    fz = ht_factor()
                    fz.kind = HT_F_DIAG
                    fz.v = self.z.data_ptr()
                    op.f[q][k] = fz
        self.op = op


# ----------------------------------------------------------------------------- calls
def ht_apply(ctx: Context, u: HTTensor, op: ht_op, dt: float, mode: int, v: HTTensor, stream=None):
    _check(load().ht_apply(ctx.ptr, C.byref(u.struct), C.byref(op), dt, mode, C.byref(v.struct),
                           _stream_ptr(stream)), "ht_apply")


def ht_truncate(ctx: Context, u: HTTensor, rel_tol: float, rmax: int, out: HTTensor, sigma=None,
                sig_stride: int = 0, norm=None, stream=None):
    _check(load().ht_truncate(ctx.ptr, C.byref(u.struct), rel_tol, rmax, C.byref(out.struct),
                              C.c_void_p(sigma.data_ptr() if sigma is not None else 0), sig_stride,
                              C.c_void_p(norm.data_ptr() if norm is not None else 0),
                              _stream_ptr(stream)), "ht_truncate")


def ht_step(ctx: Context, u: HTTensor, op: ht_op, dt: float, rel_tol: float, rmax: int,
            scheme: int = HT_SCHEME_RK2POLY, stream=None):
    _check(load().ht_step(ctx.ptr, C.byref(u.struct), C.byref(op), dt, rel_tol, rmax, scheme,
                          _stream_ptr(stream)), "ht_step")


class Batch:
    """Owns an ht_batch: independent instances (one context and one tensor each, same d) stepped
    together, every launch covering all instances."""

    def __init__(self, ctxs, tensors):
        if len(ctxs) != len(tensors) or not ctxs:
            raise ValueError("one tensor per context")
        self.ctxs, self.tensors = list(ctxs), list(tensors)
        n = len(ctxs)
        cp = (C.c_void_p * n)(*[c.ptr.value for c in ctxs])
        self._tptr = (C.c_void_p * n)(*[C.cast(C.pointer(t.struct), C.c_void_p).value for t in tensors])
        self.ptr = C.c_void_p()
        _check(load().ht_batch_create(C.byref(self.ptr), n, cp, self._tptr), "ht_batch_create")

    def step(self, ops, dts, rel_tols, rmaxs, scheme: int = HT_SCHEME_RK2POLY, stream=None):
        n = len(self.ctxs)
        self._ops = list(ops)   # the structs must outlive the call
        opp = (C.c_void_p * n)(*[C.cast(C.pointer(o), C.c_void_p).value for o in self._ops])
        _check(load().ht_batch_step(self.ptr, opp, (C.c_double * n)(*map(float, dts)),
                                    (C.c_double * n)(*map(float, rel_tols)), (C.c_int * n)(*map(int, rmaxs)),
                                    scheme, _stream_ptr(stream)), "ht_batch_step")

    def close(self):
        if self.ptr:
            load().ht_batch_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ht_step_ab2(ctx: Context, u: HTTensor, u_prev: HTTensor, op: ht_op, dt: float, rel_tol: float, rmax: int,
                stream=None):
    _check(load().ht_step_ab2(ctx.ptr, C.byref(u.struct), C.byref(u_prev.struct), C.byref(op), dt, rel_tol, rmax,
                              _stream_ptr(stream)), "ht_step_ab2")


HT_AB2_SPLIT_ARGUMENT, HT_AB2_SPLIT_DIFFERENCE = 0, 1


def ht_add(ctx: Context, a: float, u: HTTensor, b: float, w: HTTensor, out: HTTensor, stream=None):
    _check(load().ht_add(ctx.ptr, float(a), C.byref(u.struct), float(b), C.byref(w.struct), C.byref(out.struct),
                         _stream_ptr(stream)), "ht_add")


def ht_step_ab2_split(ctx: Context, u: HTTensor, u_prev: HTTensor, op: ht_op, dt: float, rel_tol: float, rmax: int,
                      variant: int = HT_AB2_SPLIT_ARGUMENT, stream=None):
    _check(load().ht_step_ab2_split(ctx.ptr, C.byref(u.struct), C.byref(u_prev.struct), C.byref(op), dt, rel_tol,
                                    rmax, variant, _stream_ptr(stream)), "ht_step_ab2_split")


def ht_from_cp(ctx: Context, x: CPTensor, out: HTTensor, stream=None):
    _check(load().ht_from_cp(ctx.ptr, C.byref(x.struct), C.byref(out.struct), _stream_ptr(stream)), "ht_from_cp")


def ht_mass(ctx: Context, u: HTTensor, out, stream=None):
    _check(load().ht_mass(ctx.ptr, C.byref(u.struct), C.c_void_p(out.data_ptr()), _stream_ptr(stream)), "ht_mass")


def ht_inner(ctx: Context, u: HTTensor, w: HTTensor, out, stream=None):
    _check(load().ht_inner(ctx.ptr, C.byref(u.struct), C.byref(w.struct), C.c_void_p(out.data_ptr()),
                           _stream_ptr(stream)), "ht_inner")


def cp_apply_rk2(ctx: Context, x: CPTensor, op: ht_op, dt: float, y: CPTensor, stream=None):
    _check(load().cp_apply_rk2(ctx.ptr, C.byref(x.struct), C.byref(op), dt, C.byref(y.struct),
                               _stream_ptr(stream)), "cp_apply_rk2")


def cp_als_sweep(ctx: Context, y: CPTensor, x: CPTensor, sweeps: int, variant: int = CP_ALS_GS, eps=None,
                 stream=None):
    _check(load().cp_als_sweep(ctx.ptr, C.byref(y.struct), C.byref(x.struct), sweeps, variant,
                               C.c_void_p(eps.data_ptr() if eps is not None else 0), _stream_ptr(stream)),
           "cp_als_sweep")


def cp_als_sweep_rk2(ctx: Context, x_old: CPTensor, op: ht_op, dt: float, x: CPTensor, sweeps: int,
                     variant: int = CP_ALS_GS, eps=None, stream=None):
    _check(load().cp_als_sweep_rk2(ctx.ptr, C.byref(x_old.struct), C.byref(op), dt, C.byref(x.struct), sweeps,
                                   variant, C.c_void_p(eps.data_ptr() if eps is not None else 0),
                                   _stream_ptr(stream)), "cp_als_sweep_rk2")


def cp_als_rk2_cluster_ctas(ctx: Context, r: int, r0: int) -> int:
    """CTAs of the thread-block cluster cp_als_sweep_rk2 (Gauss-Seidel) runs on for ranks r and r0
    on this context, 0 when it takes the cooperative grid form."""
    out = C.c_int(0)
    _check(load().cp_als_rk2_cluster_ctas(ctx.ptr, int(r), int(r0), C.byref(out)), "cp_als_rk2_cluster_ctas")
    return int(out.value)


def cp_cn_als_step(ctx: Context, x_n: CPTensor, op: ht_op, dt: float, x: CPTensor, sweeps: int,
                   variant: int = CP_ALS_GS, eps=None, stream=None):
    _check(load().cp_cn_als_step(ctx.ptr, C.byref(x_n.struct), C.byref(op), dt, C.byref(x.struct), sweeps, variant,
                                 C.c_void_p(eps.data_ptr() if eps is not None else 0), _stream_ptr(stream)),
           "cp_cn_als_step")


def cp_als_sweep_noalloc(y: CPTensor, x: CPTensor, sweeps: int, variant: int = CP_ALS_GS, eps=None, status=None,
                         stream=None):
    """ALS sweeps without a context and without any device allocation (fixed-size static
    scratch; see include/htgpu.h for the limits and the rule on overlapping calls)."""
    _check(load().cp_als_sweep_noalloc(C.byref(y.struct), C.byref(x.struct), sweeps, variant,
                                       C.c_void_p(eps.data_ptr() if eps is not None else 0),
                                       C.c_void_p(status.data_ptr() if status is not None else 0),
                                       _stream_ptr(stream)), "cp_als_sweep_noalloc")


def selftest_fastmath(x, stream=None):
    """(n, 4) tensor: library reciprocal, CUDA 1.0 / x, library rsqrt, CUDA rsqrt of x (device
    FP64 tensor)."""
    import torch
    out = torch.empty((x.numel(), 4), dtype=torch.float64, device=x.device)
    _check(load().ht_selftest_fastmath(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel(),
                                       _stream_ptr(stream)), "ht_selftest_fastmath")
    return out


def selftest_gemm_mixed(A, B, C, m, n, k, lda, ldb, ldc, tA=0, tB=0, alpha=1.0, beta=0.0, colscale=None,
                        batch=1, sA=0, sB=0, sC=0, slices=4, stream=None):
    """A contraction of the mixed form on device FP64 buffers (column-major views given by leading
    dimensions and batch strides, in elements): slices 2..4 the tensor-core kernel, slices 1 the
    split-FP32 CUDA-core kernel."""
    return int(load().ht_selftest_gemm_mixed(m, n, k, C_ptr(A), lda, tA, C_ptr(B), ldb, tB, C_ptr(C), ldc,
                                             float(alpha), float(beta), C_ptr(colscale), batch, sA, sB, sC,
                                             slices, _stream_ptr(stream)))


def tune_time_gemm(m: int, n: int, k: int, batch: int = 1, route: int = 0, slices: int = 4, ctas_per_sm: int = 4,
                   reps: int = 20) -> float:
    """Mean time (ms) of one synthetic contraction through the FP64 (route 0), the tensor-core
    (route 1) or the split-FP32 (route 2) kernel, for the autotuner."""
    ms = C.c_double(0.0)
    _check(load().ht_tune_time_gemm(m, n, k, batch, route, slices, ctas_per_sm, reps, C.byref(ms)),
           "ht_tune_time_gemm")
    return float(ms.value)


def C_ptr(t):
    return C.c_void_p(t.data_ptr() if t is not None else 0)


def selftest_grid_barrier(nblocks: int, absent: int = -1, device: int = 0) -> int:
    """Status of one bounded grid barrier over nblocks CTAs with CTA `absent` missing (-1: none)."""
    return int(load().ht_selftest_grid_barrier(nblocks, absent, device))
