"""Python binding of the GB300 HPS solver C ABI (include/hps.h).

The functions carry the C names and only marshal arguments: sizes and dtypes
are checked, tensors / arrays are turned into pointers and the current CUDA
stream is passed along.  Every step of the solver runs in libhps_gb300.so; if
the library is missing the first call raises ImportError (there is no
fallback).

Arrays may be torch tensors (CUDA or CPU) or NumPy arrays.  Host arrays are
staged to the device by the library itself.
"""

from __future__ import annotations

import ctypes
from ctypes import byref, c_int64, c_void_p

import numpy as np

from . import _capi
from ._capi import (HPS_C128, HPS_DTN, HPS_F64, HPS_ITI, HPS_OK, hps_coeffs,  # noqa: F401
                    hps_options, hps_tree)

__all__ = ["hps_nodes", "hps_sizes", "hps_build", "hps_solve", "hps_solve_batched", "hps_free",
           "hps_error_string", "hps_last_error_detail", "hps_device_bytes",
           "hps_last_launch_count", "hps_kernel_stats", "hps_set_profiling", "hps_solve_noalloc",
           "hps_solve_multi",
           "uniform_tree", "adaptive_tree", "hps_refine",
           "make_coeffs", "HPSError", "Handle"]


class HPSError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _capi.lib().hps_error_string(status).decode()
        super().__init__(f"{where}: {msg}")


def _check(status: int, where: str):
    if status != HPS_OK:
        raise HPSError(status, where)


def uniform_tree(dim: int, depth: int, lo=None, hi=None) -> hps_tree:
    lo = lo if lo is not None else (-1.0,) * dim
    hi = hi if hi is not None else (1.0,) * dim
    t = hps_tree()
    t.dim = dim
    for a in range(3):
        t.lo[a] = float(lo[a]) if a < dim else 0.0
        t.hi[a] = float(hi[a]) if a < dim else 0.0
    t.uniform_depth = depth
    t.n_leaves = 2 ** (dim * depth)
    t.morton = None
    t.level = None
    return t


def morton_code(ix) -> int:
    """Morton code of integer coordinates (x in the lowest bit)."""
    c = 0
    for b in range(21):
        for a in range(3):
            c |= ((int(ix[a]) >> b) & 1) << (3 * b + a)
    return c


def adaptive_tree(leaves, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)) -> hps_tree:
    """hps_tree of an adaptive octree from leaves [(level, (ix, iy, iz))] in
    depth-first Morton order (the arrays are kept alive by the returned
    structure)."""
    t = hps_tree()
    t.dim = 3
    for a in range(3):
        t.lo[a] = float(lo[a])
        t.hi[a] = float(hi[a])
    t.uniform_depth = -1
    t.n_leaves = len(leaves)
    mort = np.array([morton_code(ix) for _, ix in leaves], dtype=np.uint64)
    lev = np.array([lv for lv, _ in leaves], dtype=np.int8)
    t.morton = mort.ctypes.data
    t.level = lev.ctypes.data
    t._keep = (mort, lev)
    return t


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, complex_: bool, n: int, name: str, keep: list):
    """Pointer of a contiguous float64 / complex128 buffer with n elements."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        want = torch.complex128 if complex_ else torch.float64
        if x.dtype != want:
            raise TypeError(f"{name}: dtype {x.dtype}, expected {want}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if x.numel() != n:
            raise ValueError(f"{name}: {x.numel()} elements, expected {n}")
        keep.append(x)
        return x.data_ptr()
    a = np.asarray(x)
    want = np.complex128 if complex_ else np.float64
    if a.dtype != want:
        raise TypeError(f"{name}: dtype {a.dtype}, expected {np.dtype(want)}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name}: array must be C-contiguous")
    if a.size != n:
        raise ValueError(f"{name}: {a.size} elements, expected {n}")
    keep.append(a)
    return a.ctypes.data


def _stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def hps_sizes(tree: hps_tree, p: int, q: int):
    nl, ppl, nr = c_int64(), c_int64(), c_int64()
    _check(_capi.lib().hps_sizes(byref(tree), p, q, byref(nl), byref(ppl), byref(nr)), "hps_sizes")
    return nl.value, ppl.value, nr.value


def hps_nodes(tree: hps_tree, p: int, q: int):
    """(leaf_xyz, bdry_xyz) as NumPy arrays of shape (n, dim)."""
    nl, ppl, nr = hps_sizes(tree, p, q)
    leaf = np.zeros((nl * ppl, tree.dim))
    bdry = np.zeros((nr, tree.dim))
    _check(_capi.lib().hps_nodes(byref(tree), p, q, leaf.ctypes.data, bdry.ctypes.data), "hps_nodes")
    return leaf, bdry


class Handle:
    """Owns an hps_handle*; released by hps_free (or garbage collection)."""

    def __init__(self, ptr, tree, p, q, complex_):
        self.ptr = ptr
        self.dim = tree.dim
        self.tree = tree
        self.p, self.q = p, q
        self.complex = complex_
        self.n_leaves, self.ppl, self.n_root = hps_sizes(tree, p, q)

    def __del__(self):
        try:
            hps_free(self)
        except Exception:
            pass


def make_coeffs(kind: int, a=None, b=None, c=None, eta: float = 0.0, keep=None, n=None):
    cf = hps_coeffs()
    cf.kind = kind
    cf.dtype = HPS_C128 if kind == HPS_ITI else HPS_F64
    cf.eta = float(eta)
    keep = keep if keep is not None else []
    cf.a = _ptr(a, False, n, "a", keep) if a is not None else None
    for k in range(3):
        bk = b[k] if (b is not None and k < len(b)) else None
        cf.b[k] = _ptr(bk, False, n, f"b[{k}]", keep) if bk is not None else None
    cf.c = _ptr(c, False, n, "c", keep) if c is not None else None
    return cf, keep


def hps_build(tree: hps_tree, p: int, q: int, kind: int, a=None, b=None, c=None, f=None,
              eta: float = 0.0, want_root_map: bool = False, profile: bool = False,
              lazy_root: bool = False, graph_solve: bool = False, iti_leaf: int = 0, fp64_gemm: bool = False,
              recompute_budget_mb: int = 0, stream=None) -> Handle:
    """Build the solution operator; coefficient and source arrays hold
    n_leaves * p^dim values (leaf-major, tensor node order).  fp64_gemm=True
    keeps every product on the FP64 pipe (default: large products on the
    tensor cores as exact digit-slice products)."""
    nl, ppl, _ = hps_sizes(tree, p, q)
    n = nl * ppl
    keep: list = []
    cf, keep = make_coeffs(kind, a, b, c, eta, keep, n)
    fp = _ptr(f, kind == HPS_ITI, n, "f", keep)
    opts = hps_options()
    opts.version = 1
    opts.want_root_map = 1 if want_root_map else 0
    opts.profile = 1 if profile else 0
    opts.lazy_root = 1 if lazy_root else 0
    opts.graph_solve = 1 if graph_solve else 0
    opts.iti_leaf = int(iti_leaf)
    opts.fp64_gemm = 1 if fp64_gemm else 0
    opts.recompute_budget_mb = int(recompute_budget_mb)
    out = c_void_p()
    st = _stream(stream)
    _check(_capi.lib().hps_build(byref(tree), p, q, byref(cf), fp, byref(opts), st, byref(out)),
           "hps_build")
    return Handle(out.value, tree, p, q, kind == HPS_ITI)


def hps_solve_batched(h: Handle, nrhs: int, g, u, f=None, stream=None):
    keep: list = []
    gp = _ptr(g, h.complex, nrhs * h.n_root, "g", keep)
    up = _ptr(u, h.complex, nrhs * h.n_leaves * h.ppl, "u", keep)
    fp = _ptr(f, h.complex, nrhs * h.n_leaves * h.ppl, "f", keep)
    _check(_capi.lib().hps_solve_batched(h.ptr, nrhs, gp, fp, up, _stream(stream)), "hps_solve")
    return u


def hps_solve(h: Handle, g, u, f=None, stream=None):
    """u <- solution for root boundary data g (and source f, or the build-time
    source when f is None)."""
    return hps_solve_batched(h, 1, g, u, f=f, stream=stream)


def hps_solve_multi(handles, gs, us, nrhs=None, stream=None):
    """Apply-only solves (build-time source) of several different operators
    in shared launches: us[i] <- solution of handles[i] for gs[i] (nrhs[i]
    right-hand sides each, default 1).  Device tensors only."""
    n = len(handles)
    if len(gs) != n or len(us) != n:
        raise ValueError("handles, gs and us must have the same length")
    nr = [1] * n if nrhs is None else [int(k) for k in nrhs]
    keep: list = []
    hp = (c_void_p * n)(*[h.ptr for h in handles])
    gp = (c_void_p * n)(*[_ptr(gs[i], handles[i].complex, nr[i] * handles[i].n_root, "g", keep)
                          for i in range(n)])
    up = (c_void_p * n)(*[_ptr(us[i], handles[i].complex, nr[i] * handles[i].n_leaves * handles[i].ppl, "u",
                               keep) for i in range(n)])
    npr = (ctypes.c_int * n)(*nr)
    _check(_capi.lib().hps_solve_multi(n, hp, npr, gp, up, _stream(stream)), "hps_solve_multi")
    return us


def hps_solve_noalloc(h: Handle, g, u, stream=None):
    """Allocation-free variant of hps_solve with the build-time source: g and u
    must be device tensors; the library uses its static 16 MiB device array
    instead of allocating (see include/hps.h for the limits)."""
    keep: list = []
    gp = _ptr(g, h.complex, h.n_root, "g", keep)
    up = _ptr(u, h.complex, h.n_leaves * h.ppl, "u", keep)
    _check(_capi.lib().hps_solve_noalloc(h.ptr, gp, up, _stream(stream)), "hps_solve_noalloc")
    return u


def hps_refine(lo, hi, p: int, eps: float, min_depth: int, max_depth: int, funcs, stream=None):
    """Adaptive refinement in the library (device interpolation check, 2:1
    balance); funcs are Python callables f(xyz (n, 3)) -> values (n,),
    evaluated when the library asks for samples.  Returns the leaves as
    [(level, (ix, iy, iz))] in the order adaptive_tree() expects."""
    errors = []

    def wrap(fn):
        def cb(ctx, n, xyz, out):
            try:
                x = np.ctypeslib.as_array(xyz, shape=(n, 3))
                o = np.ctypeslib.as_array(out, shape=(n,))
                o[:] = np.asarray(fn(x), dtype=np.float64)
                return 0
            except Exception as e:  # noqa: BLE001
                errors.append(e)
                return 1
        return _capi.EVAL_FN(cb)

    cbs = [wrap(fn) for fn in funcs]
    arr = (_capi.EVAL_FN * len(cbs))(*cbs)
    lo3 = (ctypes.c_double * 3)(*[float(v) for v in lo])
    hi3 = (ctypes.c_double * 3)(*[float(v) for v in hi])
    L = _capi.lib()
    st = _stream(stream)
    cap = min(8 ** max_depth, 1 << 22)
    mort = np.zeros(cap, np.uint64)
    lev = np.zeros(cap, np.int8)
    n = c_int64(0)
    _check(L.hps_refine(lo3, hi3, p, eps, min_depth, max_depth, len(cbs), arr, None, cap, byref(n),
                        mort.ctypes.data, lev.ctypes.data, st), "hps_refine")
    mort, lev = mort[:n.value], lev[:n.value]
    if errors:
        raise errors[0]
    out = []
    for code, lv in zip(mort.tolist(), lev.tolist()):
        ix = [0, 0, 0]
        for b in range(lv):
            for a in range(3):
                ix[a] |= ((code >> (3 * b + a)) & 1) << b
        out.append((lv, tuple(ix)))
    return out


def hps_free(h: Handle):
    if h is not None and h.ptr:
        _capi.lib().hps_free(h.ptr)
        h.ptr = None


def hps_error_string(status: int) -> str:
    return _capi.lib().hps_error_string(status).decode()


def hps_last_error_detail(h: Handle | None = None) -> int:
    node = c_int64()
    _check(_capi.lib().hps_last_error_detail(h.ptr if h else None, byref(node)), "hps_last_error_detail")
    return node.value


def hps_device_bytes(h: Handle) -> int:
    return int(_capi.lib().hps_device_bytes(h.ptr))


def hps_last_launch_count(h: Handle) -> int:
    return int(_capi.lib().hps_last_launch_count(h.ptr))


def hps_kernel_stats(h: Handle) -> dict:
    """{class name: {"launches", "flops", "exec_flops", "ms"}} for the last
    build / solve (flops: algorithmic, complex multiply-add = 8; exec_flops:
    what the FP64 pipe executes)."""
    out = {}
    for k, name in enumerate(_capi.KCLASSES):
        st = _capi.hps_kernel_stat()
        _check(_capi.lib().hps_kernel_stats(h.ptr, k, byref(st)), "hps_kernel_stats")
        out[name] = {"launches": st.launches, "flops": st.flops, "exec_flops": st.exec_flops, "ms": st.ms}
    return out


def hps_trace(h: Handle) -> list:
    """Per-launch records of the last build / solve on h (profiling on):
    [{"kclass", "m", "n", "k", "batch", "flops", "ms"}] in launch order."""
    n = c_int64(0)
    _check(_capi.lib().hps_trace_count(h.ptr, byref(n)), "hps_trace_count")
    out = []
    rec = _capi.hps_trace_rec()
    for i in range(n.value):
        _check(_capi.lib().hps_trace_get(h.ptr, i, byref(rec)), "hps_trace_get")
        out.append({"kclass": _capi.KCLASSES[rec.kclass], "m": rec.m, "n": rec.n, "k": rec.k,
                    "batch": rec.batch, "flops": rec.flops, "ms": rec.ms})
    return out


def hps_set_profiling(h: Handle, on: bool):
    _check(_capi.lib().hps_set_profiling(h.ptr, 1 if on else 0), "hps_set_profiling")




def hps_plan_bytes(tree: hps_tree, p: int, q: int, kind: int) -> int:
    """Planned device bytes of the handle hps_build would create (uniform trees)."""
    out = c_int64(0)
    _check(_capi.lib().hps_plan_bytes(byref(tree), p, q, kind, byref(out)), "hps_plan_bytes")
    return out.value


class _Borrowed(Handle):
    """A server-owned operator, for inspection only (never freed here)."""

    def __del__(self):
        self.ptr = None


class Server:
    """Request server of include/hps_serve.h: resident operators in slots,
    solve requests merged into batched solves on a pool of streams, builds
    on a separate thread, admitted by planned device footprint.  Buffers are
    host numpy arrays; the server keeps references until a request is
    waited for."""

    def __init__(self, n_slots: int = 16, n_streams: int = 4, max_batch: int = 8, hbm_budget: int = 0,
                 lazy_root: bool = False, n_builders: int = 2, max_group: int = 8):
        o = _capi.hps_server_options()
        o.version = 1
        o.n_slots, o.n_streams, o.max_batch = n_slots, n_streams, max_batch
        o.hbm_budget = hbm_budget
        o.lazy_root = 1 if lazy_root else 0
        o.n_builders = n_builders
        o.max_group = max_group
        out = c_void_p()
        _check(_capi.lib().hps_server_create(byref(o), byref(out)), "hps_server_create")
        self.ptr = out.value
        self._keep: dict = {}
        self._meta: dict = {}   # slot -> (tree, p, q, complex) of the last submitted build

    def submit_build(self, slot: int, tree: hps_tree, p: int, q: int, kind: int, a=None, b=None, c=None,
                     f=None, eta: float = 0.0, lazy_root=None) -> int:
        nl, ppl, _ = hps_sizes(tree, p, q)
        n = nl * ppl
        keep: list = [tree]
        cf, keep = make_coeffs(kind, a, b, c, eta, keep, n)
        fp = _ptr(f, kind == HPS_ITI, n, "f", keep)
        optp = None
        if lazy_root is not None:
            opts = hps_options()
            opts.version = 1
            opts.lazy_root = 1 if lazy_root else 0
            keep.append(opts)
            optp = byref(opts)
        keep.append(cf)
        t = c_int64(0)
        _check(_capi.lib().hps_server_submit_build(self.ptr, slot, byref(tree), p, q, byref(cf), fp, optp,
                                                   byref(t)), "hps_server_submit_build")
        self._keep[t.value] = keep
        self._meta[slot] = (tree, p, q, kind == HPS_ITI)
        return t.value

    def submit_solve(self, slot: int, g, u, f=None) -> int:
        if slot not in self._meta:
            raise ValueError(f"slot {slot} has no build submitted")
        tree, p, q, cplx_ = self._meta[slot]
        nl, ppl, nr = hps_sizes(tree, p, q)
        keep: list = []
        gp = _ptr(g, cplx_, nr, "g", keep)
        up = _ptr(u, cplx_, nl * ppl, "u", keep)
        fp = _ptr(f, cplx_, nl * ppl, "f", keep)
        for x in keep:
            if _is_torch(x):
                raise TypeError("server buffers are host numpy arrays")
        t = c_int64(0)
        _check(_capi.lib().hps_server_submit_solve(self.ptr, slot, gp, fp, up, byref(t)),
               "hps_server_submit_solve")
        self._keep[t.value] = keep
        return t.value

    @staticmethod
    def _info(ti) -> dict:
        return {"status": ti.status, "kind": "build" if ti.kind == 1 else "solve", "slot": ti.slot,
                "batch": ti.batch, "t_submit_ms": ti.t_submit_ms, "t_start_ms": ti.t_start_ms,
                "t_done_ms": ti.t_done_ms}

    def wait(self, ticket: int, check: bool = True) -> dict:
        ti = _capi.hps_ticket_info()
        ti.status = 1  # stays set when the ticket is unknown (nothing filled in)
        st = _capi.lib().hps_server_wait(self.ptr, ticket, byref(ti))
        self._keep.pop(ticket, None)
        if ti.status == 1:
            ti.status = st
        if st == HPS_OK or not check:
            return self._info(ti)
        raise HPSError(st, "hps_server_wait")

    def poll(self, ticket: int):
        ti = _capi.hps_ticket_info()
        st = _capi.lib().hps_server_poll(self.ptr, ticket, byref(ti))
        if st == _capi.HPS_PENDING:
            return None
        self._keep.pop(ticket, None)
        if st != HPS_OK:
            raise HPSError(st, "hps_server_poll")
        return self._info(ti)

    def stats(self) -> dict:
        s = _capi.hps_server_stats()
        _check(_capi.lib().hps_server_get_stats(self.ptr, byref(s)), "hps_server_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def operator(self, slot: int):
        """The slot's operator (a borrowed handle) once its requests are done."""
        out = c_void_p()
        _check(_capi.lib().hps_server_operator(self.ptr, slot, byref(out)), "hps_server_operator")
        if not out.value:
            return None
        tree, p, q, cplx_ = self._meta[slot]
        return _Borrowed(out.value, tree, p, q, cplx_)

    def close(self):
        if self.ptr:
            _capi.lib().hps_server_destroy(self.ptr)
            self.ptr = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hps_solve_adjoint(h: Handle, ubar, gbar=None, fbar=None, nrhs: int = 1, stream=None):
    """(gbar, fbar) <- conjugate transpose of the solve map applied to ubar."""
    keep: list = []
    n = nrhs * h.n_leaves * h.ppl
    up = _ptr(ubar, h.complex, n, "ubar", keep)
    gp = _ptr(gbar, h.complex, nrhs * h.n_root, "gbar", keep)
    fp = _ptr(fbar, h.complex, n, "fbar", keep)
    _check(_capi.lib().hps_solve_adjoint(h.ptr, nrhs, up, gp, fp, _stream(stream)), "hps_solve_adjoint")
    return gbar, fbar


def hps_coeff_gradient(h: Handle, u, fbar, ga=None, gb=None, gc=None, nrhs: int = 1, stream=None):
    """Coefficient derivatives at the leaf interior nodes (device tensors)."""
    keep: list = []
    n = h.n_leaves * h.ppl
    up = _ptr(u, h.complex, nrhs * n, "u", keep)
    fp = _ptr(fbar, h.complex, nrhs * n, "fbar", keep)
    ap = _ptr(ga, False, n, "ga", keep)
    bp = _ptr(gb, False, h.dim * n, "gb", keep)
    cp = _ptr(gc, False, n, "gc", keep)
    _check(_capi.lib().hps_coeff_gradient(h.ptr, nrhs, up, fp, ap, bp, cp, _stream(stream)),
           "hps_coeff_gradient")


def hps_gemm(A, B, C, alpha: float = 1.0, beta: float = 0.0, mode: int = 0, stream=None):
    """C <- alpha A B + beta C for batches of column-major matrices held as
    contiguous device tensors of shape (batch, cols, rows) (that is, each
    item's columns are contiguous): A (batch, k, m), B (batch, n, k),
    C (batch, n, m); float64 or complex128.  mode 0: tensor-core digit-slice
    product; mode 1: FP64 pipe.  Synchronises the stream."""
    if not (_is_torch(A) and _is_torch(B) and _is_torch(C)):
        raise TypeError("hps_gemm: A, B and C must be device tensors")
    if A.dim() != 3 or B.dim() != 3 or C.dim() != 3:
        raise ValueError("hps_gemm: tensors must be (batch, cols, rows)")
    batch, k, m = A.shape
    _, n, k2 = B.shape
    if B.shape[0] != batch or tuple(C.shape) != (batch, n, m) or k2 != k:
        raise ValueError("hps_gemm: shapes do not match")
    cp = A.is_complex()
    keep: list = []
    ap = _ptr(A, cp, A.numel(), "A", keep)
    bp = _ptr(B, cp, B.numel(), "B", keep)
    cq = _ptr(C, cp, C.numel(), "C", keep)
    _check(_capi.lib().hps_gemm(HPS_C128 if cp else HPS_F64, int(mode), m, n, k, batch, float(alpha), ap,
                                max(m, 1), m * k, bp, max(k, 1), k * n, float(beta), cq, max(m, 1), m * n,
                                _stream(stream)), "hps_gemm")
    return C


def hps_getrf(A, ipiv=None, info=None, mode: int = 0, stream=None):
    """LU with partial pivoting, in place, of a batch of column-major n x n
    matrices held as a contiguous device tensor of shape (batch, n, n) (each
    item's columns contiguous), float64 or complex128: LAPACK's getrf
    convention (unit L below the diagonal, U on and above it, 0-based
    interchanges).  Returns (A, ipiv, info) with ipiv (batch, n) and info
    (batch,) int32 device tensors.  mode 0: trailing updates on the tensor
    cores as in hps_build; mode 1: FP64 pipe only.  Synchronises the stream."""
    import torch
    if not _is_torch(A) or A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("hps_getrf: A must be a (batch, n, n) device tensor")
    batch, n, _ = A.shape
    cp = A.is_complex()
    if ipiv is None:
        ipiv = torch.empty((batch, n), dtype=torch.int32, device=A.device)
    if info is None:
        info = torch.empty((batch,), dtype=torch.int32, device=A.device)
    for t, nm, cnt in ((ipiv, "ipiv", batch * n), (info, "info", batch)):
        if not _is_torch(t) or t.dtype != torch.int32 or not t.is_contiguous() or t.numel() != cnt:
            raise ValueError(f"hps_getrf: {nm} must be a contiguous int32 device tensor of {cnt} elements")
    keep: list = []
    ap = _ptr(A, cp, A.numel(), "A", keep)
    _check(_capi.lib().hps_getrf(HPS_C128 if cp else HPS_F64, int(mode), n, batch, ap, max(n, 1), n * n,
                                 ipiv.data_ptr(), info.data_ptr(), _stream(stream)), "hps_getrf")
    return A, ipiv, info


def hps_debug_fail_alloc(n: int) -> None:
    """Fault injection for tests: the n-th handle allocation from now on fails
    as out-of-memory (host side); n <= 0 disarms."""
    _capi.lib().hps_debug_fail_alloc(int(n))


def hps_debug_alloc_count() -> int:
    """Handle allocations made so far in this process."""
    return int(_capi.lib().hps_debug_alloc_count())


def hps_debug_wait_timeout(which: int, satisfied: bool, limit_polls: int, stream=None) -> int:
    """Run one of the library's bounded device waits on a word nothing writes
    (which 0: inter-CTA group barrier, 1: triangular-solve flag wait,
    2: tensor-core pipeline mbarrier wait).  Returns the status code:
    HPS_ERR_TIMEOUT when the wait gave up, HPS_OK when it passed."""
    return int(_capi.lib().hps_debug_wait_timeout(int(which), 1 if satisfied else 0, int(limit_polls),
                                                   _stream(stream)))


TUNE_PARAMS = {"lu_base_panels_few": 0, "lu_base_panels_many": 1, "lu_few_min_n": 2, "lu_cluster_panel": 3,
               "tc_min_work_real": 4, "tc_min_work_cplx": 5, "tc_min_k": 6,
               "tc_chunk_mb": 7, "tc_persist_min_k": 8, "lu_panel_nb_few": 9}


def hps_tune_set(name: str, value: int) -> None:
    """Set one of the batched LU's shape choices (include/hps.h)."""
    _check(_capi.lib().hps_tune_set(TUNE_PARAMS[name], int(value)), "hps_tune_set")


def hps_tune_get(name: str) -> int:
    v = ctypes.c_int(0)
    _check(_capi.lib().hps_tune_get(TUNE_PARAMS[name], byref(v)), "hps_tune_get")
    return int(v.value)
