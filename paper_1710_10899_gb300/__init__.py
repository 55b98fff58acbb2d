"""GB300 submatrix method: A^(-1/p) of a sparse SPD matrix on A's own sparsity pattern.

Thin Python binding of ``libsubmat.so`` (C ABI in ``include/submat.h``): argument
marshalling only, every step of the computation runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.

    plan = submat_plan(rowptr, colind, p=2)              # Alg. 1 index part, on the GPU
    y = submat_invroot(plan, vals)                       # Alg. 1, Sec. 3.2, Alg. 2
    g = submat_invroot_backward(plan, grad_y)            # Daleckii-Krein adjoint
    y = SubmatInvRoot.apply(vals, plan)                  # autograd
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsubmat.so")

SUBMAT_MAX_M = 1536
SUBMAT_SMALL_MAX_M = 32
SUBMAT_MIXED_MAX_P = 10
PREC_FP64 = 0
PREC_MIXED_F16 = 1
PREC_MIXED_F16_SYNC = 2
PRECISIONS = {"fp64": PREC_FP64, "mixed": PREC_MIXED_F16, "mixed_sync": PREC_MIXED_F16_SYNC}

STATUS = {
    0: "SUBMAT_OK", 1: "SUBMAT_EINVAL", 2: "SUBMAT_ENODIAG", 3: "SUBMAT_ENOTSYM",
    4: "SUBMAT_ETOOBIG", 5: "SUBMAT_ENOMEM", 6: "SUBMAT_ECUDA", 7: "SUBMAT_ENOTSPD",
    8: "SUBMAT_ENOFWD", 9: "SUBMAT_ETIMEOUT",
}


class SubmatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("tol", ctypes.c_double), ("resid_tol", ctypes.c_double),
                ("refine_steps", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("kappa_max", ctypes.c_double), ("root_sign", ctypes.c_int32),
                ("grad_deterministic", ctypes.c_int32), ("grad_wave_mib", ctypes.c_int32),
                ("shard_count", ctypes.c_int32), ("shard_rank", ctypes.c_int32),
                ("small_max_m", ctypes.c_int32), ("sync_max_m", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("m_max", ctypes.c_int32),
                ("iters_max", ctypes.c_int32), ("iters_sum", ctypes.c_int64),
                ("n_fallback", ctypes.c_int64), ("n_notspd", ctypes.c_int64),
                ("max_resid", ctypes.c_double), ("sum_m3", ctypes.c_double),
                ("flops_tensor", ctypes.c_double), ("flops_fp64", ctypes.c_double),
                ("ms_kernel", ctypes.c_float), ("ms_fallback", ctypes.c_float),
                ("n_illcond", ctypes.c_int64), ("flops_alg", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["submat_default_opts", "submat_plan", "submat_invroot", "submat_invroot_host",
           "submat_invroot_backward",
           "submat_get_report", "submat_plan_rows", "submat_plan_shape", "submat_plan_destroy",
           "submat_status_string", "submat_last_error", "submat_invroot_noalloc", "submat_pcg",
           "submat_shard_rows", "submat_test_stall", "submat_refine"]

_lib_handle = None


def load_library(path: str = LIB_PATH):
    """Load libsubmat.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_1710_10899_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.submat_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.submat_default_opts.restype = None
    lib.submat_plan.argtypes = [ctypes.POINTER(CSR), i32, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    lib.submat_plan.restype = i32
    lib.submat_invroot.argtypes = [vp, vp, vp, vp, i32]
    lib.submat_invroot.restype = i32
    lib.submat_invroot_host.argtypes = [vp, vp, vp, vp]
    lib.submat_invroot_host.restype = i32
    lib.submat_invroot_backward.argtypes = [vp, vp, vp, vp]
    lib.submat_invroot_backward.restype = i32
    lib.submat_get_report.argtypes = [vp, ctypes.POINTER(Report)]
    lib.submat_get_report.restype = i32
    lib.submat_plan_rows.argtypes = [vp, vp, vp]
    lib.submat_plan_rows.restype = i32
    lib.submat_plan_shape.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64)]
    lib.submat_plan_shape.restype = i32
    lib.submat_plan_destroy.argtypes = [vp]
    lib.submat_plan_destroy.restype = None
    lib.submat_status_string.argtypes = [i32]
    lib.submat_status_string.restype = ctypes.c_char_p
    lib.submat_last_error.argtypes = []
    lib.submat_last_error.restype = ctypes.c_char_p
    lib.submat_invroot_noalloc.argtypes = [i32, ctypes.c_int64, vp, vp, i32, i32, vp, vp, vp]
    lib.submat_invroot_noalloc.restype = i32
    lib.submat_pcg.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, i32, ctypes.POINTER(i32),
                               ctypes.POINTER(ctypes.c_double), vp]
    lib.submat_pcg.restype = i32
    lib.submat_shard_rows.argtypes = [i32, vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.submat_shard_rows.restype = i32
    lib.submat_test_stall.argtypes = [vp, i32]
    lib.submat_test_stall.restype = i32
    lib.submat_refine.argtypes = [vp, vp, vp, i32, i32, vp, vp]
    lib.submat_refine.restype = i32
    _lib_handle = lib
    return lib


def _check(lib, st):
    if st != 0:
        raise SubmatError(st, lib.submat_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A plan for one sparsity pattern and root order p (``submat_plan``)."""

    def __init__(self, rowptr, colind, p: int, precision: str = "mixed", k_max: int = 0,
                 tol: float = 0.0, resid_tol: float = 0.0, refine_steps: int = -1,
                 use_graph: bool = True, kappa_max: float = 0.0, root_sign: int = -1,
                 grad_deterministic: bool = False, grad_wave_mib: int = 0, shard=(0, 1),
                 small_max_m: int = -1, sync_max_m: int = -1):
        lib = load_library()
        self._lib = lib
        torch = _torch()
        keep = []
        if isinstance(rowptr, torch.Tensor):
            rp = rowptr.to(torch.int32).contiguous()
            ci = colind.to(device=rp.device, dtype=torch.int32).contiguous()
            on_dev = 1 if rp.is_cuda else 0
            keep += [rp, ci]
            rp_ptr, ci_ptr = rp.data_ptr(), ci.data_ptr()
            n, nnz = rp.numel() - 1, ci.numel()
        else:
            rp = np.ascontiguousarray(rowptr, dtype=np.int32)
            ci = np.ascontiguousarray(colind, dtype=np.int32)
            keep += [rp, ci]
            on_dev = 0
            rp_ptr, ci_ptr = rp.ctypes.data, ci.ctypes.data
            n, nnz = rp.shape[0] - 1, ci.shape[0]
        self.rowptr_host = (rp.cpu().numpy() if isinstance(rp, torch.Tensor) else rp).astype(np.int32)
        csr = CSR(n, nnz, rp_ptr, ci_ptr if nnz > 0 else None, on_dev)
        o = Opts()
        lib.submat_default_opts(ctypes.byref(o))
        o.precision = PRECISIONS[precision]
        o.k_max = k_max
        o.tol = tol
        o.resid_tol = resid_tol
        o.refine_steps = refine_steps
        o.use_graph = 1 if use_graph else 0
        o.kappa_max = kappa_max
        o.root_sign = int(root_sign)
        o.grad_deterministic = 1 if grad_deterministic else 0
        o.grad_wave_mib = int(grad_wave_mib)
        o.shard_rank, o.shard_count = int(shard[0]), int(shard[1])
        if small_max_m >= 0:
            o.small_max_m = int(small_max_m)
        if sync_max_m >= 0:
            o.sync_max_m = int(sync_max_m)
        h = ctypes.c_void_p()
        _check(lib, lib.submat_plan(ctypes.byref(csr), int(p), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.n = int(n)
        self.nnz = int(nnz)
        self.p = int(p)
        self.precision = precision
        self.root_sign = int(root_sign)
        self.small_max_m = int(o.small_max_m)
        self.sync_max_m = int(o.sync_max_m)
        self.shard = (int(shard[0]), int(shard[1]))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._fwd_gen = 0              # forwards run on this plan (the backward's input)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.submat_plan_destroy(h)
            self._h = None

    def rows(self):
        """(m, pos) as computed on the device: m_j = |R_j|, pos_j = R_j.indexof(j)."""
        m = np.zeros(self.n, dtype=np.int32)
        pos = np.zeros(self.n, dtype=np.int32)
        _check(self._lib, self._lib.submat_plan_rows(self._h, m.ctypes.data, pos.ctypes.data))
        return m, pos

    def engine_launches(self):
        """Kernel launches of one forward: one per engine that gets rows (the plan's size
        buckets; the FP64 path has one), plus the fallback kernel."""
        if self.precision == "fp64":
            return 2
        m, _ = self.rows()
        b, e = shard_rows(self.rowptr_host, self.shard[1], self.shard[0])
        m = m[b:e]
        if self.precision == "mixed_sync":
            return 1 + int(len(m) > 0)
        small = m <= self.small_max_m
        sync = (~small) & (m <= self.sync_max_m)
        tc = ~(small | sync)
        return 1 + int(small.any()) + int(sync.any()) + int(tc.any())

    def test_stall(self, on: bool):
        """``submat_test_stall``: make the tensor-core forward's first pipeline wait run out
        (test aid for the bounded device waits; the forward then returns SUBMAT_ETIMEOUT)."""
        _check(self._lib, self._lib.submat_test_stall(self._h, 1 if on else 0))

    def report(self) -> dict:
        r = Report()
        _check(self._lib, self._lib.submat_get_report(self._h, ctypes.byref(r)))
        return r.as_dict()

    def _vals(self, t):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
            raise TypeError("expected a CUDA float64 tensor")
        if t.numel() != self.nnz:
            raise ValueError(f"expected {self.nnz} values, got {t.numel()}")
        return t.contiguous()

    def invroot(self, vals, out=None, stream=None, sync: bool = False):
        torch = _torch()
        v = self._vals(vals)
        if out is None:
            out = torch.empty_like(v)
        self._fwd_gen += 1             # the library saves this call's input for the backward
        _check(self._lib, self._lib.submat_invroot(self._h, ctypes.c_void_p(v.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()),
                                                   _stream_ptr(stream), 1 if sync else 0))
        return out

    def invroot_host(self, vals_in, vals_out=None, stream=None):
        """Forward on host arrays (numpy float64 or CPU tensors, pinned for async copies)."""
        torch = _torch()
        if isinstance(vals_in, torch.Tensor):
            src = vals_in.contiguous()
            ptr_in = src.data_ptr()
        else:
            src = np.ascontiguousarray(vals_in, dtype=np.float64)
            ptr_in = src.ctypes.data
        if vals_out is None:
            vals_out = np.empty(self.nnz, dtype=np.float64)
        ptr_out = vals_out.data_ptr() if isinstance(vals_out, torch.Tensor) \
            else vals_out.ctypes.data
        self._fwd_gen += 1
        _check(self._lib, self._lib.submat_invroot_host(self._h, ctypes.c_void_p(ptr_in),
                                                        ctypes.c_void_p(ptr_out),
                                                        _stream_ptr(stream)))
        return vals_out

    def backward(self, grad_out, grad_in=None, stream=None):
        torch = _torch()
        g = self._vals(grad_out)
        if grad_in is None:
            grad_in = torch.empty_like(g)
        _check(self._lib, self._lib.submat_invroot_backward(
            self._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(grad_in.data_ptr()),
            _stream_ptr(stream)))
        return grad_in


def submat_plan(rowptr, colind, p: int, **kw) -> Plan:
    """``submat_plan``: validate A's pattern and build the integer plan (Alg. 1)."""
    return Plan(rowptr, colind, p, **kw)


def submat_invroot(plan: Plan, vals_in, vals_out=None, stream=None, sync: bool = False):
    """``submat_invroot``: the submatrix method's A^(-1/p) on A's pattern."""
    return plan.invroot(vals_in, vals_out, stream, sync)


def submat_invroot_backward(plan: Plan, grad_out, grad_in=None, stream=None):
    """``submat_invroot_backward``: gradient w.r.t. A's stored values (last forward)."""
    return plan.backward(grad_out, grad_in, stream)


def submat_pcg(plan: Plan, vals_a, b=None, vals_k=None, tol: float = 1e-6, max_iter: int = 0,
               stream=None):
    """``submat_pcg``: conjugate gradients on A x = b (b defaults to ones) for A on the
    plan's pattern, plain or, with ``vals_k`` (e.g. the p = 2 result of ``submat_invroot``,
    K ~ A^(-1/2)), on K^T A K y = K^T b with x = K y (Sec. 4.4).  Returns
    (x, iterations, relative residual of the iterated system)."""
    torch = _torch()
    va = plan._vals(vals_a)
    if b is None:
        b = torch.ones(plan.n, dtype=torch.float64, device=va.device)
    b = b.to(device=va.device, dtype=torch.float64).contiguous()
    if b.numel() != plan.n:
        raise ValueError(f"expected {plan.n} right-hand side values, got {b.numel()}")
    vk = plan._vals(vals_k) if vals_k is not None else None
    x = torch.empty_like(b)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    _check(plan._lib, plan._lib.submat_pcg(
        plan._h, ctypes.c_void_p(va.data_ptr()),
        ctypes.c_void_p(vk.data_ptr()) if vk is not None else None,
        ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), float(tol), int(max_iter),
        ctypes.byref(it), ctypes.byref(rel), _stream_ptr(stream)))
    return x, int(it.value), float(rel.value)


def submat_refine(plan: Plan, a_vals, x_in, p: int, iters: int, x_out=None, stream=None):
    """``submat_refine``: ``iters`` Newton steps for A^(-1/p) from the symmetric part of
    ``x_in``, every product restricted to the plan's pattern (Sec. 4.5).  ``a_vals`` and
    ``x_in`` are CUDA float64 tensors of the pattern's nnz values."""
    torch = _torch()
    av = plan._vals(a_vals)
    xv = plan._vals(x_in)
    if x_out is None:
        x_out = torch.empty_like(xv)
    _check(plan._lib, plan._lib.submat_refine(plan._h, ctypes.c_void_p(av.data_ptr()),
                                              ctypes.c_void_p(xv.data_ptr()), int(p), int(iters),
                                              ctypes.c_void_p(x_out.data_ptr()),
                                              _stream_ptr(stream)))
    return x_out


def shard_rows(rowptr, count: int, rank: int):
    """``submat_shard_rows``: the contiguous, cost-balanced row range (begin, end) of shard
    ``rank`` of ``count`` (host computation; works without a GPU)."""
    lib = load_library()
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    b, e = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib, lib.submat_shard_rows(int(rp.shape[0] - 1), rp.ctypes.data, int(count), int(rank),
                                      ctypes.byref(b), ctypes.byref(e)))
    return int(b.value), int(e.value)


def csr_arrays(mat):
    """(rowptr int32, colind int32, vals float64) of a scipy.sparse matrix (any format), in
    the form the plan expects: CSR order, column indices ascending and unique within a row
    (duplicates are summed).  Explicitly stored zeros stay: they are part of the pattern.
    Host-side conversion only."""
    import scipy.sparse as sp
    c = sp.csr_matrix(mat, dtype=np.float64, copy=True)
    c.sum_duplicates()                      # sorts the indices as well
    if c.shape[0] != c.shape[1]:
        raise ValueError(f"expected a square matrix, got {c.shape}")
    if c.nnz > np.iinfo(np.int32).max:
        raise ValueError("more than 2^31 - 1 stored entries")
    return (c.indptr.astype(np.int32), c.indices.astype(np.int32),
            np.ascontiguousarray(c.data, dtype=np.float64))


def scipy_csr(rowptr, colind, vals):
    """The result values (numpy array or tensor, on any device) on the plan's pattern as a
    scipy.sparse CSR matrix.  Host-side conversion only."""
    import scipy.sparse as sp
    if hasattr(vals, "detach"):             # a torch tensor
        vals = vals.detach().cpu().numpy()
    rp = np.asarray(rowptr, dtype=np.int64)
    n = rp.shape[0] - 1
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(colind), rp),
                         shape=(n, n))


SUBMAT_NOALLOC_MAX_M = 1024


def submat_invroot_noalloc(rowptr, colind, p: int, vals_in, vals_out=None, m_max: int = 0,
                           stream=None):
    """``submat_invroot_noalloc``: the FP64 forward without a plan and without any device
    allocation by the library (its working storage is a fixed device array inside
    libsubmat.so).  For callers that cannot allocate device memory; pass ``vals_out`` to
    keep this call free of allocations on the Python side too.  rowptr, colind, vals_in and
    vals_out are CUDA tensors; m_max bounds the row lengths (default: computed here, which
    reads rowptr back to the host).  Synchronous."""
    torch = _torch()
    lib = load_library()
    for t in (rowptr, colind, vals_in):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected CUDA tensors")
    if rowptr.dtype != torch.int32 or colind.dtype != torch.int32 or vals_in.dtype != torch.float64:
        raise TypeError("expected int32 rowptr/colind and float64 values")
    n = rowptr.numel() - 1
    if m_max <= 0:
        m_max = int((rowptr[1:] - rowptr[:-1]).max().item()) if n > 0 else 1
    if vals_out is None:
        vals_out = torch.empty_like(vals_in)
    _check(lib, lib.submat_invroot_noalloc(n, colind.numel(), ctypes.c_void_p(rowptr.data_ptr()),
                                           ctypes.c_void_p(colind.data_ptr()), int(p), int(m_max),
                                           ctypes.c_void_p(vals_in.data_ptr()),
                                           ctypes.c_void_p(vals_out.data_ptr()),
                                           _stream_ptr(stream)))
    return vals_out


def _make_function():
    torch = _torch()

    class SubmatInvRoot(torch.autograd.Function):
        """Autograd wrapper: forward = submat_invroot, backward = submat_invroot_backward.

        The plan keeps the input of its last forward, so nothing is saved on the tape; a
        backward through an earlier forward of the same plan (whose input is gone) raises
        instead of returning the gradient at the wrong point."""

        @staticmethod
        def forward(ctx, vals, plan):
            out = plan.invroot(vals)
            ctx.plan = plan
            ctx.fwd_gen = plan._fwd_gen
            return out

        @staticmethod
        def backward(ctx, grad):
            if ctx.plan._fwd_gen != ctx.fwd_gen:
                raise RuntimeError("the plan ran another forward after this one; its saved "
                                   "input is gone (use one plan per differentiated forward)")
            return ctx.plan.backward(grad.contiguous()), None

    return SubmatInvRoot


def __getattr__(name):
    if name == "SubmatInvRoot":
        f = _make_function()
        globals()["SubmatInvRoot"] = f
        return f
    raise AttributeError(name)
