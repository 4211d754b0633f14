"""GB300-native reachability-probability solver: Python binding of include/reach.h.

Argument marshalling only.  Every step of the method (validation, graph search,
extraction, the Jacobi / BiCGStab iterations, gradients) runs in the CUDA library
``libreach.so``; nothing here computes.  Arrays may be numpy arrays (host memory)
or CUDA torch tensors (device memory); the matching REACH_HOST / REACH_DEVICE flag
is passed to the library.  If the library cannot be built or loaded, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import _build

__all__ = [
    "ReachError", "ReachInfo", "lib", "header_symbols",
    "REACH_OK", "REACH_EINVAL", "REACH_ENOMEM", "REACH_ECUDA", "REACH_ESTATE", "REACH_ENOTCONV",
    "REACH_EBREAKDOWN", "REACH_ETIMEOUT", "REACH_HOST", "REACH_DEVICE", "REACH_PROB01",
    "REACH_PROB0_ONLY", "REACH_JACOBI_FP64", "REACH_JACOBI_MIXED", "REACH_BICGSTAB_FP64",
    "REACH_JACOBI_SEG", "REACH_SCC_JACOBI", "reach_scc",
    "reach_create", "reach_precompute", "reach_get_classes", "reach_solve", "reach_grad",
    "reach_grad_method",
    "reach_param_probs", "reach_param_grad_theta", "reach_last_error", "reach_destroy",
    "reach_version", "Solver", "reach_batch_create", "reach_batch_precompute",
    "reach_batch_get_classes", "reach_batch_solve", "reach_batch_destroy", "BatchSolver",
    "reach_batch_set_chains", "reach_batch_chain_info", "reach_norm_bound", "reach_batch_autotune",
]

REACH_OK, REACH_EINVAL, REACH_ENOMEM, REACH_ECUDA, REACH_ESTATE = 0, 1, 2, 3, 4
REACH_ENOTCONV, REACH_EBREAKDOWN, REACH_ETIMEOUT = 5, 6, 7
REACH_HOST, REACH_DEVICE = 0, 1
REACH_PROB01, REACH_PROB0_ONLY = 0, 1
REACH_JACOBI_FP64, REACH_JACOBI_MIXED, REACH_BICGSTAB_FP64, REACH_JACOBI_SEG = 0, 1, 2, 3
REACH_SCC_JACOBI = 4
REACH_BLOCK_P, REACH_BLOCK_S, REACH_BLOCK_XR, REACH_BLOCK_XP = 0, 1, 2, 3

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENOTCONV",
                6: "EBREAKDOWN", 7: "ETIMEOUT"}
METHODS = {"jacobi": REACH_JACOBI_FP64, "jacobi_fp64": REACH_JACOBI_FP64,
           "mixed": REACH_JACOBI_MIXED, "jacobi_mixed": REACH_JACOBI_MIXED,
           "bicgstab": REACH_BICGSTAB_FP64, "bicgstab_fp64": REACH_BICGSTAB_FP64,
           "jacobi_seg": REACH_JACOBI_SEG, "scc_jacobi": REACH_SCC_JACOBI}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "reach.h")


class ReachError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ReachInfo(C.Structure):
    _fields_ = [("iters", C.c_int64), ("n_q", C.c_int64), ("m_q", C.c_int64),
                ("last_delta", C.c_double), ("resid_inf", C.c_double),
                ("ms_precompute", C.c_double), ("ms_solve", C.c_double),
                ("bytes_moved", C.c_double), ("status", C.c_int32), ("refinements", C.c_int32),
                ("err_bound", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ReachSccInfo(C.Structure):
    _fields_ = [("n_q", C.c_int64), ("n_scc", C.c_int64), ("n_levels", C.c_int64),
                ("n_trivial", C.c_int64), ("largest", C.c_int64), ("exact", C.c_int32),
                ("rounds", C.c_int32), ("ms", C.c_double), ("passes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_P = C.c_void_p
_I64, _I32, _D = C.c_int64, C.c_int32, C.c_double

_SIGS = {
    "reach_create": (_I32, [C.POINTER(_P), _I64, _I64, _P, _P, _P, _P, _I32, _P]),
    "reach_precompute": (_I32, [_P, _I32]),
    "reach_get_classes": (_I32, [_P, _P, _I32]),
    "reach_solve": (_I32, [_P, _I32, _D, _I64, _I32, _P, _P, _I32, C.POINTER(ReachInfo)]),
    "reach_grad": (_I32, [_P, _I64, _D, _I64, _P, _I32, C.POINTER(ReachInfo)]),
    "reach_grad_method": (_I32, [_P, _I32, _I64, _D, _I64, _P, _I32, C.POINTER(ReachInfo)]),
    "reach_param_probs": (_I32, [_I64, _I64, _P, _P, _P, _P, _I32, _P, _P]),
    "reach_param_grad_theta": (_I32, [_I64, _I64, _P, _P, _P, _P, _I32, _P, _P]),
    "reach_last_error": (C.c_char_p, [_P]),
    "reach_destroy": (None, [_P]),
    "reach_version": (C.c_char_p, []),
    "reach_batch_create": (_I32, [C.POINTER(_P), _I64, _I64, _P, _P, _P, _I32, _P, _I32, _P]),
    "reach_batch_precompute": (_I32, [_P, _I32]),
    "reach_batch_get_classes": (_I32, [_P, _P, _I32]),
    "reach_batch_solve": (_I32, [_P, _D, _I64, _I32, _P, _I32, C.POINTER(ReachInfo)]),
    "reach_batch_destroy": (None, [_P]),
    "reach_batch_set_chains": (_I32, [_P, _I32, _P]),
    "reach_batch_chain_info": (_I32, [_P, _P, _P]),
    "reach_batch_autotune": (_I32, [_P, C.POINTER(_I32), C.POINTER(_D), C.POINTER(_I32)]),
    "reach_autotune": (_I32, [_P, _I32, C.POINTER(_I32), C.POINTER(_D), C.POINTER(_I32)]),
    "reach_system_create": (_I32, [C.POINTER(_P), _I64, _I64, _P, _P, _P, _P, _I32, _P]),
    "reach_time_kernel": (_I32, [_P, _I32, _I32, C.POINTER(_D)]),
    "reach_scc": (_I32, [_P, _P, _P, _I32, _I32, C.POINTER(ReachSccInfo)]),
    "reach_norm_bound": (_I32, [_P, _I32, _D, _I64, C.POINTER(_D), C.POINTER(ReachInfo)]),
    "reach_get_system": (_I32, [_P, C.POINTER(_I64), C.POINTER(_I64), _P, _P, _P, _P, _P, _P, _I32]),
    "reach_block_create": (_I32, [C.POINTER(_P), _I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _I32, _P]),
    "reach_block_halo": (_I32, [_P, _P, _P]),
    "reach_block_jacobi": (_I32, [_P, _P, _P, _P]),
    "reach_block_matvec": (_I32, [_P, _P, _P, _P, _P]),
    "reach_block_dot": (_I32, [_P, _P, _P, _P, _P]),
    "reach_block_bicgstab_update": (_I32, [_P, _I32, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P]),
    "reach_block_last_error": (C.c_char_p, [_P]),
    "reach_block_destroy": (None, [_P]),
    "reach_jacobi_solve_noalloc": (_I32, [_I64, _P, _P, _P, _P, _P, _D, _I64, _I32, _P,
                                          C.POINTER(_I64), C.POINTER(_D), _P]),
}


def lib():
    """Load libreach.so, building it first when sources are newer; raise if impossible."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        so = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(so, name)
            f.restype = res
            f.argtypes = args
        _LIB = so
    return _LIB


def header_symbols(path=HEADER):
    """Names of every function the public header declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(reach_[a-z_0-9]+)\s*\(", text)))


# ------------------------------------------------------------------ marshalling

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for host-only use
        pass
    return None


def _arg(a, dtype, n=None, name="array"):
    """(pointer, flag, keep-alive) of a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        want = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64,
                np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"{name}: need a contiguous {want} tensor")
        if n is not None and a.numel() != n:
            raise ValueError(f"{name}: need {n} elements, got {a.numel()}")
        return a.data_ptr(), (REACH_DEVICE if a.is_cuda else REACH_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if n is not None and arr.size != n:
        raise ValueError(f"{name}: need {n} elements, got {arr.size}")
    return arr.ctypes.data, REACH_HOST, arr


def _check(st, ctx=None, what=""):
    if st != REACH_OK:
        raise ReachError(st, reach_last_error(ctx) or what)


def reach_version():
    return lib().reach_version().decode()


def reach_last_error(ctx=None):
    msg = lib().reach_last_error(ctx)
    return msg.decode() if msg else ""


def reach_create(n, rowptr, col, val, goal, stream=None):
    """Context for chain (n, rowptr, col, val) with goal mask ``goal`` (§2, §4)."""
    rowptr_p, f0, k0 = _arg(rowptr, np.int64, n + 1, "rowptr")
    m = int(rowptr[-1])
    col_p, f1, k1 = _arg(col, np.int32, m, "col")
    val_p, f2, k2 = _arg(val, np.float64, m, "val")
    goal_p, f3, k3 = _arg(goal, np.uint8, n, "goal")
    if len({f0, f1, f2, f3}) != 1:
        raise ValueError("all inputs must live in the same memory (host or device)")
    if stream is None:
        stream = _torch_stream()
    ctx = _P()
    st = lib().reach_create(C.byref(ctx), int(n), m, rowptr_p, col_p, val_p, goal_p, f0, stream)
    _check(st, None, "reach_create")
    return ctx


def reach_system_create(n, rowptr, col, val, b, stream=None):
    """Context for a general system M x = b (M in CSR, any signs, non-zero diagonal)."""
    rowptr_p, f0, k0 = _arg(rowptr, np.int64, n + 1, "rowptr")
    m = int(rowptr[-1])
    col_p, f1, k1 = _arg(col, np.int32, m, "col")
    val_p, f2, k2 = _arg(val, np.float64, m, "val")
    b_p, f3, k3 = _arg(b, np.float64, n, "b")
    if len({f0, f1, f2, f3}) != 1:
        raise ValueError("all inputs must live in the same memory (host or device)")
    if stream is None:
        stream = _torch_stream()
    ctx = _P()
    st = lib().reach_system_create(C.byref(ctx), int(n), m, rowptr_p, col_p, val_p, b_p, f0, stream)
    _check(st, None, "reach_system_create")
    return ctx


def reach_precompute(ctx, mode=REACH_PROB01):
    _check(lib().reach_precompute(ctx, int(mode)), ctx)


def reach_get_classes(ctx, n, out=None):
    if out is None:
        out = np.empty(n, np.uint8)
    p, f, keep = _arg(out, np.uint8, n, "cls")
    _check(lib().reach_get_classes(ctx, p, f), ctx)
    return out


def reach_solve(ctx, n, method=REACH_JACOBI_FP64, eps=1e-10, max_iter=1_000_000, refine_k=0,
                x0=None, out=None, check=True):
    """Solve on S? and return (x over all states, info dict)."""
    method = METHODS.get(method, method) if isinstance(method, str) else int(method)
    if out is None:
        out = np.empty(n, np.float64)
    op, f, keep = _arg(out, np.float64, n, "x_out")
    x0p, f0, keep0 = _arg(x0, np.float64, n, "x0")
    if x0 is not None and f0 != f:
        raise ValueError("x0 and x_out must live in the same memory")
    info = ReachInfo()
    st = lib().reach_solve(ctx, method, float(eps), int(max_iter), int(refine_k), x0p, op, f,
                           C.byref(info))
    if check and st not in (REACH_OK,):
        raise ReachError(st, reach_last_error(ctx))
    return out, info.as_dict()


def reach_grad(ctx, m, init, eps=1e-13, max_iter=1_000_000, out=None, check=True, method="jacobi"):
    """d x_init / d P for every stored entry (input order) and the adjoint info; the adjoint
    system is solved by `method` ("jacobi" or "bicgstab")."""
    if out is None:
        out = np.empty(m, np.float64)
    op, f, keep = _arg(out, np.float64, m, "grad")
    info = ReachInfo()
    meth = METHODS.get(method, method) if isinstance(method, str) else int(method)
    st = lib().reach_grad_method(ctx, meth, int(init), float(eps), int(max_iter), op, f, C.byref(info))
    if check and st != REACH_OK:
        raise ReachError(st, reach_last_error(ctx))
    return out, info.as_dict()


def reach_norm_bound(ctx, method=REACH_BICGSTAB_FP64, eps=1e-8, max_iter=1_000_000):
    """Certified bound of ||(I - A)^-1||_inf from a solve of (I - A) tau = 1; later solves
    of the context use it for their err_bound.  Returns (bound in use, info of the tau solve)."""
    method = METHODS.get(method, method) if isinstance(method, str) else int(method)
    k = C.c_double(0.0)
    info = ReachInfo()
    _check(lib().reach_norm_bound(ctx, method, float(eps), int(max_iter), C.byref(k), C.byref(info)), ctx)
    return k.value, info.as_dict()


def reach_param_probs(rowptr, cls, offset, theta, out, stream=None):
    """P_e = row softmax of theta[cls_e] + offset_e (CUDA tensors)."""
    n = rowptr.numel() - 1
    m = cls.numel()
    args = [_arg(rowptr, np.int64, n + 1, "rowptr"), _arg(cls, np.int32, m, "cls"),
            _arg(offset, np.float64, m, "offset"), _arg(theta, np.float64, None, "theta"),
            _arg(out, np.float64, m, "p_out")]
    if any(a[1] != REACH_DEVICE for a in args):
        raise ValueError("reach_param_probs takes CUDA tensors")
    st = lib().reach_param_probs(n, m, args[0][0], args[1][0], args[2][0], args[3][0],
                                 int(theta.numel()), args[4][0],
                                 _torch_stream() if stream is None else stream)
    _check(st, None)
    return out


def reach_param_grad_theta(rowptr, cls, p, g_p, n_classes, out, stream=None):
    n = rowptr.numel() - 1
    m = cls.numel()
    args = [_arg(rowptr, np.int64, n + 1, "rowptr"), _arg(cls, np.int32, m, "cls"),
            _arg(p, np.float64, m, "p"), _arg(g_p, np.float64, m, "g_p"),
            _arg(out, np.float64, n_classes, "g_theta")]
    if any(a[1] != REACH_DEVICE for a in args):
        raise ValueError("reach_param_grad_theta takes CUDA tensors")
    st = lib().reach_param_grad_theta(n, m, args[0][0], args[1][0], args[2][0], args[3][0],
                                      int(n_classes), args[4][0],
                                      _torch_stream() if stream is None else stream)
    _check(st, None)
    return out


def reach_autotune(ctx, method=REACH_JACOBI_FP64):
    """Time the row mappings of ``method`` on this context's system; returns the choice."""
    method = METHODS.get(method, method) if isinstance(method, str) else int(method)
    lanes, ms, k = C.c_int32(0), C.c_double(0.0), C.c_int32(0)
    _check(lib().reach_autotune(ctx, method, C.byref(lanes), C.byref(ms), C.byref(k)), ctx)
    return {"lanes": lanes.value, "sweep_ms": ms.value, "check_every": k.value}


def reach_scc(ctx, labels=True, max_rounds=0, out_label=None, out_level=None):
    """Strongly connected components of the digraph of A over S? and their levels (§8).

    Returns (label, level, info): label[i] is the largest row index of row i's component
    and level[i] the component's level in the condensation (int32 over the S? rows in
    ascending state order); both None when ``labels`` is false.
    """
    info = ReachSccInfo()
    _check(lib().reach_scc(ctx, None, None, REACH_HOST, int(max_rounds), C.byref(info)), ctx)
    if not labels:
        return None, None, info.as_dict()
    nq = info.n_q
    if out_label is None:
        out_label = np.empty(nq, np.int32)
    if out_level is None:
        out_level = np.empty(nq, np.int32)
    lp, f1, k1 = _arg(out_label, np.int32, nq, "label")
    vp, f2, k2 = _arg(out_level, np.int32, nq, "level")
    if f1 != f2:
        raise ValueError("label and level must be in the same kind of memory")
    _check(lib().reach_scc(ctx, lp, vp, f1, int(max_rounds), C.byref(info)), ctx)
    return out_label, out_level, info.as_dict()


KERNELS = {"jacobi64": 0, "sweep32": 1, "resid_mixed": 2, "bicgstab_spmv": 3}


def reach_time_kernel(ctx, kernel, launches=20):
    """Average ms per launch of one solver kernel (CUDA events on the context stream)."""
    k = KERNELS.get(kernel, kernel) if isinstance(kernel, str) else int(kernel)
    ms = C.c_double(0.0)
    _check(lib().reach_time_kernel(ctx, k, int(launches), C.byref(ms)), ctx)
    return ms.value


def reach_destroy(ctx):
    if ctx:
        lib().reach_destroy(ctx)


class Solver:
    """Owns one context: ``with Solver(n, rowptr, col, val, goal) as s: x, info = s.solve()``.

    ``Solver.system(n, rowptr, col, val, b)`` builds one for a general system M x = b.
    """

    def __init__(self, n, rowptr, col, val, goal, mode=REACH_PROB01, stream=None, precompute=True,
                 _ctx=None):
        self.n = int(n)
        self.m = int(rowptr[-1])
        self.ctx = _ctx if _ctx is not None else reach_create(n, rowptr, col, val, goal, stream)
        if precompute and _ctx is None:
            self.precompute(mode)

    @classmethod
    def system(cls, n, rowptr, col, val, b, stream=None):
        return cls(n, rowptr, col, val, None, _ctx=reach_system_create(n, rowptr, col, val, b, stream))

    def precompute(self, mode=REACH_PROB01):
        reach_precompute(self.ctx, mode)

    def classes(self, out=None):
        return reach_get_classes(self.ctx, self.n, out)

    def solve(self, method="jacobi", eps=1e-10, max_iter=1_000_000, refine_k=0, x0=None, out=None,
              check=True):
        return reach_solve(self.ctx, self.n, method, eps, max_iter, refine_k, x0, out, check)

    def grad(self, init, eps=1e-13, max_iter=1_000_000, out=None, check=True, method="jacobi"):
        return reach_grad(self.ctx, self.m, init, eps, max_iter, out, check, method)

    def autotune(self, method="jacobi"):
        return reach_autotune(self.ctx, method)

    def norm_bound(self, method="bicgstab", eps=1e-8, max_iter=1_000_000):
        return reach_norm_bound(self.ctx, method, eps, max_iter)

    def scc(self, labels=True, max_rounds=0):
        return reach_scc(self.ctx, labels, max_rounds)

    def close(self):
        if self.ctx:
            reach_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched multi-RHS

def reach_batch_create(n, rowptr, col, val, goals, stream=None):
    """Batch over one chain with goal sets goals[k, n] (k <= 8)."""
    k = int(goals.shape[0]) if hasattr(goals, "shape") and len(goals.shape) == 2 else None
    if k is None:
        raise ValueError("goals must be a [k, n] array")
    rowptr_p, f0, k0 = _arg(rowptr, np.int64, n + 1, "rowptr")
    m = int(rowptr[-1])
    col_p, f1, k1 = _arg(col, np.int32, m, "col")
    val_p, f2, k2 = _arg(val, np.float64, m, "val")
    goal_p, f3, k3 = _arg(goals, np.uint8, k * n, "goals")
    if len({f0, f1, f2, f3}) != 1:
        raise ValueError("all inputs must live in the same memory (host or device)")
    if stream is None:
        stream = _torch_stream()
    b = _P()
    st = lib().reach_batch_create(C.byref(b), int(n), m, rowptr_p, col_p, val_p, k, goal_p, f0, stream)
    _check(st, None, "reach_batch_create")
    return b


def reach_batch_precompute(b, mode=REACH_PROB01):
    _check(lib().reach_batch_precompute(b, int(mode)), None, "reach_batch_precompute")


def reach_batch_get_classes(b, n, k, out=None):
    if out is None:
        out = np.empty((k, n), np.uint8)
    p, f, keep = _arg(out, np.uint8, k * n, "cls")
    _check(lib().reach_batch_get_classes(b, p, f), None, "reach_batch_get_classes")
    return out


def reach_batch_solve(b, n, k, eps=1e-8, max_iter=1_000_000, refine_k=0, out=None, check=True):
    if out is None:
        out = np.empty((k, n), np.float64)
    p, f, keep = _arg(out, np.float64, k * n, "x_out")
    info = ReachInfo()
    st = lib().reach_batch_solve(b, float(eps), int(max_iter), int(refine_k), p, f, C.byref(info))
    if check and st != REACH_OK:
        raise ReachError(st, reach_last_error(None) or "reach_batch_solve")
    return out, info.as_dict()


def reach_batch_set_chains(b, offsets):
    """Chains of a block-diagonal batch: chain c owns states [offsets[c], offsets[c+1])."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.ndim != 1 or off.size < 2:
        raise ValueError("offsets must be a 1-D array of n_chains + 1 entries")
    _check(lib().reach_batch_set_chains(b, int(off.size - 1), off.ctypes.data), None, "reach_batch_set_chains")


def reach_batch_chain_info(b, n_chains):
    """(iters[n_chains], last[n_chains]) of the last reach_batch_solve, per chain."""
    iters = np.empty(n_chains, np.int64)
    last = np.empty(n_chains, np.float64)
    _check(lib().reach_batch_chain_info(b, iters.ctypes.data, last.ctypes.data), None, "reach_batch_chain_info")
    return iters, last


def reach_batch_autotune(b):
    """Pick the batched sweep variant and refinement period by timing them on this batch."""
    v, ms, k = C.c_int32(0), C.c_double(0.0), C.c_int32(0)
    _check(lib().reach_batch_autotune(b, C.byref(v), C.byref(ms), C.byref(k)), None, "reach_batch_autotune")
    return {"variant": v.value, "sweep_ms": ms.value, "refine_k": k.value}


def reach_batch_destroy(b):
    if b:
        lib().reach_batch_destroy(b)


class BatchSolver:
    """K goal sets over one chain: ``BatchSolver(n, rowptr, col, val, goals[k, n])``."""

    def __init__(self, n, rowptr, col, val, goals, mode=REACH_PROB01, stream=None, chains=None):
        self.n = int(n)
        self.k = int(goals.shape[0])
        self.n_chains = 1
        self.b = reach_batch_create(n, rowptr, col, val, goals, stream)
        if chains is not None:
            self.set_chains(chains)
        reach_batch_precompute(self.b, mode)

    def set_chains(self, offsets):
        """Stop each chain of the block-diagonal union on its own (offsets: n_chains + 1)."""
        reach_batch_set_chains(self.b, offsets)
        self.n_chains = len(offsets) - 1

    def chain_info(self):
        return reach_batch_chain_info(self.b, self.n_chains)

    def autotune(self):
        return reach_batch_autotune(self.b)

    def classes(self, out=None):
        return reach_batch_get_classes(self.b, self.n, self.k, out)

    def solve(self, eps=1e-8, max_iter=1_000_000, refine_k=0, out=None, check=True):
        return reach_batch_solve(self.b, self.n, self.k, eps, max_iter, refine_k, out, check)

    def close(self):
        if self.b:
            reach_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
