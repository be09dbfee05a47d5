"""Python binding of the Krylov drivers (include/pjds_krylov.h): argument
marshalling only. Workspaces are torch device tensors owned by this module's
caller path (the library never allocates device memory).

    H64 = pjds_create(..., dtype="f64", permute_cols=True).to_device()   # fp64 residuals
    H32 = pjds_create(..., dtype="f32", permute_cols=True).to_device()   # inner products
    res = cg_solve(H64, H32, b_perm, x_perm)                             # x_perm updated in place
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import pjds as _p

_lib = _p.lib()
_i32, _i64, _vp, _f64, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_size_t
PJDS_CG_HISTORY = 64


class _CgOpts(ctypes.Structure):
    _fields_ = [("max_outer", _i32), ("inner_iters", _i32), ("tol", _f64), ("use_graph", _i32), ("reserved", _i32)]


class _CgResult(ctypes.Structure):
    _fields_ = [("outer", _i32), ("inner_total", _i32), ("rel_residual", _f64),
                ("history", _f64 * PJDS_CG_HISTORY), ("n_history", _i32), ("reserved", _i32)]


_P = ctypes.POINTER
for _name, _res, _args in (
        ("pjds_cg_workspace_bytes", ctypes.c_int, [_i32, _i32, _i32, _P(_sz)]),
        ("pjds_cg_solve", ctypes.c_int, [_P(_p._PjdsDevS), _P(_p._PjdsDevS), _vp, _vp, _P(_CgOpts), _P(_CgResult),
                                         _vp, _sz, _vp]),
        ("pjds_cg_solve_static", ctypes.c_int, [_P(_p._PjdsDevS), _P(_p._PjdsDevS), _vp, _vp, _P(_CgOpts),
                                                _P(_CgResult), _vp]),
        ("pjds_lanczos_workspace_bytes", ctypes.c_int, [_i32, _i32, _i32, _i32, _P(_sz)]),
        ("pjds_lanczos", ctypes.c_int, [_P(_p._PjdsDevS), _vp, _i32, _vp, _vp, _vp, _i32, _vp, _sz, _vp]),
        ("pjds_tridiag_extreme", ctypes.c_int, [_i32, _vp, _vp, _i32, _P(_f64), _vp]),
        ("pjds_ritz_workspace_bytes", ctypes.c_int, [_i32, _i32, _i32, _P(_sz)]),
        ("pjds_ritz_refine", ctypes.c_int, [_P(_p._PjdsDevS), _vp, _i32, _i32, _vp, _vp, _P(_f64), _P(_f64), _vp,
                                            _sz, _vp])):
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def cg_workspace_bytes(n_rows: int, n_pad: int, vec_dtype: int) -> int:
    out = _sz()
    _p._check(_lib.pjds_cg_workspace_bytes(n_rows, n_pad, vec_dtype, ctypes.byref(out)), "pjds_cg_workspace_bytes")
    return int(out.value)


def cg_solve(A_hi, A_lo, b: torch.Tensor, x: torch.Tensor, max_outer: int = 6, inner_iters: int = 50,
             tol: float = 0.0, use_graph: bool = True, stream=None, work: torch.Tensor | None = None) -> dict:
    """Mixed-precision CG with fp64 refinement (pjds_cg_solve). b, x: fp64
    device vectors in the permuted basis; x is updated in place."""
    for t, nm in ((b, "b"), (x, "x")):
        _p._check_vec(t, A_hi.n_rows, torch.float64, nm)
    low = A_lo is not None and A_lo.dtype != 0
    need = cg_workspace_bytes(A_hi.n_rows, A_hi.n_pad, 1 if low else 0)
    if work is None or work.numel() < need:
        work = _workspace(need, x.device)
    o = _CgOpts(max_outer, inner_iters, tol, 1 if use_graph else 0, 0)
    r = _CgResult()
    _p._check(_lib.pjds_cg_solve(ctypes.byref(A_hi.struct), ctypes.byref(A_lo.struct) if A_lo is not None else None,
                                 b.data_ptr(), x.data_ptr(), ctypes.byref(o), ctypes.byref(r), work.data_ptr(),
                                 work.numel(), _p._stream_ptr(stream)), "pjds_cg_solve")
    return {"outer": r.outer, "inner_total": r.inner_total, "rel_residual": r.rel_residual,
            "history": list(r.history[:r.n_history])}


def cg_solve_static(A_hi, A_lo, b: torch.Tensor, x: torch.Tensor, max_outer: int = 6, inner_iters: int = 50,
                    tol: float = 0.0, stream=None) -> dict:
    """pjds_cg_solve_static: the same solve as cg_solve, for callers that
    cannot allocate device memory; the library's static device workspace
    (at most 131072 rows) is used instead of a caller workspace, and the
    inner steps are launched one by one (no CUDA graph is created)."""
    for t, nm in ((b, "b"), (x, "x")):
        _p._check_vec(t, A_hi.n_rows, torch.float64, nm)
    o = _CgOpts(max_outer, inner_iters, tol, 0, 0)
    r = _CgResult()
    _p._check(_lib.pjds_cg_solve_static(ctypes.byref(A_hi.struct),
                                        ctypes.byref(A_lo.struct) if A_lo is not None else None, b.data_ptr(),
                                        x.data_ptr(), ctypes.byref(o), ctypes.byref(r), _p._stream_ptr(stream)),
              "pjds_cg_solve_static")
    return {"outer": r.outer, "inner_total": r.inner_total, "rel_residual": r.rel_residual,
            "history": list(r.history[:r.n_history])}


def lanczos(A, v0: torch.Tensor, steps: int, keep_basis: bool = False, use_graph: bool = True, stream=None):
    """`steps` Lanczos steps (pjds_lanczos). Returns (alpha[steps],
    beta[steps+1], basis tensor (steps x n) or None)."""
    _p._check_vec(v0, A.n_rows, A.vec_dtype, "v0")
    vec = 0 if A.dtype == 0 else 1
    need = _sz()
    _p._check(_lib.pjds_lanczos_workspace_bytes(A.n_rows, A.n_pad, vec, steps, ctypes.byref(need)),
              "pjds_lanczos_workspace_bytes")
    work = _workspace(need.value, v0.device)
    basis = torch.empty((steps, A.n_rows), dtype=A.vec_dtype, device=v0.device) if keep_basis else None
    alpha = np.zeros(steps)
    beta = np.zeros(steps + 1)
    _p._check(_lib.pjds_lanczos(ctypes.byref(A.struct), v0.data_ptr(), steps, alpha.ctypes.data, beta.ctypes.data,
                                basis.data_ptr() if basis is not None else None, 1 if use_graph else 0,
                                work.data_ptr(), work.numel(), _p._stream_ptr(stream)), "pjds_lanczos")
    return alpha, beta, basis


def tridiag_extreme(alpha, beta, which: str = "largest"):
    """(theta, s): extreme eigenpair of the Lanczos tridiagonal (host)."""
    a = np.ascontiguousarray(alpha, np.float64)
    bta = np.ascontiguousarray(beta, np.float64)
    k = len(a)
    if len(bta) < k:
        raise ValueError("beta needs at least len(alpha) entries (beta[0] unused)")
    th = _f64()
    s = np.zeros(k)
    _p._check(_lib.pjds_tridiag_extreme(k, a.ctypes.data, bta.ctypes.data, 0 if which == "largest" else 1,
                                        ctypes.byref(th), s.ctypes.data), "pjds_tridiag_extreme")
    return float(th.value), s


def ritz_refine(A_hi, basis: torch.Tensor, s, stream=None):
    """(y, theta, rel_residual): y = basis^T s, fp64 Rayleigh quotient and
    residual with A_hi (pjds_ritz_refine)."""
    k = basis.shape[0]
    s = np.ascontiguousarray(s, np.float64)
    need = _sz()
    _p._check(_lib.pjds_ritz_workspace_bytes(A_hi.n_rows, A_hi.n_pad, k, ctypes.byref(need)),
              "pjds_ritz_workspace_bytes")
    work = _workspace(need.value, basis.device)
    y = torch.empty(A_hi.n_rows, dtype=torch.float64, device=basis.device)
    th, rr = _f64(), _f64()
    bdt = 0 if basis.dtype == torch.float64 else 1
    _p._check(_lib.pjds_ritz_refine(ctypes.byref(A_hi.struct), basis.data_ptr(), bdt, k, s.ctypes.data,
                                    y.data_ptr(), ctypes.byref(th), ctypes.byref(rr), work.data_ptr(), work.numel(),
                                    _p._stream_ptr(stream)), "pjds_ritz_refine")
    return y, float(th.value), float(rr.value)
