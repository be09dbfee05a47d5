"""Python binding of the batched products (include/pjds_batch.h): argument
marshalling only; the plan buffer is a torch device tensor."""
from __future__ import annotations

import ctypes

import torch

from . import pjds as _p

_lib = _p.lib()
_i32, _vp, _sz = ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t
_P = ctypes.POINTER
for _name, _res, _args in (
        ("pjds_spmm", ctypes.c_int, [_P(_p._PjdsDevS), _i32, _vp, _vp, _vp]),
        ("pjds_batch_plan_bytes", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_sz)]),
        ("pjds_batch_create", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_vp), _P(_vp), _vp, _sz, _P(_vp), _vp]),
        ("pjds_batch_run", ctypes.c_int, [_vp, _i32, _vp]),
        ("pjds_batch_info", ctypes.c_int, [_vp, _P(_i32), _P(_i32)]),
        ("pjds_batch_destroy", ctypes.c_int, [_vp])):
    getattr(_lib, _name).restype = _res
    getattr(_lib, _name).argtypes = _args


def spmm(A, X: torch.Tensor, Y: torch.Tensor, stream=None) -> torch.Tensor:
    """Y = A X (pjds_spmm); X: (n_cols, k), Y: (n_rows, k), row-major, A's vector type."""
    if X.dim() != 2 or Y.dim() != 2 or X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y must be 2-D with the same number of columns")
    k = X.shape[1]
    _p._check_vec(X.reshape(-1), A.n_cols * k, A.vec_dtype, "X")
    _p._check_vec(Y.reshape(-1), A.n_rows * k, A.vec_dtype, "Y")
    if not (X.is_contiguous() and Y.is_contiguous()):
        raise ValueError("X and Y must be contiguous (row-major)")
    _p._check(_lib.pjds_spmm(ctypes.byref(A.struct), k, X.data_ptr(), Y.data_ptr(), _p._stream_ptr(stream)),
              "pjds_spmm")
    return Y


class Batch:
    """y_m = A_m x_m for many matrices in one persistent launch (pjds_batch_*)."""

    def __init__(self, mats, xs, ys, stream=None):
        n = len(mats)
        if not (n == len(xs) == len(ys)) or n == 0:
            raise ValueError("need equal, non-empty lists of matrices, x and y")
        for A, x, y in zip(mats, xs, ys):
            _p._check_vec(x, A.n_cols, A.vec_dtype, "x")
            _p._check_vec(y, A.n_rows, A.vec_dtype, "y")
        self._structs = (_p._PjdsDevS * n)(*[A.struct for A in mats])
        self._keep = (list(mats), list(xs), list(ys))
        need = _sz()
        _p._check(_lib.pjds_batch_plan_bytes(n, self._structs, ctypes.byref(need)), "pjds_batch_plan_bytes")
        self.plan = torch.empty(max(need.value, 1), dtype=torch.uint8, device=xs[0].device)
        xp = (_vp * n)(*[x.data_ptr() for x in xs])
        yp = (_vp * n)(*[y.data_ptr() for y in ys])
        h = _vp()
        _p._check(_lib.pjds_batch_create(n, self._structs, xp, yp, self.plan.data_ptr(), self.plan.numel(),
                                         ctypes.byref(h), _p._stream_ptr(stream)), "pjds_batch_create")
        self._h = h

    def run(self, use_graph: bool = True, stream=None):
        _p._check(_lib.pjds_batch_run(self._h, 1 if use_graph else 0, _p._stream_ptr(stream)), "pjds_batch_run")

    def info(self) -> dict:
        nt, nc = _i32(), _i32()
        _p._check(_lib.pjds_batch_info(self._h, ctypes.byref(nt), ctypes.byref(nc)), "pjds_batch_info")
        return {"n_tiles": nt.value, "n_ctas": nc.value}

    def destroy(self):
        if getattr(self, "_h", None):
            _lib.pjds_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
