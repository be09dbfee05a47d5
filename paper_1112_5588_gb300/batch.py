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
        ("pjds_spmm_pattern", ctypes.c_int, [_P(_p._PjdsDevS), _i32, _vp, _vp, _vp]),
        ("pjds_batch_plan_bytes", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_sz)]),
        ("pjds_batch_create", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_vp), _P(_vp), _vp, _sz, _P(_vp), _vp]),
        ("pjds_batch_create_lanes", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_vp), _P(_vp), _P(_i32), _vp, _sz,
                                                   _P(_vp), _vp]),
        ("pjds_batch_create_rule", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_vp), _P(_vp), _P(_i32), _vp, _sz,
                                                  _P(_vp), _vp]),
        ("pjds_batch_tune_rule", ctypes.c_int, [_i32, _P(_p._PjdsDevS), _P(_vp), _P(_vp), _P(_i32), _i32, _i32, _vp,
                                                _sz, _vp, _sz, _P(ctypes.c_double), _P(_i32), _vp]),
        ("pjds_batch_run", ctypes.c_int, [_vp, _i32, _vp]),
        ("pjds_batch_run_pattern", ctypes.c_int, [_vp, _vp]),
        ("pjds_batch_info", ctypes.c_int, [_vp, _P(_i32), _P(_i32)]),
        ("pjds_batch_destroy", ctypes.c_int, [_vp])):
    getattr(_lib, _name).restype = _res
    getattr(_lib, _name).argtypes = _args


def _spmm_call(fn, name, A, X, Y, stream):
    if X.dim() != 2 or Y.dim() != 2 or X.shape[1] != Y.shape[1]:
        raise ValueError("X and Y must be 2-D with the same number of columns")
    k = X.shape[1]
    _p._check_vec(X.reshape(-1), A.n_cols * k, A.vec_dtype, "X")
    _p._check_vec(Y.reshape(-1), A.n_rows * k, A.vec_dtype, "Y")
    if not (X.is_contiguous() and Y.is_contiguous()):
        raise ValueError("X and Y must be contiguous (row-major)")
    _p._check(fn(ctypes.byref(A.struct), k, X.data_ptr(), Y.data_ptr(), _p._stream_ptr(stream)), name)
    return Y


def spmm(A, X: torch.Tensor, Y: torch.Tensor, stream=None) -> torch.Tensor:
    """Y = A X (pjds_spmm); X: (n_cols, k), Y: (n_rows, k), row-major, A's vector type."""
    return _spmm_call(_lib.pjds_spmm, "pjds_spmm", A, X, Y, stream)


def spmm_pattern(A, X: torch.Tensor, Y: torch.Tensor, stream=None) -> torch.Tensor:
    """Y = S X, S the sparsity pattern of A (pjds_spmm_pattern): the launch of
    spmm without the value stream, its gather ceiling."""
    return _spmm_call(_lib.pjds_spmm_pattern, "pjds_spmm_pattern", A, X, Y, stream)


class Batch:
    """y_m = A_m x_m for many matrices in one persistent launch (pjds_batch_*)."""

    def __init__(self, mats, xs, ys, lanes=None, rule=None, stream=None):
        """lanes: None (the block-length rule) or one of 0, 1, 2, 4, 8 per
        matrix (0 = the rule). rule: None (the built-in rule) or (L2, L4, L8),
        the block lengths from which tiles get 2, 4 and 8 lanes per row (e.g.
        from tune_rule)."""
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
        if rule is not None:
            if lanes is not None:
                raise ValueError("give lanes or rule, not both")
            mr = (_i32 * 3)(*[int(v) for v in rule])
            _p._check(_lib.pjds_batch_create_rule(n, self._structs, xp, yp, mr, self.plan.data_ptr(),
                                                  self.plan.numel(), ctypes.byref(h), _p._stream_ptr(stream)),
                      "pjds_batch_create_rule")
        elif lanes is None:
            _p._check(_lib.pjds_batch_create(n, self._structs, xp, yp, self.plan.data_ptr(), self.plan.numel(),
                                             ctypes.byref(h), _p._stream_ptr(stream)), "pjds_batch_create")
        else:
            if len(lanes) != n:
                raise ValueError("lanes needs one entry per matrix")
            ln = (_i32 * n)(*[int(v) for v in lanes])
            _p._check(_lib.pjds_batch_create_lanes(n, self._structs, xp, yp, ln, self.plan.data_ptr(),
                                                   self.plan.numel(), ctypes.byref(h), _p._stream_ptr(stream)),
                      "pjds_batch_create_lanes")
        self._h = h

    def run(self, use_graph: bool = True, stream=None):
        _p._check(_lib.pjds_batch_run(self._h, 1 if use_graph else 0, _p._stream_ptr(stream)), "pjds_batch_run")

    def run_pattern(self, stream=None):
        """The pattern products of the batch (pjds_batch_run_pattern): the
        same launch without the value streams, its gather ceiling."""
        _p._check(_lib.pjds_batch_run_pattern(self._h, _p._stream_ptr(stream)), "pjds_batch_run_pattern")

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


NEVER = 2**31 - 1
# candidate block-length rules (L2, L4, L8) of tune_rule; the first is the built-in one
DEFAULT_RULES = [(16, 64, 256), (NEVER, NEVER, 64), (NEVER, NEVER, 32), (NEVER, NEVER, 128), (NEVER, NEVER, 16),
                 (NEVER, 32, 128), (NEVER, 16, 64), (NEVER, 64, 256), (8, 32, 128), (4, 16, 64), (32, 128, 512)]


def tune_rule(mats, xs, ys, rules=None, reps: int = 5, flush_bytes: int = 256 << 20, stream=None):
    """Time the batch under each block-length rule (pjds_batch_tune_rule);
    returns (best rule, [(rule, median us), ...]). Overwrites ys."""
    rules = list(rules) if rules is not None else DEFAULT_RULES
    n = len(mats)
    for A, x, y in zip(mats, xs, ys):
        _p._check_vec(x, A.n_cols, A.vec_dtype, "x")
        _p._check_vec(y, A.n_rows, A.vec_dtype, "y")
    structs = (_p._PjdsDevS * n)(*[A.struct for A in mats])
    need = _sz()
    _p._check(_lib.pjds_batch_plan_bytes(n, structs, ctypes.byref(need)), "pjds_batch_plan_bytes")
    plan = torch.empty(max(need.value, 1), dtype=torch.uint8, device=xs[0].device)
    flush = torch.empty(max(flush_bytes, 1), dtype=torch.uint8, device=xs[0].device) if flush_bytes else None
    xp = (_vp * n)(*[x.data_ptr() for x in xs])
    yp = (_vp * n)(*[y.data_ptr() for y in ys])
    rr = (_i32 * (3 * len(rules)))(*[int(v) for r in rules for v in r])
    us = (ctypes.c_double * len(rules))()
    best = _i32()
    _p._check(_lib.pjds_batch_tune_rule(n, structs, xp, yp, rr, len(rules), reps, plan.data_ptr(), plan.numel(),
                                        flush.data_ptr() if flush is not None else None,
                                        flush_bytes if flush is not None else 0, us, ctypes.byref(best),
                                        _p._stream_ptr(stream)), "pjds_batch_tune_rule")
    return tuple(rules[best.value]), [(tuple(r), float(u)) for r, u in zip(rules, us)]
