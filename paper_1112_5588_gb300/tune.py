"""Python binding of the exhaustive autotuner (include/pjds_tune.h):
argument marshalling only; the arena and the L2-flush buffer are torch device
tensors, the sweep itself runs in libpjds."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import pjds as _p

_lib = _p.lib()
_i32, _i64, _vp, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
DTYPE_NAMES = {0: "f64", 1: "f32", 2: "bf16"}


class _Cand(ctypes.Structure):
    _fields_ = [("b", _i32), ("dtype", _i32), ("rows_per_thread", _i32), ("threads_per_row", _i32),
                ("block_threads", _i32), ("unroll", _i32), ("staged", _i32), ("plan", _i32), ("tile_order", _i32),
                ("reserved", _i32)]


class _Entry(ctypes.Structure):
    _fields_ = [("cand", _Cand), ("us", ctypes.c_double), ("n_stored", _i64), ("status", _i32), ("reserved", _i32)]


_P = ctypes.POINTER
for _name, _args in (("pjds_tune_arena_bytes", [_i32, _i32, _vp, _P(_Cand), _i32, _P(_sz)]),
                     ("pjds_tune_sweep", [_i32, _i32, _vp, _vp, _vp, _P(_Cand), _i32, _i32, _vp, _sz, _vp, _sz,
                                          _P(_Entry), _P(_i32), _vp]),
                     ("pjds_tune_default_space", [_i32, _P(_Cand), _i32, _P(_i32)])):
    getattr(_lib, _name).restype = ctypes.c_int
    getattr(_lib, _name).argtypes = _args


def _cand_dict(c) -> dict:
    return {"b": c.b, "dtype": DTYPE_NAMES.get(c.dtype, c.dtype), "rows_per_thread": c.rows_per_thread,
            "threads_per_row": c.threads_per_row, "block_threads": c.block_threads, "unroll": c.unroll,
            "staged": c.staged, "plan": c.plan, "tile_order": c.tile_order}


def default_space(dtypes=("f64",), plan: bool = True) -> list:
    """The tuners' candidate space (pjds_tune_default_space): per dtype, b in
    {32,64,128,256} x threads per row in {1,2,4,8} x tile order in {sorted,
    table}, then the per-tile mapping for every b (36 per dtype); plan=False
    leaves the per-tile mapping out."""
    mask = 0
    for d in dtypes:
        mask |= 1 << _p.DTYPES[d]
    buf = (_Cand * 128)()
    n = _i32()
    _p._check(_lib.pjds_tune_default_space(mask, buf, 128, ctypes.byref(n)), "pjds_tune_default_space")
    out = [_cand_dict(buf[i]) for i in range(n.value)]
    return out if plan else [c for c in out if c["plan"] != 1]


def cand_key(c: dict) -> str:
    """Short name of a candidate: b32_T1_sorted, b64_T2_table, b32_plan."""
    if c.get("plan") == 1:
        return f"b{c['b']}_plan"
    order = {1: "table", -1: "sorted"}.get(c.get("tile_order", 0), "auto")
    return f"b{c['b']}_T{c.get('threads_per_row', 0)}_{order}"


def _to_cands(cands) -> ctypes.Array:
    arr = (_Cand * len(cands))()
    for i, c in enumerate(cands):
        arr[i] = _Cand(int(c["b"]), _p._dtype_code(c.get("dtype", "f64")), int(c.get("rows_per_thread", 0)),
                       int(c.get("threads_per_row", 0)), int(c.get("block_threads", 0)), int(c.get("unroll", 0)),
                       int(c.get("staged", 0)), int(c.get("plan", 0)), int(c.get("tile_order", 0)), 0)
    return arr


def arena_bytes(A, cands) -> int:
    rp = np.ascontiguousarray(A.row_ptr, np.int64)
    out = _sz()
    arr = _to_cands(cands)
    _p._check(_lib.pjds_tune_arena_bytes(A.n_rows, A.n_cols, rp.ctypes.data, arr, len(cands), ctypes.byref(out)),
              "pjds_tune_arena_bytes")
    return int(out.value)


def sweep(A, cands=None, reps: int = 5, flush_bytes: int = 256 << 20, device="cuda", stream=None):
    """Time every candidate on CRS matrix A (pjds_tune_sweep). Returns
    (entries, best_index); each entry: dict(cand..., us, n_stored, status)."""
    cands = cands if cands is not None else default_space()
    rp, col, val = _p._crs_args(A.row_ptr, A.col, A.val)
    arr = _to_cands(cands)
    need = arena_bytes(A, cands)
    arena = torch.empty(need, dtype=torch.uint8, device=device)
    flush = torch.empty(max(flush_bytes, 1), dtype=torch.uint8, device=device) if flush_bytes else None
    out = (_Entry * len(cands))()
    best = _i32()
    _p._check(_lib.pjds_tune_sweep(A.n_rows, A.n_cols, rp.ctypes.data, col.ctypes.data, val.ctypes.data, arr,
                                   len(cands), reps, arena.data_ptr(), need,
                                   flush.data_ptr() if flush is not None else None, flush_bytes if flush is not None
                                   else 0, out, ctypes.byref(best), _p._stream_ptr(stream)), "pjds_tune_sweep")
    entries = []
    for e in out:
        d = _cand_dict(e.cand)
        d.update(us=e.us, n_stored=e.n_stored, status=e.status)
        entries.append(d)
    return entries, best.value
