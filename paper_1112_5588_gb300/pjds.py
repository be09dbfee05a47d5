"""Python binding of libpjds (ctypes): argument marshalling only.

Names follow the C ABI in include/pjds.h. Every step of the product runs in the
library's CUDA kernels; this module only moves host arrays into torch device
tensors, fills the ABI structs and passes pointers and the current torch stream.
There is no CPU fallback: if libpjds.so is missing, importing this module fails.

Typical use::

    H = pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64")
    D = H.to_device("cuda")          # torch-owned device buffers
    y = torch.empty(H.n_rows, dtype=D.vec_dtype, device="cuda")
    pjds_spmv(D, x, y)               # y = A x on the current stream
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# PJDS_LIBRARY=checked loads the checked build (device-side extent checks,
# a test build); the product library otherwise
LIB_PATH = os.path.join(_HERE, "libpjds_checked.so" if os.environ.get("PJDS_LIBRARY") == "checked" else "libpjds.so")

DTYPES = {"f64": 0, "f32": 1, "bf16": 2}
_VEC_TORCH = {0: torch.float64, 1: torch.float32, 2: torch.float32}
_VAL_NP = {0: np.float64, 1: np.float32, 2: np.uint16}
_VAL_BYTES = {0: 8, 1: 4, 2: 2}

_i32, _i64, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p


class PjdsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


class _PjdsHostS(ctypes.Structure):
    _fields_ = [("n_rows", _i32), ("n_cols", _i32), ("n_pad", _i32), ("b", _i32), ("n_blocks", _i32),
                ("n_max", _i32), ("nnz", _i64), ("n_stored", _i64), ("dtype", _i32), ("permute_cols", _i32),
                ("perm", _vp), ("inv_perm", _vp), ("block_len", _vp), ("row_len", _vp), ("col_start", _vp),
                ("col", _vp), ("val", _vp), ("tile_order", _vp), ("plan", _vp), ("n_plan", _i32),
                ("pair_share", _i32)]


class _PjdsDevS(ctypes.Structure):
    _fields_ = [("n_rows", _i32), ("n_cols", _i32), ("n_pad", _i32), ("b", _i32), ("n_blocks", _i32),
                ("n_max", _i32), ("nnz", _i64), ("n_stored", _i64), ("dtype", _i32), ("permute_cols", _i32),
                ("perm", _vp), ("block_len", _vp), ("row_len", _vp), ("col_start", _vp), ("col", _vp),
                ("val", _vp), ("tile_order", _vp), ("plan", _vp), ("n_plan", _i32), ("pair_share", _i32)]


class _LaunchS(ctypes.Structure):
    _fields_ = [("rows_per_thread", _i32), ("threads_per_row", _i32), ("block_threads", _i32), ("unroll", _i32),
                ("staged", _i32), ("index64", _i32), ("tile_order", _i32), ("plan", _i32)]


class _EllrHostS(ctypes.Structure):
    _fields_ = [("n_rows", _i32), ("n_cols", _i32), ("n_pad", _i32), ("n_max", _i32), ("nnz", _i64),
                ("n_stored", _i64), ("dtype", _i32), ("reserved", _i32), ("row_max", _vp), ("col", _vp),
                ("val", _vp)]


class _EllrDevS(ctypes.Structure):
    _fields_ = [("n_rows", _i32), ("n_cols", _i32), ("n_pad", _i32), ("n_max", _i32), ("nnz", _i64),
                ("n_stored", _i64), ("dtype", _i32), ("reserved", _i32), ("row_max", _vp), ("col", _vp),
                ("val", _vp)]


def _load_lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1112_5588_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "pjds_last_error": (ctypes.c_char_p, []),
        "pjds_version": (_i32, []),
        "pjds_abi_sizes": (None, [_vp]),
        "pjds_create": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _i32, P(P(_PjdsHostS))]),
        "pjds_create_shape": (ctypes.c_int, [_i32, _i32, _vp, _i32, _i32, P(P(_PjdsHostS))]),
        "pjds_destroy": (ctypes.c_int, [P(_PjdsHostS)]),
        "pjds_spmv": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, _vp]),
        "pjds_spmv_cfg": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, P(_LaunchS), _vp]),
        "pjds_spmv_pattern": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, P(_LaunchS), _vp]),
        "pjds_spmv_host": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, _vp, _vp, _vp]),
        "pjds_spmv_host_stream": (ctypes.c_int, [P(_PjdsDevS), _i32, P(_vp), P(_vp), P(_vp), P(_vp), _vp]),
        "pjds_spmv_resolve": (ctypes.c_int, [P(_PjdsDevS), P(_LaunchS), P(_LaunchS)]),
        "pjds_device_status": (ctypes.c_int, [P(_i32), _i32, _vp]),
        "pjds_check_word": (ctypes.c_int, [P(ctypes.c_uint64), _i32, _vp]),
        "pjds_wait_selftest": (ctypes.c_int, [_i32, _vp]),
        "pjds_permute": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, _vp]),
        "pjds_unpermute": (ctypes.c_int, [P(_PjdsDevS), _vp, _vp, _vp]),
        "ellr_create": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp, _i32, P(P(_EllrHostS))]),
        "ellr_destroy": (ctypes.c_int, [P(_EllrHostS)]),
        "ellr_spmv": (ctypes.c_int, [P(_EllrDevS), _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    sizes = (ctypes.c_int32 * 5)()
    lib.pjds_abi_sizes(sizes)
    want = [ctypes.sizeof(s) for s in (_PjdsHostS, _PjdsDevS, _LaunchS, _EllrHostS, _EllrDevS)]
    if list(sizes) != want:
        raise ImportError(f"libpjds ABI struct sizes {list(sizes)} differ from the binding's {want}")
    return lib


_lib = _load_lib()


def lib():
    """The loaded ctypes library (for tests that call the C ABI directly)."""
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise PjdsError(rc, where, _lib.pjds_last_error().decode(errors="replace"))


def _dtype_code(dtype) -> int:
    if isinstance(dtype, str):
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {sorted(DTYPES)}")
        return DTYPES[dtype]
    return int(dtype)


def _np_view(ptr, n, np_dtype):
    n = int(n)
    if n == 0 or not ptr:
        return np.zeros(0, np_dtype)
    buf = (ctypes.c_char * (n * np.dtype(np_dtype).itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype=np_dtype, count=n)


def _stream_ptr(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _crs_args(row_ptr, col, val):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    return rp, c, v


# --------------------------------------------------------------------------- pJDS

class PjdsHost:
    """pJDS arrays owned by the library (pjds_host); numpy views stay valid
    until destroy()."""

    def __init__(self, ptr):
        self._ptr = ptr
        s = ptr.contents
        for f, _ in _PjdsHostS._fields_[:10]:
            setattr(self, f, int(getattr(s, f)))
        self.perm = _np_view(s.perm, s.n_rows, np.int32)
        self.inv_perm = _np_view(s.inv_perm, s.n_rows, np.int32)
        self.block_len = _np_view(s.block_len, s.n_blocks, np.int32)
        self.row_len = _np_view(s.row_len, s.n_pad, np.int32)
        self.col_start = _np_view(s.col_start, s.n_max + 1, np.int64)
        self.col = _np_view(s.col, s.n_stored, np.int32)
        self.val = _np_view(s.val, s.n_stored, _VAL_NP[s.dtype])
        self.tile_order = _np_view(s.tile_order, s.n_pad // 32, np.int32)
        self.n_plan = int(s.n_plan)
        # per mille of entries sharing the paired row's column (the default mapping's statistic)
        self.pair_share = int(s.pair_share)
        # per-tile mapping: n_plan rows of (0, first sorted row, rows, kind)
        self.plan = _np_view(s.plan, 4 * s.n_plan, np.int32).reshape(-1, 4)

    def arrays(self) -> dict:
        """Copies of every array plus the sizes (survive destroy())."""
        out = {k: getattr(self, k) for k, _ in _PjdsHostS._fields_[:10]}
        for k in ("perm", "inv_perm", "block_len", "row_len", "col_start", "col", "val", "tile_order", "plan"):
            out[k] = getattr(self, k).copy()
        out["n_plan"] = self.n_plan
        out["pair_share"] = self.pair_share
        return out

    def to_device(self, device="cuda", tile_order: bool = True, plan: bool = True) -> "PjdsDevice":
        """Upload; tile_order=False leaves the traversal table out (tiles in
        sorted order), plan=False the per-tile mapping (uniform mappings only):
        same results, for comparisons."""
        return PjdsDevice(self, device, tile_order, plan)

    def destroy(self):
        if self._ptr is not None:
            _lib.pjds_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pjds_create(n_rows: int, n_cols: int, row_ptr, col, val, b: int = 32, dtype="f64",
                permute_cols: bool = False) -> PjdsHost:
    """CRS -> pJDS on the host (pjds_create)."""
    rp, c, v = _crs_args(row_ptr, col, val)
    if len(rp) != n_rows + 1:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    out = ctypes.POINTER(_PjdsHostS)()
    _check(_lib.pjds_create(n_rows, n_cols, rp.ctypes.data, c.ctypes.data, v.ctypes.data, b, _dtype_code(dtype),
                            1 if permute_cols else 0, ctypes.byref(out)), "pjds_create")
    return PjdsHost(out)


def pjds_create_shape(n_rows: int, n_cols: int, row_ptr, b: int = 32, dtype="f64") -> PjdsHost:
    """The pJDS structure from the row lengths alone (pjds_create_shape):
    col and val are empty; PjdsDevice(host, col=..., val=...) takes them as
    caller-filled device tensors."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    if len(rp) != n_rows + 1:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    out = ctypes.POINTER(_PjdsHostS)()
    _check(_lib.pjds_create_shape(n_rows, n_cols, rp.ctypes.data, b, _dtype_code(dtype), ctypes.byref(out)),
           "pjds_create_shape")
    return PjdsHost(out)


class PjdsDevice:
    """Device copy of a pJDS matrix in torch-owned buffers plus its pjds_dev
    struct. col / val: device tensors of n_stored entries (int32, and the
    value type; bf16 as int16 bits) to use instead of uploading the host's."""

    def __init__(self, host: PjdsHost, device="cuda", tile_order: bool = True, plan: bool = True,
                 col: torch.Tensor | None = None, val: torch.Tensor | None = None):
        dev = torch.device(device)
        self.device = dev
        self.dtype = host.dtype
        self.vec_dtype = _VEC_TORCH[host.dtype]
        self.n_rows, self.n_cols, self.n_pad = host.n_rows, host.n_cols, host.n_pad
        self.nnz, self.n_stored, self.b, self.n_max = host.nnz, host.n_stored, host.b, host.n_max
        self.permute_cols = host.permute_cols

        def up(a, np_dt):
            return torch.from_numpy(np.ascontiguousarray(a).view(np_dt).copy()).to(dev)

        self.perm = up(host.perm, np.int32)
        self.block_len = up(host.block_len, np.int32)
        self.row_len = up(host.row_len, np.int32)
        self.col_start = up(host.col_start, np.int64)
        if col is not None or val is not None:
            vt = {0: torch.float64, 1: torch.float32, 2: torch.int16}[host.dtype]
            for t, n, dt, nm in ((col, host.n_stored, torch.int32, "col"), (val, host.n_stored, vt, "val")):
                if t is None or t.device.type != "cuda" or t.dtype != dt or t.numel() != n or not t.is_contiguous():
                    raise ValueError(f"{nm} must be a contiguous CUDA {dt} tensor with {n} elements")
            self.col, self.val = col, val
        else:
            self.col = up(host.col, np.int32)
            self.val = up(host.val, {0: np.float64, 1: np.float32, 2: np.int16}[host.dtype])
        self.tile_order = up(host.tile_order, np.int32) if tile_order else None
        self.n_plan = host.n_plan if plan else 0
        self.plan = up(host.plan, np.int32) if plan and host.n_plan > 0 else None
        s = _PjdsDevS()
        for f, _ in _PjdsDevS._fields_[:10]:
            setattr(s, f, getattr(host, f))
        s.perm = self.perm.data_ptr() or None
        s.block_len = self.block_len.data_ptr() or None
        s.row_len = self.row_len.data_ptr() or None
        s.col_start = self.col_start.data_ptr() or None
        s.col = self.col.data_ptr() or None
        s.val = self.val.data_ptr() or None
        s.tile_order = (self.tile_order.data_ptr() or None) if tile_order else None
        s.plan = self.plan.data_ptr() if self.plan is not None else None
        s.n_plan = self.n_plan if self.plan is not None else 0
        s.pair_share = host.pair_share
        self.pair_share = host.pair_share
        self._s = s

    @property
    def struct(self):
        return self._s

    def device_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.perm, self.block_len, self.row_len, self.col_start,
                                                           self.col, self.val, self.tile_order, self.plan)
                   if t is not None)


def _check_vec(t: torch.Tensor, n: int, dtype, name: str):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or t.numel() != n or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor with {n} elements")


def pjds_spmv(A: PjdsDevice, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = A x (pjds_spmv). Original basis unless A was built with permute_cols."""
    _check_vec(x, A.n_cols, A.vec_dtype, "x")
    _check_vec(y, A.n_rows, A.vec_dtype, "y")
    _check(_lib.pjds_spmv(ctypes.byref(A.struct), x.data_ptr(), y.data_ptr(), _stream_ptr(stream)), "pjds_spmv")
    return y


def pjds_spmv_cfg(A: PjdsDevice, x: torch.Tensor, y: torch.Tensor, rows_per_thread: int = 0,
                  threads_per_row: int = 0, block_threads: int = 0, unroll: int = 0, staged: int = 0,
                  index64: int = 0, tile_order: int = 0, plan: int = 0, stream=None) -> torch.Tensor:
    """y = A x with an explicit kernel configuration (pjds_spmv_cfg).
    tile_order: 0 automatic, 1 traversal table, -1 sorted order; plan: 0
    automatic, 1 the per-tile mapping, -1 a uniform mapping."""
    _check_vec(x, A.n_cols, A.vec_dtype, "x")
    _check_vec(y, A.n_rows, A.vec_dtype, "y")
    cfg = _LaunchS(rows_per_thread, threads_per_row, block_threads, unroll, staged, index64, tile_order, plan)
    _check(_lib.pjds_spmv_cfg(ctypes.byref(A.struct), x.data_ptr(), y.data_ptr(), ctypes.byref(cfg),
                              _stream_ptr(stream)), "pjds_spmv_cfg")
    return y


def pjds_spmv_pattern(A: PjdsDevice, x: torch.Tensor, y: torch.Tensor, stream=None, **cfg) -> torch.Tensor:
    """y = S x, S the sparsity pattern of A (values taken as 1; pjds_spmv_pattern):
    the traversal of pjds_spmv_cfg(**cfg) without the value stream."""
    _check_vec(x, A.n_cols, A.vec_dtype, "x")
    _check_vec(y, A.n_rows, A.vec_dtype, "y")
    keys = ("rows_per_thread", "threads_per_row", "block_threads", "unroll", "staged", "index64", "tile_order",
            "plan")
    c = _LaunchS(*[int(cfg.pop(k, 0)) for k in keys])
    if cfg:
        raise TypeError(f"unknown launch fields {sorted(cfg)}")
    _check(_lib.pjds_spmv_pattern(ctypes.byref(A.struct), x.data_ptr(), y.data_ptr(), ctypes.byref(c),
                                  _stream_ptr(stream)), "pjds_spmv_pattern")
    return y


def pjds_spmv_resolve(A, rows_per_thread: int = 0, threads_per_row: int = 0, block_threads: int = 0,
                      unroll: int = 0, staged: int = 0, index64: int = 0, tile_order: int = 0, plan: int = 0) -> dict:
    """The launch configuration pjds_spmv_cfg would use (no launch). `A` is a
    PjdsDevice or a PjdsHost (only sizes and alignment are read)."""
    s = A.struct if isinstance(A, PjdsDevice) else _dev_struct_from_host(A)
    cfg = _LaunchS(rows_per_thread, threads_per_row, block_threads, unroll, staged, index64, tile_order, plan)
    out = _LaunchS()
    _check(_lib.pjds_spmv_resolve(ctypes.byref(s), ctypes.byref(cfg), ctypes.byref(out)), "pjds_spmv_resolve")
    return {"rows_per_thread": out.rows_per_thread, "threads_per_row": out.threads_per_row,
            "block_threads": out.block_threads, "unroll": out.unroll, "staged": out.staged,
            "index64": out.index64, "tile_order": out.tile_order, "plan": out.plan}


def pjds_check_word(clear: bool = True, stream=None) -> int:
    """The checked build's first out-of-extent access, (code << 56) | index,
    0 when none (pjds_check_word; PjdsError in the normal build)."""
    w = ctypes.c_uint64()
    _check(_lib.pjds_check_word(ctypes.byref(w), 1 if clear else 0, _stream_ptr(stream)), "pjds_check_word")
    return int(w.value)


def pjds_wait_selftest(which: int = 0, stream=None) -> None:
    """Launch the bounded-wait self-test (pjds_wait_selftest)."""
    _check(_lib.pjds_wait_selftest(which, _stream_ptr(stream)), "pjds_wait_selftest")


def pjds_device_status(clear: bool = True, stream=None) -> int:
    """The staged kernel's device status word (0 = every wait completed)."""
    st = _i32()
    _check(_lib.pjds_device_status(ctypes.byref(st), 1 if clear else 0, _stream_ptr(stream)), "pjds_device_status")
    return st.value


def _dev_struct_from_host(H: "PjdsHost"):
    s = _PjdsDevS()
    for f, _ in _PjdsDevS._fields_[:10]:
        setattr(s, f, getattr(H, f))
    # alignment of torch allocations (512 B) stands in for the device pointers
    s.val = s.col = s.col_start = s.block_len = s.perm = 512
    s.tile_order = 512 if len(H.tile_order) else None
    s.plan = 512 if H.n_plan else None
    s.n_plan = H.n_plan
    s.pair_share = H.pair_share
    return s


def pjds_spmv_host(A: PjdsDevice, x_host: torch.Tensor, y_host: torch.Tensor, x_dev: torch.Tensor,
                   y_dev: torch.Tensor, stream=None) -> torch.Tensor:
    """Host x -> device -> y = A x -> host y, synchronous (pjds_spmv_host)."""
    for t, n, name in ((x_host, A.n_cols, "x_host"), (y_host, A.n_rows, "y_host")):
        if t.device.type != "cpu" or t.dtype != A.vec_dtype or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU {A.vec_dtype} tensor with {n} elements")
    _check_vec(x_dev, A.n_cols, A.vec_dtype, "x_dev")
    _check_vec(y_dev, A.n_rows, A.vec_dtype, "y_dev")
    _check(_lib.pjds_spmv_host(ctypes.byref(A.struct), x_host.data_ptr(), y_host.data_ptr(), x_dev.data_ptr(),
                               y_dev.data_ptr(), _stream_ptr(stream)), "pjds_spmv_host")
    return y_host


def pjds_spmv_host_stream(A: PjdsDevice, xs_host, ys_host, x_dev, y_dev, stream=None):
    """y_v = A x_v for a list of host vectors, copies overlapped with the
    products (pjds_spmv_host_stream). x_dev, y_dev: two device buffers each."""
    if len(xs_host) != len(ys_host):
        raise ValueError("xs_host and ys_host must have the same length")
    for lst, n, name in ((xs_host, A.n_cols, "x_host"), (ys_host, A.n_rows, "y_host")):
        for t in lst:
            if t.device.type != "cpu" or t.dtype != A.vec_dtype or t.numel() != n or not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous CPU {A.vec_dtype} tensors with {n} elements")
    if len(x_dev) != 2 or len(y_dev) != 2:
        raise ValueError("x_dev and y_dev must hold two device buffers each")
    for t in x_dev:
        _check_vec(t, A.n_cols, A.vec_dtype, "x_dev")
    for t in y_dev:
        _check_vec(t, A.n_rows, A.vec_dtype, "y_dev")
    n = len(xs_host)
    xp = (_vp * max(n, 1))(*[t.data_ptr() for t in xs_host])
    yp = (_vp * max(n, 1))(*[t.data_ptr() for t in ys_host])
    xd = (_vp * 2)(*[t.data_ptr() for t in x_dev])
    yd = (_vp * 2)(*[t.data_ptr() for t in y_dev])
    _check(_lib.pjds_spmv_host_stream(ctypes.byref(A.struct), n, xp, yp, xd, yd, _stream_ptr(stream)),
           "pjds_spmv_host_stream")
    return ys_host


def pjds_permute(A: PjdsDevice, v: torch.Tensor, v_perm: torch.Tensor, stream=None) -> torch.Tensor:
    """v_perm[i] = v[perm[i]] (original -> permuted basis)."""
    _check_vec(v, A.n_rows, A.vec_dtype, "v")
    _check_vec(v_perm, A.n_rows, A.vec_dtype, "v_perm")
    _check(_lib.pjds_permute(ctypes.byref(A.struct), v.data_ptr(), v_perm.data_ptr(), _stream_ptr(stream)),
           "pjds_permute")
    return v_perm


def pjds_unpermute(A: PjdsDevice, v_perm: torch.Tensor, v: torch.Tensor, stream=None) -> torch.Tensor:
    """v[perm[i]] = v_perm[i] (permuted -> original basis)."""
    _check_vec(v_perm, A.n_rows, A.vec_dtype, "v_perm")
    _check_vec(v, A.n_rows, A.vec_dtype, "v")
    _check(_lib.pjds_unpermute(ctypes.byref(A.struct), v_perm.data_ptr(), v.data_ptr(), _stream_ptr(stream)),
           "pjds_unpermute")
    return v


# --------------------------------------------------------------------------- ELLPACK-R

class EllrHost:
    """ELLPACK-R arrays owned by the library (ellr_host)."""

    def __init__(self, ptr):
        self._ptr = ptr
        s = ptr.contents
        for f, _ in _EllrHostS._fields_[:8]:
            setattr(self, f, int(getattr(s, f)))
        self.row_max = _np_view(s.row_max, s.n_pad, np.int32)
        self.col = _np_view(s.col, s.n_stored, np.int32)
        self.val = _np_view(s.val, s.n_stored, _VAL_NP[s.dtype])

    def arrays(self) -> dict:
        out = {k: getattr(self, k) for k, _ in _EllrHostS._fields_[:8]}
        for k in ("row_max", "col", "val"):
            out[k] = getattr(self, k).copy()
        return out

    def to_device(self, device="cuda") -> "EllrDevice":
        return EllrDevice(self, device)

    def destroy(self):
        if self._ptr is not None:
            _lib.ellr_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ellr_create(n_rows: int, n_cols: int, row_ptr, col, val, dtype="f64") -> EllrHost:
    """CRS -> ELLPACK-R on the host (ellr_create)."""
    rp, c, v = _crs_args(row_ptr, col, val)
    if len(rp) != n_rows + 1:
        raise ValueError("row_ptr must have n_rows + 1 entries")
    out = ctypes.POINTER(_EllrHostS)()
    _check(_lib.ellr_create(n_rows, n_cols, rp.ctypes.data, c.ctypes.data, v.ctypes.data, _dtype_code(dtype),
                            ctypes.byref(out)), "ellr_create")
    return EllrHost(out)


class EllrDevice:
    def __init__(self, host: EllrHost, device="cuda"):
        dev = torch.device(device)
        self.device = dev
        self.dtype = host.dtype
        self.vec_dtype = _VEC_TORCH[host.dtype]
        self.n_rows, self.n_cols, self.n_pad, self.n_max = host.n_rows, host.n_cols, host.n_pad, host.n_max
        self.nnz, self.n_stored = host.nnz, host.n_stored
        vt = {0: torch.float64, 1: torch.float32, 2: torch.int16}[host.dtype]
        npt = {torch.float64: np.float64, torch.float32: np.float32, torch.int16: np.int16}[vt]
        self.row_max = torch.from_numpy(host.row_max.copy()).to(dev)
        self.col = torch.from_numpy(host.col.copy()).to(dev)
        self.val = torch.from_numpy(host.val.copy().view(npt)).to(dev)
        s = _EllrDevS()
        for f, _ in _EllrDevS._fields_[:8]:
            setattr(s, f, getattr(host, f))
        s.row_max = self.row_max.data_ptr() or None
        s.col = self.col.data_ptr() or None
        s.val = self.val.data_ptr() or None
        self._s = s

    @property
    def struct(self):
        return self._s


def ellr_spmv(A: EllrDevice, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y = A x with A in ELLPACK-R (ellr_spmv)."""
    _check_vec(x, A.n_cols, A.vec_dtype, "x")
    _check_vec(y, A.n_rows, A.vec_dtype, "y")
    _check(_lib.ellr_spmv(ctypes.byref(A.struct), x.data_ptr(), y.data_ptr(), _stream_ptr(stream)), "ellr_spmv")
    return y
