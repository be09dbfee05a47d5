"""Python binding of the learned tuner (include/pjds_mlp.h): argument
marshalling, plus saving and loading a trained model as JSON. The model's
training and inference run in libpjds's CUDA kernels; features and the
candidate encoding are computed in libpjds on the host."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import pjds as _p
from . import tune as _t

_lib = _p.lib()
IN, HID, NFEAT = 15, 64, 8
_f = ctypes.c_float
_vp, _i32, _u64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuner_mlp.json")


class Mlp(ctypes.Structure):
    _fields_ = [("w1", _f * (HID * IN)), ("b1", _f * HID), ("w2", _f * (HID * HID)), ("b2", _f * HID),
                ("w3", _f * HID), ("b3", _f), ("in_mean", _f * IN), ("in_std", _f * IN), ("out_mean", _f),
                ("out_std", _f), ("feat_lo", _f * NFEAT), ("feat_hi", _f * NFEAT)]

    def to_dict(self) -> dict:
        return {k: (list(getattr(self, k)) if hasattr(getattr(self, k), "__len__") else float(getattr(self, k)))
                for k, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "Mlp":
        m = cls()
        for k, _ in cls._fields_:
            if k not in d and k in ("feat_lo", "feat_hi"):
                # a model saved without a feature range: none set
                getattr(m, k)[:] = [1.0 if k == "feat_lo" else -1.0] * NFEAT
                continue
            v = d[k]
            if isinstance(v, list):
                getattr(m, k)[:] = v
            else:
                setattr(m, k, v)
        return m


_P = ctypes.POINTER

class Pick(ctypes.Structure):
    _fields_ = [("cand", _t._Cand), ("index", _i32), ("source", _i32), ("us", ctypes.c_double),
                ("n_outside", _i32), ("reserved", _i32)]


for _name, _args in (("pjds_mlp_init", [_P(Mlp), _u64]),
                     ("pjds_mlp_fit_range", [_P(Mlp), _vp, _i32]),
                     ("pjds_tune_pick", [_i32, _i32, _vp, _vp, _vp, _P(Mlp), _P(_t._Cand), _i32, _i32, _vp, _sz, _vp,
                                         _sz, _vp, _sz, _P(Pick), _vp]),
                     ("pjds_mlp_fit_scaling", [_P(Mlp), _vp, _vp, _i32]),
                     ("pjds_mlp_workspace_bytes", [_i32, _i32, _P(_sz)]),
                     ("pjds_mlp_train", [_P(Mlp), _vp, _vp, _i32, _i32, _i32, _f, _u64, _vp, _vp, _sz, _vp]),
                     ("pjds_mlp_predict", [_P(Mlp), _vp, _i32, _vp, _vp, _sz, _vp]),
                     ("pjds_features", [_i32, _i32, _vp, _vp, _vp]),
                     ("pjds_tune_encode", [_vp, _P(_t._Cand), _i32, _vp])):
    getattr(_lib, _name).restype = ctypes.c_int
    getattr(_lib, _name).argtypes = _args


def init(seed: int = 0) -> Mlp:
    m = Mlp()
    _p._check(_lib.pjds_mlp_init(ctypes.byref(m), seed), "pjds_mlp_init")
    return m


def fit_scaling(m: Mlp, X: np.ndarray, y: np.ndarray) -> Mlp:
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    _p._check(_lib.pjds_mlp_fit_scaling(ctypes.byref(m), X.ctypes.data, y.ctypes.data, len(y)),
              "pjds_mlp_fit_scaling")
    return m


def fit_range(m: Mlp, feats: np.ndarray) -> Mlp:
    """Set the model's feature range from the training matrices' features
    (pjds_mlp_fit_range)."""
    f = np.ascontiguousarray(feats, np.float32)
    _p._check(_lib.pjds_mlp_fit_range(ctypes.byref(m), f.ctypes.data, len(f)), "pjds_mlp_fit_range")
    return m


def _work(n: int, batch: int, device) -> torch.Tensor:
    b = _sz()
    _p._check(_lib.pjds_mlp_workspace_bytes(n, batch, ctypes.byref(b)), "pjds_mlp_workspace_bytes")
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def train(m: Mlp, X: np.ndarray, y: np.ndarray, epochs: int, batch: int, lr: float, seed: int = 0,
          device="cuda", stream=None) -> np.ndarray:
    """Train m in place (pjds_mlp_train); returns the per-epoch loss."""
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    n = len(y)
    work = _work(n, batch, device)
    hist = np.zeros(max(epochs, 1), np.float32)
    _p._check(_lib.pjds_mlp_train(ctypes.byref(m), X.ctypes.data, y.ctypes.data, n, epochs, batch, lr, seed,
                                  hist.ctypes.data, work.data_ptr(), work.numel(), _p._stream_ptr(stream)),
              "pjds_mlp_train")
    return hist[:epochs]


def predict(m: Mlp, X: np.ndarray, device="cuda", stream=None) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float32)
    n = X.shape[0]
    out = np.zeros(n, np.float32)
    work = _work(n, 1, device)
    _p._check(_lib.pjds_mlp_predict(ctypes.byref(m), X.ctypes.data, n, out.ctypes.data, work.data_ptr(),
                                    work.numel(), _p._stream_ptr(stream)), "pjds_mlp_predict")
    return out


def features(A) -> np.ndarray:
    rp, col, _ = _p._crs_args(A.row_ptr, A.col, np.zeros(0))
    out = np.zeros(NFEAT, np.float32)
    _p._check(_lib.pjds_features(A.n_rows, A.n_cols, rp.ctypes.data, col.ctypes.data, out.ctypes.data),
              "pjds_features")
    return out


def encode(feat: np.ndarray, cands) -> np.ndarray:
    feat = np.ascontiguousarray(feat, np.float32)
    arr = _t._to_cands(cands)
    out = np.zeros((len(cands), IN), np.float32)
    _p._check(_lib.pjds_tune_encode(feat.ctypes.data, arr, len(cands), out.ctypes.data), "pjds_tune_encode")
    return out


def save(m: Mlp, path: str = MODEL_PATH, meta: dict | None = None) -> None:
    with open(path, "w") as fh:
        json.dump({"model": m.to_dict(), "meta": meta or {}}, fh)


def load(path: str = MODEL_PATH) -> Mlp:
    with open(path) as fh:
        return Mlp.from_dict(json.load(fh)["model"])


def pick(A, dtype="f64", cands=None, model: Mlp | None = None, reps: int = 5, flush_bytes: int = 256 << 20,
         device="cuda", stream=None) -> dict:
    """Launch configuration for CRS matrix A (pjds_tune_pick): the model's
    choice among the candidates when A's features lie within the model's
    training range, else the exhaustive sweep's fastest. Returns the
    candidate dict plus index, source ("model" or "sweep"), us (predicted or
    measured) and n_outside. The sweep's arena and L2-flush buffer are
    allocated here only when the sweep has to run."""
    cands = cands if cands is not None else _t.default_space((dtype,))
    model = model if model is not None else load()
    rp, col, val = _p._crs_args(A.row_ptr, A.col, A.val)
    arr = _t._to_cands(cands)
    work = _work(len(cands), 1, device)
    out = Pick()
    # without an arena pjds_tune_pick answers from the model, or reports that
    # the sweep is needed
    feat = features(A)
    lo, hi = np.array(model.feat_lo), np.array(model.feat_hi)
    tol = 0.02 * (hi - lo)
    inside = bool(np.all((lo > hi) | ((feat >= lo - tol) & (feat <= hi + tol))))
    arena = flush = None
    if not inside:
        arena = torch.empty(_t.arena_bytes(A, cands), dtype=torch.uint8, device=device)
        flush = torch.empty(max(flush_bytes, 1), dtype=torch.uint8, device=device) if flush_bytes else None
    _p._check(_lib.pjds_tune_pick(A.n_rows, A.n_cols, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                  ctypes.byref(model), arr, len(cands), reps, work.data_ptr(), work.numel(),
                                  arena.data_ptr() if arena is not None else None,
                                  arena.numel() if arena is not None else 0,
                                  flush.data_ptr() if flush is not None else None,
                                  flush.numel() if flush is not None else 0, ctypes.byref(out),
                                  _p._stream_ptr(stream)), "pjds_tune_pick")
    res = dict(cands[out.index])
    res.update(index=int(out.index), source="model" if out.source == 0 else "sweep", us=float(out.us),
               n_outside=int(out.n_outside))
    return res


def choose(A, cands=None, model: Mlp | None = None, device="cuda") -> tuple:
    """Candidate with the smallest predicted time for CRS matrix A:
    (index, candidate, predicted microseconds per candidate)."""
    cands = cands if cands is not None else _t.default_space(("f64", "f32", "bf16"))
    model = model if model is not None else load()
    pred = np.exp(predict(model, encode(features(A), cands), device=device))
    i = int(np.argmin(pred))
    return i, cands[i], pred
