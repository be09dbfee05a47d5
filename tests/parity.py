"""Shared parity checks for the CUDA path against the oracle.

Tolerances (written here, used by every GPU test):
  FP64 (stated bound): ||y - y_ref||_inf / || |A||x| ||_inf <= 1e-14, and
    element by element |y_i - y_ref_i| <= (gamma_n(2^-53) + gamma_n(2^-53)) (|A||x|)_i,
    n = row length: the kernel's fused multiply-adds and the oracle's separate
    multiply and add are each within gamma_n (|A||x|)_i of the exact sum.
  FP32 / BF16 values with FP32 accumulation: the oracle runs in fp64 on the
    values the kernel holds (rounded by the oracle's own definition) and on
    x as stored; |y_i - y_ref_i| <= (gamma_n(2^-24) + gamma_n(2^-53)) (|A||x|)_i
    plus one rounding of y_ref to binary32.
"""
from __future__ import annotations

import numpy as np

U64 = 2.0 ** -53
U32 = 2.0 ** -24
FP64_NORMWISE_TOL = 1e-14


def gamma(n: np.ndarray, u: float) -> np.ndarray:
    n = np.asarray(n, np.float64)
    return n * u / (1.0 - n * u)


def normwise_error(y, y_ref, absax) -> float:
    scale = float(np.max(absax)) if len(absax) else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(y - y_ref))) if len(y) else 0.0
    return float(np.max(np.abs(y - y_ref))) / scale


def check_fp64(y, y_ref, absax, row_lens) -> dict:
    y = np.asarray(y, np.float64)
    err = np.abs(y - y_ref)
    bound = 2.0 * gamma(row_lens, U64) * absax
    bad = np.nonzero(err > bound)[0]
    nw = normwise_error(y, y_ref, absax)
    return {"normwise": nw, "n_bad": int(len(bad)), "first_bad": bad[:5].tolist(),
            "ok": len(bad) == 0 and nw <= FP64_NORMWISE_TOL}


def check_fp32(y, y_ref, absax, row_lens) -> dict:
    y = np.asarray(y, np.float64)
    err = np.abs(y - y_ref)
    bound = (gamma(row_lens, U32) + gamma(row_lens, U64)) * absax + U32 * np.abs(y_ref)
    bad = np.nonzero(err > bound)[0]
    return {"normwise": normwise_error(y, y_ref, absax), "n_bad": int(len(bad)), "first_bad": bad[:5].tolist(),
            "ok": len(bad) == 0}
