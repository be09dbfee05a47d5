"""The paper's node-level performance model (Sect. 2.2, Eqs. 1-4) and the
storage arithmetic of Sect. 2.1, as host-side helpers for reporting.

Notation: N rows, N_nzr nonzeros per row (average), alpha in [1/N_nzr, 1] the
fraction of right-hand-side loads that miss the cache (alpha = 1/N_nzr: every
x element is loaded once; alpha = 1: no cache), B_GPU and B_PCI the device
memory and PCIe bandwidths.

Reading: Eq. 1 is written with N_nzr^max, while the text then assumes an
average N_nzr; this module takes the average throughout. The worst-case values
the paper prints after Eqs. 3 and 4 (25 and 266) follow when alpha = 1/N_nzr
is neglected against 3/2, so ``alpha=0`` reproduces them.
"""
from __future__ import annotations


def code_balance(alpha: float, n_nzr: float, precision: str = "dp") -> float:
    """Bytes per flop of y = A x (Eq. 1): per nonzero one value, one 4-byte
    index and alpha right-hand-side elements; per row one load and one store of
    the result (16/N_nzr bytes in double precision); two flops per nonzero.
    Double: 6 + 4 alpha + 8/N_nzr. Single: 4 + 2 alpha + 4/N_nzr."""
    w = 8.0 if precision == "dp" else 4.0
    return (w + 4.0 + w * alpha + 2.0 * w / n_nzr) / 2.0


def t_mvm(n: float, n_nzr: float, alpha: float, b_gpu: float) -> float:
    """Kernel time at bandwidth b_gpu (Eq. 2, left): 8N/B_GPU [N_nzr(alpha + 3/2) + 2]."""
    return 8.0 * n / b_gpu * (n_nzr * (alpha + 1.5) + 2.0)


def t_pci(n: float, b_pci: float) -> float:
    """Transfer of x to and y from the device (Eq. 2, right): 16N/B_PCI."""
    return 16.0 * n / b_pci


def nnzr_pcie_dominates(bw_ratio: float, alpha: float) -> float:
    """Eq. 3: T_MVM <= T_PCI (more than 50% penalty) for N_nzr at or below
    2 (B_GPU/B_PCI - 1) / (alpha + 3/2)."""
    return 2.0 * (bw_ratio - 1.0) / (alpha + 1.5)


def nnzr_pcie_below_10pct(bw_ratio: float, alpha: float) -> float:
    """Eq. 4: T_MVM >= 10 T_PCI (under 10% penalty) for N_nzr at or above
    (20 B_GPU/B_PCI - 2) / (alpha + 3/2)."""
    return (20.0 * bw_ratio - 2.0) / (alpha + 1.5)


def roofline_gflops(b_gpu_gbs: float, alpha: float, n_nzr: float, precision: str = "dp") -> float:
    """Attainable GF/s = bandwidth / code balance."""
    return b_gpu_gbs / code_balance(alpha, n_nzr, precision)


def ellpack_entries(n_pad: int, n_max: int) -> int:
    """ELLPACK / ELLPACK-R stored entries: the full N_pad x N_max rectangle."""
    return n_pad * n_max


def one_full_row_pjds_entries(n: int, b: int) -> int:
    """pJDS entries for one full row plus one entry in each other row
    (Sect. 2.1): b N + N - b = (b + 1) N - b (N a multiple of b)."""
    return (b + 1) * n - b


def data_reduction(n_stored_pjds: int, n_stored_ellpack: int) -> float:
    """Fraction of ELLPACK storage that pJDS saves (Table 1's row), taken as
    1 - S_pJDS / S_ELLPACK on stored (value, index) pairs."""
    return 1.0 - n_stored_pjds / n_stored_ellpack if n_stored_ellpack else 0.0
