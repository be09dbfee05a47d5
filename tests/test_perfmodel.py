"""The performance model against the numbers the paper prints (Sect. 2.1, 2.2)."""
import json
import math
import os

import pytest

from paper_1112_5588_gb300 import perfmodel as pm


@pytest.fixture(scope="module")
def g(golden_dir):
    with open(os.path.join(golden_dir, "paper_numbers.json")) as fh:
        return json.load(fh)


def test_eq1_terms():
    # 6 + 4 alpha + 8/N_nzr in double precision
    assert pm.code_balance(1.0, 8.0) == 6 + 4 + 1
    assert pm.code_balance(0.25, 16.0) == 6 + 1 + 0.5
    assert pm.code_balance(1.0, 8.0, "sp") == 4 + 2 + 0.5


def test_eq2_consistent_with_eq1():
    # T_MVM * B_GPU = bytes = flops * balance, flops = 2 N N_nzr
    n, nzr, a, bw = 1e6, 15.0, 0.3, 100e9
    assert math.isclose(pm.t_mvm(n, nzr, a, bw) * bw, 2 * n * nzr * pm.code_balance(a, nzr), rel_tol=1e-12)
    assert pm.t_pci(1e6, 8e9) == 16e6 / 8e9


def test_eq3_printed_bounds(g):
    assert g["eq3_worst_case"]["printed_bound"] == math.floor(pm.nnzr_pcie_dominates(20, 0.0)) == 25
    assert g["eq3_alpha1"]["printed_bound"] == math.floor(pm.nnzr_pcie_dominates(10, 1.0)) == 7


def test_eq4_printed_bounds(g):
    assert g["eq4_alpha1"]["printed_bound"] == math.ceil(pm.nnzr_pcie_below_10pct(10, 1.0)) == 80
    assert g["eq4_worst_case"]["printed_bound"] == math.ceil(pm.nnzr_pcie_below_10pct(20, 0.0)) == 266


def test_eq3_is_the_crossing_of_eq2():
    # at the Eq. 3 bound T_MVM == T_PCI
    ratio, a, n = 12.0, 0.5, 1e6
    nzr = pm.nnzr_pcie_dominates(ratio, a)
    assert math.isclose(pm.t_mvm(n, nzr, a, ratio * 1e9), pm.t_pci(n, 1e9), rel_tol=1e-12)
    nzr4 = pm.nnzr_pcie_below_10pct(ratio, a)
    assert math.isclose(pm.t_mvm(n, nzr4, a, ratio * 1e9), 10 * pm.t_pci(n, 1e9), rel_tol=1e-12)


def test_storage_closed_forms():
    assert pm.one_full_row_pjds_entries(64, 32) == 33 * 64 - 32
    assert pm.ellpack_entries(64, 64) == 64 * 64
    assert pm.data_reduction(50, 100) == 0.5
