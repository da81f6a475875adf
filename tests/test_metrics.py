"""Host-side benchmark accounting: the product's closed-form flop model agrees
with the oracle's matrix-based count, and the penalty reproduces the paper's
printed validation ratio."""

import json
import os

import pytest

from oracle import hpg_oracle as O
from paper_2507_11512_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.mark.parametrize("dims,levels", [((16, 16, 16), 4), ((12, 12, 12), 4), ((8, 6, 4), 3),
                                         ((5, 7, 3), 4), ((32, 16, 8), 4)])
def test_flop_model_matches_oracle_count(dims, levels):
    lv = O.build_hierarchy(*dims, levels=levels)
    dl = metrics.level_dims(dims, levels)
    assert dl == [l.dims for l in lv]
    for l, L in enumerate(lv):
        assert metrics.nnz(L.dims) == L.A.nnz
        if L.fc is not None:
            assert metrics.coarse_point_nnz(L.dims) == L.A[L.fc].nnz
    for cyc in ([3], [30, 30, 7], [1]):
        assert metrics.solve_flops(dl, cyc) == O.solve_flops(lv, cyc)
        assert metrics.vcycle_flops(dl) == O.vcycle_flops(lv)


def test_cycles_from_info():
    assert metrics.cycles_from_info(67, 3, 30) == [30, 30, 7]
    assert metrics.cycles_from_info(30, 1, 30) == [30]
    assert metrics.cycles_from_info(0, 0, 30) == []


def test_penalty_reproduces_paper_ratio():
    g = json.load(open(GOLDEN))["validation"]
    assert round(metrics.penalty(g["n_d"], g["n_ir"]), 3) == g["standard_ratio"]
    assert metrics.penalty(2400, 2382) == 1.0   # faster MxP is not rewarded (Sec. 3)


def test_fullscale_table_ratios_are_consistent():
    # Table 2: ratios above 1 are not applied as a bonus
    rows = json.load(open(GOLDEN))["fullscale_table"]["rows"]
    for r in rows:
        assert metrics.penalty(r["fullscale_ratio"], 1.0) == min(1.0, r["fullscale_ratio"])


def test_gs_row_bytes_fp32_and_fp64():
    # 27 values + 26 int32 indices + r_i, z_i written, z_j gathered
    assert metrics.gs_row_bytes(4, 4) == 27 * 4 + 26 * 4 + 12 == 224
    assert metrics.gs_row_bytes(8, 8) == 27 * 8 + 26 * 4 + 24 == 344
