"""Pins the instruction-roofline arithmetic (Sec. 2.2) to the numbers the paper
prints in Table 2 and Table 1 (fixture: tests/golden/paper_hardware.txt)."""
import os

import pytest

from paper_2608_13696_gb300 import roofline as rf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_hardware.txt")


def _rows():
    gpus, sfs = {}, {}
    for line in open(GOLD):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0].startswith("SF"):
            sfs[line[0]] = tuple(float(x) for x in line[1:])
        else:
            gpus[line[0]] = tuple(float(x) for x in line[1:])
    return gpus, sfs


GPUS, SFS = _rows()


@pytest.mark.parametrize("gpu", ["L4", "GH200"])
def test_throughput_from_sms_smsp_clock(gpu):
    n_sm, smsp, clk, inst, _, _ = GPUS[gpu]
    got = rf.inst_throughput(int(n_sm), int(smsp), clk * 1e9) / 1e9
    # the printed clock has two decimals: +-0.005 GHz x N_SM x N_SMSP
    assert abs(got - inst) <= 0.005 * n_sm * smsp + 0.5


@pytest.mark.parametrize("gpu", ["L4", "GH200"])
def test_ridge_matches_table2(gpu):
    n_sm, smsp, clk, inst, bw, ridge = GPUS[gpu]
    # throughput and ridge are both printed rounded (to 1 G inst/s and 0.1);
    # from the printed throughput the ridge lands within that rounding
    assert abs(rf.ridge(inst * 1e9, bw * 1e9) - ridge) <= 0.06
    if gpu == "L4":  # from the unrounded 58 x 4 x 1.78 GHz it rounds exactly
        assert round(rf.ridge(rf.inst_throughput(58, 4, 1.78e9), bw * 1e9), 1) == ridge


def test_ratios_of_table2():
    l4, gh = GPUS["L4"], GPUS["GH200"]
    assert round(gh[3] / l4[3], 2) == 2.51
    assert round(gh[4] / l4[4], 2) == 13.41  # printed as 13.42 / 13.4x
    assert round(gh[5] / l4[5], 2) == 0.19
    # "5.3x fewer instructions per memory access" at the ridge
    assert round(rf.ridge(l4[3], l4[4]) / rf.ridge(gh[3], gh[4]), 1) == 5.3


def test_table1_speedups():
    for sf, (l4, gh, printed) in SFS.items():
        r = l4 / gh
        # SF1 prints 2.4 for 84/34 = 2.47: a truncation, not a rounding
        assert int(r * 10) / 10 == printed or round(r, 1) == printed, sf


def test_bound_classification_and_roof():
    ridge = rf.ridge(1037e9, 4022e9)
    assert rf.bound(ridge * 0.9, ridge) == "memory"
    assert rf.bound(ridge * 1.1, ridge) == "compute"
    assert rf.attainable(ridge, 1037e9, 4022e9) == pytest.approx(1037e9)
    assert rf.attainable(ridge / 2, 1037e9, 4022e9) == pytest.approx(1037e9 / 2)
    assert rf.intensity(64, 32 * 8) == 8.0


def test_full_wave():
    assert rf.full_wave(152, 1, 152) and not rf.full_wave(151, 1, 152)
    assert not rf.full_wave(152, 2, 152)
