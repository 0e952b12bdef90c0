"""Pins of the Section III models (Eqs. 2-5) used by the tuner and the bench."""
import os

import pytest

from paper_1410_5561_gb300 import model

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cache_model_example.txt")


def _golden():
    vals = {}
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    return vals


def test_worked_example_eq2():
    g = _golden()
    assert model.wavefront_width(g["D_w"], g["N_F"], g["R"]) == g["W_w"]
    assert model.cache_block_bytes_r1(g["D_w"], g["N_F"], 1, g["N_D"]) == g["C_S_per_N_xb"]
    assert model.cache_block_bytes(g["D_w"], g["N_F"], 1, g["N_D"], g["R"]) == g["C_S_per_N_xb"]


@pytest.mark.parametrize("dw", [4, 8, 12, 16, 20, 32, 64])
@pytest.mark.parametrize("nf", [1, 2, 4, 10])
@pytest.mark.parametrize("nd", [2, 9, 15])
def test_eq3_reduces_to_eq2(dw, nf, nd):
    assert model.cache_block_bytes(dw, nf, 7, nd, 1) == pytest.approx(model.cache_block_bytes_r1(dw, nf, 7, nd))


def test_code_balance_forms_agree():
    for r in (1, 4):
        for dw in (8, 16, 32, 64):
            if dw % (2 * r):
                continue
            for nc in (0, 7, 13):
                assert model.code_balance(dw, r, 8, nc, 8) == pytest.approx(model.code_balance_dp(dw, 2 + nc, r))


def test_code_balance_closed_form():
    # 2R(4 s_f + n_c s_c)/D_w: the (2D_w - 2R) writes and the 2R extra reads cancel
    for (r, sf, nc, sc) in [(1, 4, 0, 4), (1, 8, 7, 8), (1, 4, 7, 2), (4, 4, 13, 4)]:
        for dw in (8, 16, 32):
            assert model.code_balance(dw, r, sf, nc, sc) == pytest.approx(2 * r * (4 * sf + nc * sc) / dw)


def test_plain_and_example_values():
    assert model.bytes_per_lup("7pt_const", "f32", None, "plain") == 8
    assert model.bytes_per_lup("7pt_var", "f32", "bf16", "plain") == 22
    assert model.bytes_per_lup("25pt_var", "f32", None, "plain") == 60
    assert model.bytes_per_lup("7pt_const", "f32", None, "blocked", 16) == 2
    assert model.bytes_per_lup("7pt_var", "f64", None, "blocked", 16) == 11
    assert model.bytes_per_lup("25pt_var", "f32", None, "blocked", 32) == 17
    # the paper's DP 7-point constant case: D_w = 8 gives 64/8 = 8 bytes per LUP
    assert model.code_balance_dp(8, 2) == 8
    assert model.diamond_levels(16, 1) == 15 and model.diamond_levels(32, 4) == 7
