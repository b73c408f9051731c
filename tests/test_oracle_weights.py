"""Pins for the weight functions and the robust sigma (Sect. 5.1.2)."""
import json
import os

import numpy as np

from oracle import weights as WF

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "weights_printed.json")))


def test_printed_values():
    assert abs(WF.w_agis(10.0) - GOLD["w_agis"]["10"]) < 5e-4
    assert abs(WF.w_agis(100.0) / GOLD["w_agis"]["100"] - 1) < 0.2
    assert abs(WF.w_huber(10.0) - GOLD["w_huber_c2"]["10"]) < 5e-3
    assert abs(WF.w_huber(100.0) - GOLD["w_huber_c2"]["100"]) < 5e-5


def test_smooth_join_and_symmetry():
    z = GOLD["w_agis_join"]["z"]
    e = 1e-7
    assert abs(WF.w_agis(z - e) - WF.w_agis(z + e)) < 1e-6
    slope_l = (WF.w_agis(z - e) - WF.w_agis(z - 2 * e)) / e
    slope_r = (WF.w_agis(z + 2 * e) - WF.w_agis(z + e)) / e
    assert abs(slope_l - slope_r) < 1e-4
    assert abs(slope_r + np.exp(-1.0) / 3) < 1e-4
    assert WF.w_agis(2.0) == 1.0 and WF.w_agis(-1.5) == 1.0
    zz = np.linspace(-20, 20, 4001)
    assert np.allclose(WF.w_agis(zz), WF.w_agis(-zz))
    assert np.all(np.diff(WF.w_agis(zz[2000:])) <= 1e-15)


def test_intersextile_of_gaussian():
    # half the range between the 1/6 and 5/6 quantiles of N(0,1) is Phi^-1(5/6) = 0.96742...
    rng = np.random.default_rng(0)
    x = rng.normal(size=400_000)
    assert abs(WF.intersextile_half_range(x) - 0.9674216) < 0.01
    # type-7 definition on a small sample
    assert WF.intersextile_half_range(np.arange(7.0)) == 0.5 * (5.0 - 1.0)
