"""The learning-rate and SR-shift schedules (supplement, "Learning Rate Scheduling"): the oracle's
formula against its closed-form points, and the library's host function against the oracle."""
import numpy as np
import pytest

from oracle import estimators as E


def test_oracle_schedule_closed_form_points():
    eta0, isw, idc, a = 0.0061, 30000, 40000, 0.001
    assert E.lr_schedule(0) == eta0 and E.lr_schedule(isw - 1) == eta0
    assert E.lr_schedule(isw) == pytest.approx(eta0 + a * eta0, rel=1e-15)             # cos 0 = 1
    assert E.lr_schedule(isw + idc // 2) == pytest.approx(eta0 / 2 + a * eta0, rel=1e-12)   # cos(pi/2) = 0
    assert E.lr_schedule(isw + idc) == pytest.approx(a * eta0, rel=1e-9)                # cos pi = -1


def test_library_schedule_matches_oracle():
    from paper_2502_20723_gb300 import build, tdo
    build.build()
    steps = [0, 1, 29999, 30000, 30001, 41234, 50000, 69999, 70000, 90000]
    for st in steps:
        assert tdo.schedule_value(st, 0.0061, 30000, 40000, 0.001) == pytest.approx(E.lr_schedule(st), rel=1e-14)
        ref_sr = E.lr_schedule(st, eta0=0.004, i_switch=30000, i_decay=40000, alpha=0.01)
        assert tdo.schedule_value(st, 0.004, 30000, 40000, 0.01) == pytest.approx(ref_sr, rel=1e-14)
    s = tdo.Schedule()
    assert (s.eta0, s.i_switch, s.i_decay, s.alpha, s.lambda0, s.alpha_sr) == (0.0061, 30000, 40000, 0.001, 0.004, 0.01)
