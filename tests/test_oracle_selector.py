"""Pins for exhaustive selection and regret on hand-made timing tables (CPU only)."""
import math

from oracle import selector_ref as S


def test_fastest_feasible_wins():
    times = {0: 5.0, 1: 2.0, 2: 1.0, 5: 1.5}
    errs = {0: 1e-7, 1: 1e-7, 2: 1e-4, 5: 3e-6}
    assert S.exhaustive_pick(times, errs, tol=1e-5) == 5        # 2 infeasible
    assert S.exhaustive_pick(times, errs, tol=1e-3) == 2


def test_ties_go_to_lowest_id():
    times = {1: 1.015, 3: 1.0, 5: 1.3}
    errs = {1: 0.0, 3: 0.0, 5: 0.0}
    assert S.exhaustive_pick(times, errs, tol=1e-5) == 1
    assert S.regret(3, times, errs, 1e-5) == 0.0
    assert S.regret(1, times, errs, 1e-5) == 0.0


def test_regret_values():
    times = {0: 4.0, 1: 2.0, 2: 1.0}
    errs = {0: 0.0, 1: 0.0, 2: 1.0}
    assert S.regret(1, times, errs, 1e-5) == 0.0
    assert S.regret(0, times, errs, 1e-5) == 1.0                 # 4/2 - 1
    assert S.regret(2, times, errs, 1e-5) == 0.5                 # (1+2)/2 - 1 infeasible


def test_no_feasible_variant():
    assert S.exhaustive_pick({0: 1.0}, {0: 1.0}, tol=1e-5) is None
    assert math.isnan(S.regret(0, {0: 1.0}, {0: 1.0}, 1e-5))
