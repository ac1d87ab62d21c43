"""Exhaustive variant selection and regret — TEST INFRASTRUCTURE ONLY.

The paper observes that its runtime often picked a slower variant of matrix
multiply than the best one (Sec. 3.2: BLAS best at size 32 but OpenMP picked;
CUDA best for 64..4096 but OpenMP/BLAS picked).  The quality of a pick is
measured here against the plain rule "measure every variant and take the
fastest one that meets the accuracy asked":

* feasible(v)  <=>  err(v) <= tol
* best = the fastest feasible variant; variants whose time is within
  ``tie`` (relative) of the fastest are tied with it and the lowest id wins.
* regret(pick) = t(pick)/t(best) - 1 for a feasible pick (0 when the pick is
  tied with best); an infeasible pick costs a rerun with the best variant:
  (t(pick) + t(best))/t(best) - 1.
"""
import math

TIE = 0.02


def feasible(errs, tol):
    return {v for v, e in errs.items() if e is not None and e <= tol}


def exhaustive_pick(times, errs, tol, tie=TIE):
    """Best variant id, or None when no variant is feasible.

    times, errs: dicts variant_id -> median time / measured relative error.
    """
    ok = [v for v in sorted(feasible(errs, tol)) if v in times]
    if not ok:
        return None
    t_min = min(times[v] for v in ok)
    for v in ok:                       # ascending id: lowest tied id wins
        if times[v] <= t_min * (1.0 + tie):
            return v
    return None  # unreachable


def regret(pick, times, errs, tol, tie=TIE):
    """Regret of ``pick`` against the exhaustive choice (fraction, not %)."""
    best = exhaustive_pick(times, errs, tol, tie)
    if best is None:
        return math.nan
    t_best = min(times[v] for v in feasible(errs, tol) if v in times)
    if pick not in feasible(errs, tol):
        return (times[pick] + t_best) / t_best - 1.0
    if times[pick] <= t_best * (1.0 + tie):
        return 0.0
    return times[pick] / t_best - 1.0
