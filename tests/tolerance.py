"""How the GPU reductions are judged against the exactly rounded reference.

The dot product and the norm are the points where the paper's lazily
evaluated expressions are finally summed (Section 2; xDOT in Section 5).  A
reduction's error is stated on two measures:

* relative to its own value, ``|got - exact| / |exact|`` -- the relative
  error of the result, the measure the tolerances are stated in: FP64
  reductions 1e-13, compensated FP32 reductions 1e-6;
* relative to the condition scale, ``|got - exact| / sum|x_i y_i|`` -- the
  quantity a summation error bound is proportional to (Higham, *Accuracy and
  Stability of Numerical Algorithms*, 2nd ed., Eq. 3.5).

The two coincide for sums of squares and same-sign terms.  For a dot
product whose terms cancel, the relative error of any accumulation in
working precision grows with the condition number
``cond = sum|x_i y_i| / |sum x_i y_i|``; no bound on it holds for every
input.  So the bound is asserted relative to the value whenever
``cond <= COND_LITERAL`` (every random-sign test input here: uniform data
of length n has cond of order 2.25 sqrt(n), a few 10^4 at n = 2^28), and
relative to the condition scale for the deliberately ill-conditioned rest.
"""
from __future__ import annotations

import math

import numpy as np

TOL = {np.float64: 1e-13, np.float32: 1e-6}
COND_LITERAL = 1e6


def errors(got: float, exact: float, scale: float) -> dict:
    """Error of a reduction on both measures, and the condition number."""
    err = abs(got - exact)
    if math.isnan(got) or math.isnan(exact):
        err = math.inf if math.isnan(got) != math.isnan(exact) else 0.0
    rel_value = err / abs(exact) if exact != 0 else (0.0 if err == 0 else math.inf)
    rel_scale = err / scale if scale > 0 else (0.0 if err == 0 else math.inf)
    cond = scale / abs(exact) if exact != 0 else (1.0 if scale == 0 else math.inf)
    return {"rel_value": rel_value, "rel_scale": rel_scale, "cond": cond}


def check(got: float, exact: float, scale: float, dt, what="", factor: float = 1.0) -> dict:
    """Asserts the tolerance of ``dt`` (times ``factor``) on the result's
    relative error when the sum is not ill-conditioned, else on the error
    relative to ``scale``; returns both measures."""
    e = errors(got, exact, scale)
    tol = TOL[dt] * factor
    if e["cond"] <= COND_LITERAL:
        assert e["rel_value"] <= tol, (what, "relative to the value", got, exact, e)
    else:
        assert e["rel_scale"] <= tol, (what, "relative to sum|x y| (ill-conditioned)", got, exact, e)
    return e


def check_dot(got: float, x, y, dt, what="", factor: float = 1.0) -> dict:
    from oracle import exact
    return check(got, exact.exact_dot(x, y), exact.abs_dot(x, y), dt, what, factor)
