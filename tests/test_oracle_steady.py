"""Pins of the oracle's steady-state criterion of Sec. 3.2 (porous flow).

* The physical time step of the paper's units reproduces the two time steps
  the paper prints for the ends of its streaming-distance range (MLBM1,
  tau = 1, nu = 1, side length 1): dx = 2e-3 -> dt = 6.67e-7, dx = 1.5e-4 ->
  dt = 3.75e-9.
* On a mean velocity that approaches its limit exponentially,
  <u>(t) = U (1 - exp(-t/T)), the criterion can be solved in closed form:
  with b = exp(-(t - dn)/T) and c = (1 - exp(-dn/T)) / (dt dn),
  Delta u = b c / (1 - b) < thr  <=>  t > dn + T ln((c + thr) / thr),
  so the first recorded step is the first multiple of `check` above that
  bound (and >= dn).  The same from above, <u> = U (1 + exp(-t/T)), with
  Delta u = b c / (1 + b).  A constant record is steady at t = dn; a record
  that starts from rest is never steady against the zero mean.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_paper_time_steps():
    # the printed values of Sec. 3.2, to the digits printed
    assert abs(O.paper_time_step(1.0, 2e-3, 1.0) / 6.67e-7 - 1) < 1e-3
    assert abs(O.paper_time_step(1.0, 1.5e-4, 1.0) / 3.75e-9 - 1) < 1e-12
    # scale-free: s and the side in any common unit
    assert O.paper_time_step(1.0, 1.0, 500.0) == pytest.approx(O.paper_time_step(1.0, 2e-3, 1.0), rel=1e-14)


def _closed_form_step(T, dn, dt, thr, check, above=False):
    c = (1.0 - math.exp(-dn / T)) / (dt * dn)
    if above:
        # b c / (1 + b) < thr  <=>  b (c - thr) < thr
        if c <= thr:
            return dn
        bound = dn + T * math.log((c - thr) / thr)
    else:
        bound = dn + T * math.log((c + thr) / thr)
    t = max(dn, (math.floor(bound / check) + 1) * check)
    return t


@pytest.mark.parametrize("T,dn,check,dt,thr", [
    (3000.0, 2000, 100, 1e-4, 1e-2),
    (1234.5, 1000, 10, 5e-4, 3e-2),
    (20000.0, 20000, 1000, 6.67e-7 * 1.0, 1e-2 * 300),
    (777.0, 300, 1, 1e-3, 1e-1),
])
def test_exponential_approach_closed_form(T, dn, check, dt, thr):
    t = np.arange(0, 60 * T + 2 * dn, check, dtype=np.float64)
    up = 0.37 * (1.0 - np.exp(-t / T))
    assert O.steady_mean_step(up, check, dn, dt, thr) == _closed_form_step(T, dn, dt, thr, check)
    down = 0.37 * (1.0 + np.exp(-t / T))
    assert O.steady_mean_step(down, check, dn, dt, thr) == _closed_form_step(T, dn, dt, thr, check, above=True)
    # a negative flow (g along -x) is the same criterion
    assert O.steady_mean_step(-up, check, dn, dt, thr) == _closed_form_step(T, dn, dt, thr, check)


def test_special_records():
    assert O.steady_mean_step(np.full(50, 0.2), 10, 100, 1.0, 1e-6) == 100
    # from rest, compared at t = dn with <u>(0) = 0: not steady there
    r = np.array([0.0, 1.0, 1.0, 1.0])
    assert O.steady_mean_step(r, 10, 10, 1.0, 1e-3) == 20
    assert O.steady_mean_step(np.zeros(10), 10, 10, 1.0, 1.0) == -1
    assert O.steady_mean_step(np.linspace(0.1, 1.0, 20), 5, 10, 1.0, 1e-9) == -1
    with pytest.raises(ValueError):
        O.steady_mean_step(np.ones(4), 3, 10, 1.0, 1.0)
