"""Pins of the oracle's Keplerian drift (Sec. 3.1, third block) and Stumpff functions.

Each check compares against something other than the oracle's own formulas:
closed-form trigonometric/hyperbolic Stumpff functions in mpmath, and the
two-body solution by the eccentric-anomaly route (tests/kepler_reference.py).
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
import opal_ic as ic
from kepler_reference import propagate


def stumpff_closed(z):
    with mp.workdps(40):
        z = mp.mpf(z)
        if z > 0:
            s = mp.sqrt(z)
            return [mp.cos(s), mp.sin(s) / s, (1 - mp.cos(s)) / z, (s - mp.sin(s)) / s ** 3]
        if z < 0:
            s = mp.sqrt(-z)
            return [mp.cosh(s), mp.sinh(s) / s, (mp.cosh(s) - 1) / (-z), (mp.sinh(s) - s) / s ** 3]
        return [mp.mpf(1), mp.mpf(1), mp.mpf(1) / 2, mp.mpf(1) / 6]


@pytest.mark.parametrize("z", [0.0, 1e-9, -1e-9, 0.004, -0.004, 0.0999, 0.1001, 0.37, -0.37, 2.5,
                               -2.5, 9.0, -9.0, 30.0, -30.0, 60.0])
def test_stumpff_matches_closed_form(z):
    c = oracle.stumpff(z)
    ref = stumpff_closed(z)
    for k in range(4):
        scale = max(1.0, abs(float(ref[k])))
        assert abs(c[k] - float(ref[k])) <= 2e-14 * scale * (1 + abs(z)), (k, c[k], ref[k])


CASES = [
    # (a, e, true anomaly, dt)
    (1.0, 0.0, 0.3, 0.01 * ic.YEAR),
    (1.0, 0.0, 1.0, 1.7 * ic.YEAR),
    (1.0, 0.22, 0.0, 0.01 * ic.YEAR),
    (5.2, 0.22, 2.0, 0.01 * ic.YEAR),
    (1.0, 0.22, 4.0, -0.37),
    (1.0, 0.22, 1.0, 3.3 * ic.YEAR),
    (1.0, 0.9, 0.0, 0.01 * ic.YEAR),
    (1.0, 0.9, 3.1, 0.2),
    (1.0, 0.9, 0.5, 2.0 * ic.YEAR),
    (-1.0, 1.5, 0.3, 0.5),
    (-2.0, 3.0, -0.4, 4.0),
]


@pytest.mark.parametrize("a,e,f,dt", CASES)
def test_drift_matches_two_body_closed_form(a, e, f, dt):
    mu = 1.0
    x, v = ic.elements_to_state(mu, a, e, 0.3, 0.7, 1.1, f)
    st, x1, v1, it = oracle.kepler_drift(mu, dt, x, v)
    assert st == oracle.OK
    xr, vr = propagate(mu, dt, x, v)
    ex = np.linalg.norm(x1 - xr) / np.linalg.norm(xr)
    ev = np.linalg.norm(v1 - vr) / np.linalg.norm(vr)
    tol = 1e-13 if e < 0.5 else 2e-12
    assert ex <= tol and ev <= tol, (ex, ev, it)


def test_drift_conserves_energy_and_angular_momentum():
    rng = np.random.default_rng(5)
    for _ in range(50):
        a = rng.uniform(0.5, 5)
        e = rng.uniform(0, 0.8)
        x, v = ic.elements_to_state(1.0, a, e, rng.uniform(0, 1), rng.uniform(0, 6), rng.uniform(0, 6),
                                    rng.uniform(0, 6))
        dt = rng.uniform(-3, 3)
        st, x1, v1, _ = oracle.kepler_drift(1.0, dt, x, v)
        assert st == oracle.OK
        E0 = 0.5 * v @ v - 1 / np.linalg.norm(x)
        E1 = 0.5 * v1 @ v1 - 1 / np.linalg.norm(x1)
        L0, L1 = np.cross(x, v), np.cross(x1, v1)
        assert abs(E1 - E0) <= 1e-13 * abs(E0)
        assert np.linalg.norm(L1 - L0) <= 1e-13 * np.linalg.norm(L0)


def test_drift_is_time_reversible():
    x, v = ic.elements_to_state(1.0, 1.3, 0.3, 0.2, 0.1, 0.2, 0.9)
    _, x1, v1, _ = oracle.kepler_drift(1.0, 0.77, x, v)
    _, x2, v2, _ = oracle.kepler_drift(1.0, -0.77, x1, v1)
    assert np.linalg.norm(x2 - x) <= 1e-14 * np.linalg.norm(x)
    assert np.linalg.norm(v2 - v) <= 1e-14 * np.linalg.norm(v)


def test_drift_reports_nonconvergence_and_keeps_state():
    x, v = ic.elements_to_state(1.0, 1.0, 0.3, 0.0, 0.0, 0.0, 1.0)
    st, x1, v1, it = oracle.kepler_drift(1.0, 0.5, x, v, max_iter=1)
    assert st == oracle.EKEPLER
    assert np.array_equal(x1, x) and np.array_equal(v1, v)


def test_drift_iterations_are_few_for_small_steps():
    x, v = ic.elements_to_state(1.0, 1.0, 0.05, 0.0, 0.0, 0.0, 1.0)
    _, _, _, it = oracle.kepler_drift(1.0, 0.0628, x, v)
    assert it <= 5
