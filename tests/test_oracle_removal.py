"""Pins of the oracle's star collisions and ejections (Sec. 2.1.2: mce_cent,
and bodies beyond 400 au removed every 200 yr).

References that stand without the oracle: the closest approach of a Kepler
orbit over an interval from the orbit's geometry (the pericentre is where
the true anomaly passes a multiple of 2 pi; the end state from the
high-precision two-body propagation), where the oracle reads the mean
anomaly; mass conservation; the frame of a merged star (the other bodies'
barycentric velocities unchanged, their heliocentric positions moved by the
new star's offset); the removal interval.
"""
import math

import numpy as np
import pytest

import oracle
import opal_ic as ic
from kepler_reference import propagate

DT = 0.01 * ic.YEAR


def _true_anomaly(mu, x, v):
    """True anomaly from the orbit's geometry: the angle from the eccentricity
    vector to x, measured in the direction of motion."""
    h = np.cross(x, v)
    evec = np.cross(v, h) / mu - x / np.linalg.norm(x)
    f = math.atan2(np.linalg.norm(h) * (x @ v) / mu, (h @ h) / mu - np.linalg.norm(x))
    return f, np.linalg.norm(evec)


def _closed_form_min_r(mu, dt, x0, v0):
    """min over [0, dt] of |x(t)|: the pericentre (true anomaly 0) is passed
    when the swept true anomaly covers a multiple of 2 pi (any step of a period
    or more on an ellipse); the end state comes from the independent
    high-precision two-body propagation."""
    x1, v1 = (np.array(t, float) for t in propagate(mu, dt, x0, v0))
    r0, r1 = np.linalg.norm(x0), np.linalg.norm(x1)
    f0, e = _true_anomaly(mu, x0, v0)
    f1, _ = _true_anomaly(mu, x1, v1)
    h = np.cross(x0, v0)
    q = (h @ h) / mu / (1.0 + e)
    a = 1.0 / (2.0 / r0 - v0 @ v0 / mu)
    if a > 0 and abs(dt) >= 2 * math.pi * math.sqrt(a ** 3 / mu):
        passed = True
    elif a > 0:
        # the anomaly advances by less than 2 pi in the direction of time
        if dt > 0:
            swept = (f1 - f0) % (2 * math.pi)
            passed = f0 % (2 * math.pi) + swept >= 2 * math.pi
        else:
            swept = (f0 - f1) % (2 * math.pi)
            passed = (f0 % (2 * math.pi)) - swept <= 0.0
    else:
        passed = min(f0, f1) <= 0.0 <= max(f0, f1)
    return (min(r0, r1, q) if passed else min(r0, r1)), x1, v1


@pytest.mark.parametrize("seed", range(6))
def test_drift_closest_approach_matches_the_anomaly_closed_form(seed):
    rng = np.random.default_rng(seed)
    for _ in range(8):
        if rng.uniform() < 0.25:
            a, e = -rng.uniform(0.5, 3.0), rng.uniform(1.05, 3.0)
            f = rng.uniform(-0.7, 0.7) * math.acos(-1.0 / e)
        else:
            a, e, f = rng.uniform(0.3, 5.0), rng.uniform(0.0, 0.97), rng.uniform(0, 2 * math.pi)
        x0, v0 = ic.elements_to_state(1.0, a, e, rng.uniform(0, 1), rng.uniform(0, 6), rng.uniform(0, 6), f)
        dt = rng.choice([1, -1]) * rng.uniform(0.02, 30.0)
        ref, x1, v1 = _closed_form_min_r(1.0, dt, x0, v0)
        got = oracle.drift_min_r(1.0, dt, x0, v0, x1, v1)
        assert abs(got - ref) <= 1e-10 * ref, (a, e, dt, got, ref)


def _plunge(q, r_start=0.5, mu=1.0):
    """A body at r_start falling towards pericentre q on an orbit of e = 0.99."""
    e = 0.99
    a = q / (1.0 - e)
    cosf = (a * (1 - e * e) / r_start - 1.0) / e
    f = -math.acos(max(-1.0, min(1.0, cosf)))            # inbound
    return ic.elements_to_state(mu, a, e, 0.1, 0.2, 0.3, f)


def test_a_body_whose_drift_passes_within_the_star_is_accreted():
    mp = 1e-3
    xp, vp = ic.elements_to_state(1.0 + mp, 1.5, 0.02, 0.0, 0.0, 0.0, 1.0)
    mb = 2e-6
    xb, vb = _plunge(q=0.002)
    m = np.array([mp, mb])
    x, v, R = np.array([xp, xb]), np.array([vp, vb]), np.array([1e-4, 1e-5])
    # step until the plunging body reaches pericentre
    ref = oracle.Sim(m, x, v, R, dt=DT)
    acc = oracle.Sim(m, x, v, R, dt=DT, r_star=0.005)
    for _ in range(400):
        assert ref.step(1) == oracle.OK
        assert acc.step(1) == oracle.OK
        if acc.stats.n_accreted:
            break
    assert acc.stats.n_accreted == 1 and acc.alive.tolist() == [1, 0]
    # mass conserved exactly, momentum by the frame change
    assert acc.M0 == 1.0 + mb
    assert acc.m[0] == mp and acc.m[1] == 0.0
    # the planet: same barycentric velocity, position moved by the new star's offset
    Xc = mb * ref.x[1] / (1.0 + mb)
    assert np.array_equal(acc.V[0], ref.V[0])
    assert np.allclose(acc.x[0], ref.x[0] - Xc, rtol=0, atol=1e-15 * np.linalg.norm(ref.x[0]))
    # the bookkeeping: E + E_lost is the energy of the step without the accretion
    E_ref = ref.energy()[0]
    E_acc, _, _, El = acc.energy()
    assert abs(E_acc + El - E_ref) <= 1e-13 * abs(E_ref)
    # and the run goes on, with the accelerations evaluated afresh
    assert acc.step(10) == oracle.OK and acc.stats.n_accreted == 0


def test_a_near_miss_is_not_accreted():
    xb, vb = _plunge(q=0.0056)
    sim = oracle.Sim(np.array([2e-6]), xb[None], vb[None], np.array([1e-5]), dt=DT, r_star=0.005)
    for _ in range(300):
        assert sim.step(1) == oracle.OK
        assert sim.stats.n_accreted == 0
    assert sim.alive.tolist() == [1]


def test_ejection_happens_at_the_first_check_beyond_the_distance():
    mp = 1e-3
    xp, vp = ic.elements_to_state(1.0 + mp, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    xe = np.array([3.0, 0.0, 0.0])
    ve = np.array([0.0, 1.2, 0.0])                       # above escape speed at 3 au
    m = np.array([mp, 1e-6])
    every = 25
    sim = oracle.Sim(m, np.array([xp, xe]), np.array([vp, ve]), np.array([1e-4, 1e-5]), dt=DT,
                     r_eject=5.0, eject_every=every)
    ref = oracle.Sim(m, np.array([xp, xe]), np.array([vp, ve]), np.array([1e-4, 1e-5]), dt=DT)
    crossed = None
    for k in range(1, 400):
        assert sim.step(1) == oracle.OK and ref.step(1) == oracle.OK
        r = np.linalg.norm(ref.x[1])
        if crossed is None and r > 5.0:
            crossed = k
        if sim.stats.n_ejected:
            break
    assert crossed is not None
    # removed at the first multiple of the interval at or after the crossing
    assert k == every * math.ceil(crossed / every)
    assert sim.alive.tolist() == [1, 0] and sim.m[1] == 0.0
    assert sim.M0 == 1.0                                  # an ejection does not change the star
    E, _, _, El = sim.energy()
    assert abs(E + El - ref.energy()[0]) <= 1e-13 * abs(E)
