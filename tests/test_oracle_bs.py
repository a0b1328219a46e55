"""Pins of the oracle's Bulirsch-Stoer encounter integration and mergers.

References: the two-body closed form (tests/kepler_reference.py), scipy's
DOP853 on the same equations at tight tolerance, and conservation laws.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle
import opal_ic as ic
from kepler_reference import propagate


def _group(x, V, m, R, rc):
    n = len(m)
    return (np.arange(n, dtype=np.int32), np.ascontiguousarray(m, float).copy(),
            np.ascontiguousarray(R, float).copy(), np.ascontiguousarray(rc, float).copy(),
            np.ones(n, np.int32), np.ascontiguousarray(x, float).copy(), np.ascontiguousarray(V, float).copy())


@pytest.mark.parametrize("e,dt", [(0.05, 0.0628), (0.22, 0.3), (0.6, 0.5)])
def test_single_body_bs_equals_kepler(e, dt):
    x, v = ic.elements_to_state(1.0, 1.2, e, 0.1, 0.2, 0.3, 2.0)
    p = oracle.make_params(dt=dt)
    mem, m, R, rc, alive, X, V = _group(x[None], v[None], [1e-9], [1e-9], [1e-9])
    st, El, nm, sub = oracle.bs_group(p, mem, m, R, rc, alive, X, V)
    assert st == oracle.OK
    xr, vr = propagate(1.0, dt, x, v)
    assert np.linalg.norm(X[0] - xr) <= 5e-11 * np.linalg.norm(xr)
    assert np.linalg.norm(V[0] - vr) <= 5e-11 * np.linalg.norm(vr)


def test_separated_members_follow_their_kepler_orbits():
    """Members farther apart than rc feel no (1 - K) force: each is a Kepler orbit."""
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.1, 0.0, 0.0, 0.0, 0.0)
    x2, v2 = ic.elements_to_state(1.0, 1.5, 0.1, 0.0, 0.0, 0.0, 1.0)
    p = oracle.make_params(dt=0.2)
    mem, m, R, rc, alive, X, V = _group(np.array([x1, x2]), np.array([v1, v2]), [1e-5, 1e-5], [1e-6, 1e-6],
                                        [0.01, 0.01])
    st, *_ = oracle.bs_group(p, mem, m, R, rc, alive, X, V)
    assert st == oracle.OK
    for k, (x, v) in enumerate([(x1, v1), (x2, v2)]):
        xr, vr = propagate(1.0, 0.2, x, v)
        assert np.linalg.norm(X[k] - xr) <= 5e-11 * np.linalg.norm(xr)


def _encounter_pair():
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.02, 0.0, 0.0, 0.0, 0.0)
    x2 = x1 + np.array([0.0, 0.004, 0.0002])
    v2 = v1 + np.array([0.01, -0.02, 0.0])
    return np.array([x1, x2]), np.array([v1, v2]), np.array([3e-6, 2e-6])


def _full_ode(m, G=1.0, M0=1.0):
    def f(t, y):
        X = y[:6].reshape(2, 3)
        V = y[6:].reshape(2, 3)
        A = np.empty((2, 3))
        d = X[1] - X[0]
        r = np.linalg.norm(d)
        for b in range(2):
            A[b] = -G * M0 * X[b] / np.linalg.norm(X[b]) ** 3
        A[0] += G * m[1] * d / r ** 3
        A[1] -= G * m[0] * d / r ** 3
        return np.concatenate([V.ravel(), A.ravel()])
    return f


def test_encounter_matches_independent_integrator_and_conserves_energy():
    X0, V0, mass = _encounter_pair()
    dt = 0.0628
    # rc so large that the pair stays inside 0.1 rc: 1 - K = 1, the full mutual force
    p = oracle.make_params(dt=dt)
    mem, m, R, rc, alive, X, V = _group(X0, V0, mass, [1e-8, 1e-8], [1.0, 1.0])
    st, El, nmg, sub = oracle.bs_group(p, mem, m, R, rc, alive, X, V)
    assert st == oracle.OK and nmg == 0
    sol = solve_ivp(_full_ode(mass), (0, dt), np.concatenate([X0.ravel(), V0.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-16)
    yr = sol.y[:, -1]
    assert np.abs(X.ravel() - yr[:6]).max() <= 1e-10
    assert np.abs(V.ravel() - yr[6:]).max() <= 1e-9

    def HA(X, V):
        e = sum(0.5 * mass[b] * V[b] @ V[b] - mass[b] / np.linalg.norm(X[b]) for b in range(2))
        return e - mass[0] * mass[1] / np.linalg.norm(X[1] - X[0])
    assert abs(HA(X, V) - HA(X0, V0)) <= 1e-10 * abs(HA(X0, V0))


def test_merger_conserves_mass_momentum_and_reports_energy_loss():
    X0, V0, mass = _encounter_pair()
    V0 = V0.copy()
    V0[1] = V0[0] + np.array([0.0, -0.08, -0.004])   # head-on towards body 0
    dt = 0.0628
    R = np.array([3e-4, 2e-4])
    p = oracle.make_params(dt=dt)
    mem, m, Rg, rc, alive, X, V = _group(X0, V0, mass, R, [1.0, 1.0])
    st, El, nmg, sub = oracle.bs_group(p, mem, m, Rg, rc, alive, X, V)
    assert st == oracle.OK
    assert nmg == 1
    assert alive.tolist() == [1, 0]                 # heavier body survives
    assert m[0] == mass.sum() and m[1] == 0.0
    assert abs(Rg[0] - np.cbrt(R[0] ** 3 + R[1] ** 3)) <= 1e-18
    assert El > 0


def test_merger_bookkeeping_at_contact():
    """Merge two bodies already in contact: exact conservation of mass, momentum and centre of mass."""
    x = np.array([[1.0, 0.0, 0.0], [1.0, 1e-4, 0.0]])
    v = np.array([[0.0, 1.0, 0.0], [0.001, 1.0, 0.0]])
    mass = np.array([2e-6, 2e-6])   # tie: the lower index survives
    p = oracle.make_params(dt=1e-6)
    mem, m, R, rc, alive, X, V = _group(x, v, mass, [1e-4, 1e-4], [1.0, 1.0])
    st, El, nmg, sub = oracle.bs_group(p, mem, m, R, rc, alive, X, V)
    assert st == oracle.OK and nmg == 1 and alive.tolist() == [1, 0]
    # after the single tiny substep the pair merged; compare with the merged
    # state of the substep's end computed from the unmerged flow over 1e-6
    # momentum changes only by the star's pull over the substep (mutual forces cancel)
    P1 = (mass[:, None] * v).sum(0) - 1e-6 * (mass[:, None] * x / np.linalg.norm(x, axis=1)[:, None] ** 3).sum(0)
    assert np.abs(m[0] * V[0] - P1).max() <= 1e-16
    cm0 = (mass[:, None] * x).sum(0) / mass.sum()
    assert np.abs(X[0] - cm0).max() <= 2e-6
    # energy lost by the perfect merger = relative kinetic + mutual potential (+ central change)
    mu_red = mass[0] * mass[1] / mass.sum()
    approx = 0.5 * mu_red * 0.001 ** 2 - mass[0] * mass[1] / 1e-4
    assert abs(El - approx) <= 1e-6 * abs(approx)


def test_bs_substep_cap_reports_failure():
    X0, V0, mass = _encounter_pair()
    p = oracle.make_params(dt=2.0, bs_max_substeps=1)
    mem, m, R, rc, alive, X, V = _group(X0, V0, mass, [1e-8, 1e-8], [1.0, 1.0])
    st, El, nmg, sub = oracle.bs_group(p, mem, m, R, rc, alive, X, V)
    assert st == oracle.EBS
    assert np.array_equal(X, X0) and np.array_equal(V, V0)
