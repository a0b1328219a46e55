"""Pins of the oracle's small bodies (Sec. 2.1: only the big bodies are
gravity sources; small bodies are massless particles that feel the star and
the big bodies).

References that stand without the oracle: exact invariance of the big bodies
when no small body meets one; the exact Kepler orbit of a small body that
meets nothing big; the Jacobi integral of the circular restricted three-body
problem; brute-force minimum separations; the merger rule's closed forms.
"""
import numpy as np

import oracle
import opal_ic as ic
from kepler_reference import propagate
from test_oracle_scan import brute_force_flags

DT = 0.01 * ic.YEAR


def _small_ring(n, a_lo, a_hi, seed=5, R=1e-6):
    """n massless bodies on near-circular, slightly inclined orbits."""
    s = ic.Stream(seed, 20)
    u = s.take(4 * n).reshape(n, 4)
    a = a_lo + (a_hi - a_lo) * u[:, 0]
    x, v = ic.elements_to_state(1.0, a, 0.02 * u[:, 1], 0.01 * u[:, 2], 0.0, 0.0, ic.TWOPI * u[:, 3])
    return np.zeros(n), x, v, np.full(n, R)


def _join(big, small):
    return tuple(np.concatenate([b, s]) for b, s in zip(big, small))


def test_big_bodies_are_blind_to_small_ones_that_meet_none():
    """With every small body far from the big ones, the big bodies' states are
    the same bits with and without them: a small body adds nothing to any
    force, momentum or encounter of a big one."""
    t = ic.tiny(seed=3, n=10)
    big = (t.m, t.x, t.v, t.R)
    small = _small_ring(40, 4.0, 6.0)
    a = oracle.Sim(*big, dt=DT)
    b = oracle.Sim(*_join(big, small), dt=DT)
    for _ in range(10):
        assert a.step(20) == oracle.OK and b.step(20) == oracle.OK
        assert np.array_equal(a.x, b.x[:10]) and np.array_equal(a.V, b.V[:10])
    assert b.alive.all()


def test_small_bodies_never_interact_with_each_other():
    """Two small bodies that pass through one another are not flagged, not
    merged, and each follows its exact Kepler orbit."""
    x1, v1 = ic.elements_to_state(1.0, 1.3, 0.1, 0.05, 0.3, 0.2, 1.0)
    v2 = v1 * np.array([1.01, 0.98, -1.0])          # same place, other velocity
    m = np.zeros(2)
    sim = oracle.Sim(m, np.array([x1, x1]), np.array([v1, v2]), np.full(2, 1e-3), dt=DT)
    assert sim.step(50) == oracle.OK
    assert sim.alive.tolist() == [1, 1]
    assert sim.stats.n_pairs == 0
    for k, v in enumerate((v1, v2)):
        xr, _ = propagate(1.0, 50 * DT, x1, v)
        assert np.linalg.norm(sim.x[k] - xr) <= 1e-12 * np.linalg.norm(xr)


def test_scan_skips_only_pairs_of_two_small_bodies():
    """The flagged set is brute force's minus the pairs of two small bodies;
    a small-big pair is flagged at the big body's critical radius."""
    for seed in range(4):
        s = ic.random_cluster(seed=seed, n=12, spread=0.015, vspread=0.05)
        m = s.m.copy()
        m[6:] = 0.0                                     # six small bodies
        M0, dt = 1.0, 0.05
        V0 = oracle.helio_to_dh(M0, m, s.v)
        x0 = s.x.copy()
        x1, V1 = x0.copy(), V0.copy()
        for i in range(s.n):
            st, x1[i], V1[i], _ = oracle.kepler_drift(1.0, dt, x0[i], V0[i])
            assert st == oracle.OK
        rc = oracle.hill_rcrit(M0, 2.0, m, x1)
        assert (rc[6:] == 0).all() and (rc[:6] > 0).all()
        alive = np.ones(s.n, np.int32)
        pi, pj, _ = oracle.scan(dt, x0, V0, x1, V1, rc, alive, m=m)
        got = set(zip(pi.tolist(), pj.tolist()))
        # brute force with every small body given a tiny radius: two small ones
        # then flag only when their paths cross, which must not happen either
        ref, margins = brute_force_flags(dt, x0, V0, x1, V1, np.where(m > 0, rc, 1e-30), alive)
        ref = {p for p in ref if m[p[0]] > 0 or m[p[1]] > 0}
        assert not {p for p in got ^ ref if margins[p] > 1e-6}
        assert any(m[i] > 0 and m[j] == 0 for i, j in got), "no small-big pair in the test"
        assert all(m[i] > 0 or m[j] > 0 for i, j in got)


def _jacobi(sim, k, n_rot, mJ, jup=0):
    """Jacobi integral of small body k in the restricted three-body problem:
    J = |V|^2 / 2 - M0/|x| - mJ/|x - xJ| - n (X x V)_z, with V the barycentric
    velocity (the democratic heliocentric V), X the barycentric position and
    n the rate at which the primaries turn."""
    x, V = sim.x[k], sim.V[k]
    X = x - mJ * sim.x[jup] / (1.0 + mJ)
    return (0.5 * V @ V - 1.0 / np.linalg.norm(x) - mJ / np.linalg.norm(x - sim.x[jup])
            - n_rot * (X[0] * V[1] - X[1] * V[0]))


def test_small_bodies_keep_their_jacobi_integral():
    """A Jupiter-mass planet on a circular orbit and massless bodies inside
    its orbit: each small body's Jacobi integral stays constant to the
    integrator's error, while ignoring the planet would change it by far more."""
    mJ, aJ = ic.M_JUP, 5.2
    xJ, vJ = ic.elements_to_state(1.0 + mJ, aJ, 0.0, 0.0, 0.0, 0.0, 0.0)
    n_rot = np.sqrt((1.0 + mJ) / aJ ** 3)
    small = _small_ring(6, 2.5, 3.2, seed=11)
    m, x, v, R = _join((np.array([mJ]), xJ[None], vJ[None], np.array([4.7e-4])), small)
    sim = oracle.Sim(m, x, v, R, dt=DT)
    J0 = np.array([_jacobi(sim, k, n_rot, mJ) for k in range(1, 7)])
    assert sim.step(1000) == oracle.OK
    assert sim.stats.n_pairs == 0
    J1 = np.array([_jacobi(sim, k, n_rot, mJ) for k in range(1, 7)])
    drift = np.abs(J1 / J0 - 1).max()
    # the same bodies on pure Kepler orbits (the planet ignored)
    ref = oracle.Sim(m, x, v, R, dt=DT)
    for k in range(1, 7):
        xr, vr = propagate(1.0, 1000 * DT, x[k], v[k])
        ref.x[k], ref.V[k] = np.array(xr, float), np.array(vr, float)
    ref.x[0], ref.V[0] = sim.x[0], sim.V[0]
    J_kep = np.array([_jacobi(ref, k, n_rot, mJ) for k in range(1, 7)])
    assert drift <= 1e-7
    assert np.abs(J_kep / J0 - 1).min() >= 1000 * drift


def test_small_body_merges_into_a_big_one():
    """A small body in contact with an embryo is absorbed: the embryo keeps
    its mass and (to rounding) its momentum, its radius grows by the small
    body's volume, and no energy is lost."""
    mb = 0.05 * ic.M_EARTH
    xb, vb = ic.elements_to_state(1.0 + mb, 1.0, 0.01, 0.0, 0.0, 0.0, 0.0)
    Rb, Rs = 3e-5, 1e-5
    xs = xb + np.array([0.0, 2e-5, 0.0])                 # inside Rb + Rs already
    vs = vb + np.array([1e-4, 0.0, 0.0])
    m = np.array([mb, 0.0])
    sim = oracle.Sim(m, np.array([xb, xs]), np.array([vb, vs]), np.array([Rb, Rs]), dt=DT)
    assert sim.step(1) == oracle.OK
    assert sim.alive.tolist() == [1, 0]
    assert sim.m[0] == mb and sim.m[1] == 0.0
    assert abs(sim.R[0] - np.cbrt(Rb ** 3 + Rs ** 3)) <= 4e-16 * sim.R[0]
    assert sim.stats.n_mergers == 1
    E, _, P, E_lost = sim.energy()
    assert abs(E_lost) <= 1e-14 * abs(E)
    # the embryo alone, integrated the same way, ends where the merged one does
    alone = oracle.Sim(np.array([mb]), xb[None], vb[None], np.array([Rb]), dt=DT)
    assert alone.step(1) == oracle.OK
    assert np.linalg.norm(sim.x[0] - alone.x[0]) <= 1e-11 * np.linalg.norm(alone.x[0])
    P_alone = alone.energy()[2]
    assert np.linalg.norm(P - P_alone) <= 1e-11 * np.linalg.norm(P_alone)
