"""Pins of the oracle's kick forces, changeover, Hill radii, coordinates and energy.

References: brute force at 40 digits in mpmath, Newton's third law, the
symmetry of the changeover, closed forms of the two-body problem.
"""
import math

import mpmath as mp
import numpy as np
import pytest

import oracle
import opal_ic as ic


def brute_force_newton(G, m, x):
    """All-pairs Newtonian accelerations at 40 digits."""
    n = len(m)
    out = np.zeros((n, 3))
    with mp.workdps(40):
        X = [[mp.mpf(float(t)) for t in row] for row in x]
        M = [mp.mpf(float(t)) for t in m]
        for i in range(n):
            acc = [mp.mpf(0)] * 3
            for j in range(n):
                if j == i:
                    continue
                d = [X[j][k] - X[i][k] for k in range(3)]
                r = mp.sqrt(sum(t * t for t in d))
                for k in range(3):
                    acc[k] += G * M[j] * d[k] / r ** 3
            out[i] = [float(t) for t in acc]
    return out


@pytest.mark.parametrize("n,seed", [(2, 1), (5, 2), (16, 3)])
def test_accel_matches_brute_force_when_no_pair_is_close(n, seed):
    s = ic.tiny(seed=seed, n=n)
    rc = np.full(n, 1e-9)
    a = oracle.accel(1.0, s.m, s.x, rc)
    ref = brute_force_newton(1.0, s.m, s.x)
    err = np.abs(a - ref).max() / np.abs(ref).max()
    assert err <= 1e-15


def test_accel_applies_changeover_per_pair_with_max_rcrit():
    s = ic.random_cluster(seed=4, n=8, spread=0.01)
    rc = oracle.hill_rcrit(1.0, 30.0, s.m, s.x)   # large factor: many pairs inside rc
    a = oracle.accel(1.0, s.m, s.x, rc)
    n = s.n
    ref = np.zeros((n, 3))
    with mp.workdps(40):
        for i in range(n):
            for j in range(n):
                if i == j:
                    continue
                d = [mp.mpf(float(s.x[j, k])) - mp.mpf(float(s.x[i, k])) for k in range(3)]
                r = mp.sqrt(sum(t * t for t in d))
                K = oracle.changeover(float(r), max(rc[i], rc[j]))
                for k in range(3):
                    ref[i, k] += float(mp.mpf(float(s.m[j])) * K * d[k] / r ** 3)
    inside = sum(1 for i in range(n) for j in range(i + 1, n)
                 if np.linalg.norm(s.x[i] - s.x[j]) < max(rc[i], rc[j]))
    assert inside >= 3
    assert np.abs(a - ref).max() <= 1e-13 * np.abs(ref).max()


def test_kick_conserves_momentum_and_has_no_torque():
    s = ic.random_cluster(seed=7, n=12, spread=0.01)
    rc = oracle.hill_rcrit(1.0, 10.0, s.m, s.x)
    a = oracle.accel(1.0, s.m, s.x, rc)
    F = s.m[:, None] * a
    scale = np.abs(F).sum()
    assert np.abs(F.sum(axis=0)).max() <= 1e-15 * scale
    torque = np.cross(s.x, F).sum(axis=0)
    assert np.abs(torque).max() <= 1e-15 * scale * np.abs(s.x).max()


def test_dead_bodies_exert_and_feel_nothing():
    s = ic.tiny(seed=1, n=6)
    rc = np.full(6, 1e-9)
    alive = np.array([1, 1, 0, 1, 1, 1], np.int32)
    a = oracle.accel(1.0, s.m, s.x, rc, alive)
    keep = alive > 0
    ref = brute_force_newton(1.0, s.m[keep], s.x[keep])
    assert np.allclose(a[keep], ref, rtol=0, atol=1e-15 * np.abs(ref).max())
    assert np.all(a[~keep] == 0)


@pytest.mark.parametrize("form", [0, 1])
def test_changeover_shape(form):
    rc = 0.02
    assert oracle.changeover(rc, rc, form) == 1.0
    assert oracle.changeover(2 * rc, rc, form) == 1.0
    assert oracle.changeover(0.1 * rc, rc, form) == 0.0
    assert oracle.changeover(0.0, rc, form) == 0.0
    assert abs(oracle.changeover(0.55 * rc, rc, form) - 0.5) <= 1e-15
    r = np.linspace(0.1 * rc, rc, 401)
    K = np.array([oracle.changeover(t, rc, form) for t in r])
    assert np.all(np.diff(K) >= 0)
    # symmetric about the midpoint: K(y) + K(1 - y) = 1
    for y in np.linspace(0.01, 0.99, 23):
        r1 = 0.1 * rc + 0.9 * rc * y
        r2 = 0.1 * rc + 0.9 * rc * (1 - y)
        assert abs(oracle.changeover(r1, rc, form) + oracle.changeover(r2, rc, form) - 1) <= 1e-14
    # continuous at both ends
    assert oracle.changeover(rc * (1 - 1e-9), rc, form) > 1 - 1e-6
    assert oracle.changeover(0.1 * rc * (1 + 1e-9), rc, form) < 1e-6


def test_hill_radius_closed_form():
    m = np.array([3e-6, 1e-3, 0.0])
    x = np.array([[1.0, 0, 0], [0, 5.2, 0], [0, 0, 2.0]])
    rc = oracle.hill_rcrit(1.0, 3.0, m, x)
    assert abs(rc[0] - 3 * 1.0 * (1e-6) ** (1 / 3)) <= 1e-16
    assert abs(rc[1] - 3 * 5.2 * (1e-3 / 3) ** (1 / 3)) <= 1e-15
    assert rc[2] == 0.0


def test_dh_coordinates_give_the_two_body_energy():
    """For one planet, the DH Hamiltonian equals the relative two-body energy
    1/2 mu_red v_rel^2 - G M0 m / r, mu_red = M0 m / (M0 + m)."""
    M0, m = 1.0, np.array([1e-3])
    x, v = ic.elements_to_state(M0 + m[0], 2.0, 0.3, 0.1, 0.2, 0.3, 1.4)
    V = oracle.helio_to_dh(M0, m, v[None, :])
    E, L, P = oracle.energy(1.0, M0, m, x[None, :], V)
    mu_red = M0 * m[0] / (M0 + m[0])
    E2 = 0.5 * mu_red * v @ v - M0 * m[0] / np.linalg.norm(x)
    assert abs(E - E2) <= 1e-15 * abs(E2)
    L2 = mu_red * np.cross(x, v)
    assert np.abs(L - L2).max() <= 1e-15 * np.linalg.norm(L2)


def test_dh_velocities_are_barycentric():
    s = ic.tiny(seed=3, n=7)
    V = oracle.helio_to_dh(1.0, s.m, s.v)
    # the star's barycentric velocity is -(sum m v)/(M0 + sum m); the bodies'
    # barycentric momenta plus the star's must vanish
    vstar = -(s.m[:, None] * s.v).sum(0) / (1.0 + s.m.sum())
    total = (s.m[:, None] * V).sum(0) + 1.0 * vstar
    assert np.abs(total).max() <= 1e-20
    back = oracle.dh_to_helio(1.0, s.m, V)
    assert np.abs(back - s.v).max() <= 1e-15


def test_energy_matches_barycentric_definition():
    """E(DH) equals the plain barycentric kinetic energy of star + bodies plus all potentials."""
    s = ic.tiny(seed=4, n=9)
    V = oracle.helio_to_dh(1.0, s.m, s.v)
    E, L, P = oracle.energy(1.0, 1.0, s.m, s.x, V)
    Mt = 1.0 + s.m.sum()
    rcm = (s.m[:, None] * s.x).sum(0) / Mt
    vcm = (s.m[:, None] * s.v).sum(0) / Mt
    xs = np.vstack([-rcm, s.x - rcm])
    vs = np.vstack([-vcm, s.v - vcm])
    ms = np.concatenate([[1.0], s.m])
    with mp.workdps(30):
        T = sum(mp.mpf(0.5) * float(ms[i]) * sum(mp.mpf(float(t)) ** 2 for t in vs[i]) for i in range(len(ms)))
        U = mp.mpf(0)
        for i in range(len(ms)):
            for j in range(i + 1, len(ms)):
                U -= float(ms[i]) * float(ms[j]) / mp.sqrt(sum((mp.mpf(float(xs[i, k])) - float(xs[j, k])) ** 2
                                                               for k in range(3)))
        Eb = float(T + U)
        Lb = np.array([float(sum(ms[i] * np.cross(xs[i], vs[i])[k] for i in range(len(ms)))) for k in range(3)])
    assert abs(E - Eb) <= 1e-14 * abs(Eb)
    assert np.abs(L - Lb).max() <= 1e-14 * np.linalg.norm(Lb)
