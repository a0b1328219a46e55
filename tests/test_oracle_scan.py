"""Pins of the oracle's close-encounter scan (Sec. 3.1, mce_snif LOOPs 1-3).

References: the closed-form minimum of straight-line relative motion (which
the cubic Hermite interpolant reproduces exactly), scipy's
CubicHermiteSpline sampled densely, and brute force over all pairs.
"""
import numpy as np
import pytest
from scipy.interpolate import CubicHermiteSpline

import oracle
import opal_ic as ic


def sampled_min2(T, d0, u0, d1, u1, n=20001):
    sp = CubicHermiteSpline([0.0, T] if T > 0 else [T, 0.0],
                            np.array([d0, d1]) if T > 0 else np.array([d1, d0]),
                            np.array([u0, u1]) if T > 0 else np.array([u1, u0]))
    t = np.linspace(min(0, T), max(0, T), n)
    D = (sp(t) ** 2).sum(axis=1)
    k = int(np.argmin(D))
    # refine around the best sample by golden section on the spline itself
    lo, hi = t[max(k - 1, 0)], t[min(k + 1, n - 1)]
    g = (np.sqrt(5) - 1) / 2
    for _ in range(80):
        a = hi - g * (hi - lo)
        b = lo + g * (hi - lo)
        if (sp(a) ** 2).sum() < (sp(b) ** 2).sum():
            hi = b
        else:
            lo = a
    return min(D[k], (sp(0.5 * (lo + hi)) ** 2).sum())


def test_linear_motion_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(200):
        T = rng.uniform(0.01, 0.2) * rng.choice([-1, 1])
        u = rng.normal(size=3)
        d0 = rng.normal(size=3) * 0.01
        d1 = d0 + u * T
        got = oracle.min_sep2(T, d0, u, d1, u)
        # closest approach along the line, clamped to the step
        tstar = np.clip(-(d0 @ u) / (u @ u), min(0, T), max(0, T))
        dmin = d0 + u * tstar
        assert abs(got - dmin @ dmin) <= 1e-12 * (d0 @ d0 + d1 @ d1)


def test_min_sep_matches_dense_sampling_of_the_hermite_path():
    rng = np.random.default_rng(1)
    for _ in range(300):
        T = rng.uniform(0.01, 0.3) * rng.choice([-1, 1])
        d0, u0, u1 = rng.normal(size=3) * 0.02, rng.normal(size=3), rng.normal(size=3)
        d1 = d0 + 0.5 * (u0 + u1) * T + rng.normal(size=3) * 0.002
        got = oracle.min_sep2(T, d0, u0, d1, u1)
        ref = sampled_min2(T, d0, u0, d1, u1)
        assert got <= ref * (1 + 1e-9) + 1e-30
        assert got >= ref * (1 - 1e-6) - 1e-18


def brute_force_flags(T, x0, V0, x1, V1, rc, alive):
    n = len(rc)
    flags = set()
    margins = {}
    for i in range(n):
        for j in range(i + 1, n):
            if not (alive[i] and alive[j]):
                continue
            D = sampled_min2(T, x0[j] - x0[i], V0[j] - V0[i], x1[j] - x1[i], V1[j] - V1[i], n=2001)
            r2 = max(rc[i], rc[j]) ** 2
            margins[(i, j)] = abs(D - r2) / r2
            if D <= r2:
                flags.add((i, j))
    return flags, margins


@pytest.mark.parametrize("seed,f_hill", [(k, f) for k in range(6) for f in (0.5, 1.0, 2.0)])
def test_scan_equals_brute_force_on_drifted_clusters(seed, f_hill):
    s = ic.random_cluster(seed=seed, n=10, spread=0.015, vspread=0.05)
    M0, dt = 1.0, 0.05
    V0 = oracle.helio_to_dh(M0, s.m, s.v)
    x0 = s.x.copy()
    x1, V1 = x0.copy(), V0.copy()
    for i in range(s.n):
        st, x1[i], V1[i], _ = oracle.kepler_drift(1.0, dt, x0[i], V0[i])
        assert st == oracle.OK
    rc = oracle.hill_rcrit(M0, f_hill, s.m, x1)
    alive = np.ones(s.n, np.int32)
    alive[seed % s.n] = 0
    pi, pj, ncand = oracle.scan(dt, x0, V0, x1, V1, rc, alive)
    got = set(zip(pi.tolist(), pj.tolist()))
    ref, margins = brute_force_flags(dt, x0, V0, x1, V1, rc, alive)
    # pairs within sampling precision of the threshold may legitimately differ
    diff = {p for p in got ^ ref if margins[p] > 1e-6}
    assert not diff
    assert len(got) < 36 and (f_hill < 1.0 or len(got) > 0)
    assert ncand >= len(got)
    assert list(zip(pi.tolist(), pj.tolist())) == sorted(got)


def test_scan_flags_fast_flyby_caught_only_mid_step():
    """Ends far apart, closest approach mid-step: bounds must not discard it."""
    T = 0.1
    x0 = np.array([[1.0, 0.0, 0.0], [1.0, -0.05, 0.0005]])
    V = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    x1 = x0 + V * T
    rc = np.array([0.002, 0.001])
    pi, pj, ncand = oracle.scan(T, x0, V, x1, V, rc)
    assert list(zip(pi, pj)) == [(0, 1)]
    rc = np.array([0.0004, 0.0004])
    pi, pj, ncand = oracle.scan(T, x0, V, x1, V, rc)
    assert len(pi) == 0


def test_groups_are_connected_components():
    pi = np.array([0, 2, 5, 3, 7], np.int32)
    pj = np.array([4, 5, 9, 9, 8], np.int32)
    ng, label = oracle.groups(10, pi, pj)
    assert ng == 3
    assert label.tolist() == [0, -1, 2, 2, 0, 2, -1, 7, 7, 2]
