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


def _drifted_system(s, dt):
    V0 = oracle.helio_to_dh(s.M0, s.m, s.v)
    x0 = s.x.copy()
    x1, V1 = x0.copy(), V0.copy()
    for i in range(s.n):
        st, x1[i], V1[i], _ = oracle.kepler_drift(s.G * s.M0, dt, x0[i], V0[i])
        assert st == oracle.OK
    return x0, V0, x1, V1


@pytest.mark.parametrize("kind,n,f_hill,dt_mult", [
    ("planetesimals", 300, 3.0, 1.0), ("planetesimals", 1000, 3.0, 1.0), ("planetesimals", 2000, 3.0, 1.0),
    ("planetesimals", 1000, 30.0, 4.0), ("disk", 2000, 3.0, 1.0), ("disk", 2000, 10.0, 1.0),
    ("disk", 2000, 30.0, 3.0), ("disk", 1000, 60.0, -2.0)])
def test_pruned_scan_equals_the_all_pairs_scan(kind, n, f_hill, dt_mult):
    """The skip bound only saves time: on systems built like the 1000-
    planetesimal and the equal-mass disk workloads (the disk at its own
    surface density, in an annulus; drifted by the oracle's
    own Kepler solver), with Hill factors and steps up to 30x and 4x the
    workloads' (forward and backward), the pruned scan flags exactly the
    pairs the exact test flags on every pair, while the bound removes almost
    all of them."""
    if kind == "planetesimals":
        s = ic.planetesimals_jupiter(7, n=n)
    else:
        # a 0.3 au wide annulus of the 16384-body disk: its bodies at the
        # workload's own surface density (about n of them)
        s = ic.equal_mass_disk(7)
        r = np.linalg.norm(s.x, axis=1)
        keep = np.nonzero((r > 1.0) & (r < 1.3))[0][:n]
        s = ic.System(s.name, s.m[keep], s.x[keep], s.v[keep], s.R[keep], dt=s.dt, nsteps=1)
    dt = s.dt * dt_mult
    x0, V0, x1, V1 = _drifted_system(s, dt)
    rc = oracle.hill_rcrit(s.M0, f_hill, s.m, x1)
    alive = np.ones(s.n, np.int32)
    alive[::97] = 0
    pi0, pj0, nc0 = oracle.scan(dt, x0, V0, x1, V1, rc, alive, prune=0)
    pi1, pj1, nc1 = oracle.scan(dt, x0, V0, x1, V1, rc, alive, prune=1)
    nlive = int(alive.sum())
    assert nc0 == nlive * (nlive - 1) // 2                  # every live pair got the exact test
    assert pi1.tolist() == pi0.tolist() and pj1.tolist() == pj0.tolist()
    assert len(pi0) > 0
    # the bound removes almost every pair at the workloads' parameters, and
    # most of them in the stress cases
    assert nc1 < (0.05 if (f_hill == 3.0 and dt_mult == 1.0) else 0.25) * nc0


def test_pruned_scan_keeps_pairs_just_inside_the_bound():
    """Pairs placed so that the minimum separation over the step sits just
    inside and just outside the critical distance, around many random
    directions and speeds: the pruned and the exact scans agree on each."""
    rng = np.random.default_rng(5)
    T = 0.0628
    for _ in range(40):
        n = 40
        x0 = rng.normal(size=(n, 3)) * 0.05 + [1.0, 0.0, 0.0]
        V0 = rng.normal(size=(n, 3)) * 0.3 + [0.0, 1.0, 0.0]
        x1, V1 = x0.copy(), V0.copy()
        for i in range(n):
            st, x1[i], V1[i], _ = oracle.kepler_drift(1.0, T, x0[i], V0[i])
            assert st == oracle.OK
        rc = np.full(n, 0.0)
        # each pair's critical distance set at its own minimum, scaled by 1 -/+ 1e-7:
        # use one radius per body equal to the median minimum of its pairs
        D = np.array([[oracle.min_sep2(T, x0[j] - x0[i], V0[j] - V0[i], x1[j] - x1[i], V1[j] - V1[i])
                       if j != i else np.inf for j in range(n)] for i in range(n)])
        rc = np.sqrt(np.median(np.where(np.isfinite(D), D, np.nan), axis=1, keepdims=False)) * rng.uniform(0.2, 0.6)
        pi0, pj0, _ = oracle.scan(T, x0, V0, x1, V1, rc, prune=0)
        pi1, pj1, _ = oracle.scan(T, x0, V0, x1, V1, rc, prune=1)
        assert pi1.tolist() == pi0.tolist() and pj1.tolist() == pj0.tolist()


def test_pruned_scan_on_paths_that_bulge_to_the_bound():
    """The end-point bound is tight for paths that leave and come back within
    the step.  With x1 = x0 and V1 = 0, body i's interpolated path is
    x0 + T h10(s) V0, whose largest excursion is (4/27) T |V0| at s = 1/3, the
    bound's own coefficient; with V1 = -V0 it is T |V0| / 4 at s = 1/2.  A
    partner at rest just inside (or outside) the critical distance of that
    apex, where the two end points are far apart, must be flagged (or not)
    alike by the pruned and the exact scans, and the exact minimum is checked
    against the apex distance."""
    rng = np.random.default_rng(17)
    T = 0.0628
    for kind in ("third", "half"):
        n = 80
        x0 = np.zeros((n, 3))
        V0 = np.zeros((n, 3))
        V1 = np.zeros((n, 3))
        rc = np.zeros(n)
        expect = {}
        for b in range(n // 2):
            i, j = 2 * b, 2 * b + 1
            x0[i] = rng.normal(size=3) * 3.0 + [20.0 * b, 0.0, 0.0]
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            speed = rng.uniform(0.5, 5.0)
            V0[i] = speed * u
            V1[i] = 0.0 if kind == "third" else -V0[i]
            apex = (4.0 / 27.0 if kind == "third" else 0.25) * T * speed
            rc[i] = rc[j] = rng.uniform(0.02, 0.2) * apex
            inside = b % 2 == 0
            x0[j] = x0[i] + u * (apex + rc[i] * (0.999 if inside else 1.001))
            expect[(i, j)] = inside
        x1 = x0.copy()
        pi0, pj0, _ = oracle.scan(T, x0, V0, x1, V1, rc, prune=0)
        pi1, pj1, _ = oracle.scan(T, x0, V0, x1, V1, rc, prune=1)
        got = set(zip(pi0.tolist(), pj0.tolist()))
        assert got == {p for p, f in expect.items() if f}, kind
        assert pi1.tolist() == pi0.tolist() and pj1.tolist() == pj0.tolist(), kind


def test_groups_are_connected_components():
    pi = np.array([0, 2, 5, 3, 7], np.int32)
    pj = np.array([4, 5, 9, 9, 8], np.int32)
    ng, label = oracle.groups(10, pi, pj)
    assert ng == 3
    assert label.tolist() == [0, -1, 2, 2, 0, 2, -1, 7, 7, 2]
