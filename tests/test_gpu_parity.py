"""GPU parity: every stage of the CUDA path, and whole steps, against the oracle.

All calls go through the C ABI (include/opal.h, include/opal_testing.h).
Tolerances:
  - FP64 form: 1e-12 relative position error after 100 steps (1e-13 for
    a single stage); the two sides differ only in summation order and fused
    multiply-adds, except where a Bulirsch-Stoer accept/reject decision sits
    within rounding of the tolerance.
  - mixed form: 1e-6 relative position error after 100 steps, and |dE/E|
    within 2x the oracle's (plus 1e-14 absolute slack for round-off).
  - flagged pair sets: identical, except pairs whose exact minimum sits
    within 1e-9 relative of the critical distance.
"""
import json
import os

import numpy as np
import pytest

import oracle
import opal_ic as ic

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opal():
    from paper_2601_19654_gb300.build import build
    build()
    oracle.build()
    from paper_2601_19654_gb300 import opal as o
    return o


def relpos(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def drifted(s, dt):
    """(x0, V0) at the start of a drift and (x1, V1) after it, by the oracle."""
    V0 = oracle.helio_to_dh(s.M0, s.m, s.v)
    x0 = s.x.copy()
    x1, V1 = x0.copy(), V0.copy()
    for i in range(s.n):
        st, x1[i], V1[i], _ = oracle.kepler_drift(s.G * s.M0, dt, x0[i], V0[i])
        assert st == oracle.OK
    return x0, V0, x1, V1


# ---------------------------------------------------------------- drift
def test_drift_matches_oracle(opal):
    rng = np.random.default_rng(11)
    cases = []
    for k in range(300):
        if k % 10 == 9:
            a, e = -rng.uniform(0.5, 3), rng.uniform(1.1, 3)
            f = rng.uniform(-0.8, 0.8) * np.arccos(-1 / e)
        else:
            a, e, f = rng.uniform(0.3, 10), rng.uniform(0, 0.95), rng.uniform(0, 2 * np.pi)
        x, v = ic.elements_to_state(1.0, a, e, rng.uniform(0, 1), rng.uniform(0, 6), rng.uniform(0, 6), f)
        cases.append((x, v))
    x = np.array([c[0] for c in cases])
    v = np.array([c[1] for c in cases])
    for dt in (0.0628, -0.3, 7.7):
        xg, vg, itg = opal.debug_drift(1.0, dt, x, v)
        for i in range(len(x)):
            st, xo, vo, ito = oracle.kepler_drift(1.0, dt, x[i], v[i])
            assert st == oracle.OK and itg[i] > 0
            assert np.linalg.norm(xg[i] - xo) <= 1e-13 * np.linalg.norm(xo) * max(1.0, abs(dt))
            assert np.linalg.norm(vg[i] - vo) <= 1e-13 * np.linalg.norm(vo) * max(1.0, abs(dt))
            # iteration counts may differ where both sides stop at the round-off floor
            assert abs(int(itg[i]) - ito) <= 3


def test_drift_reports_nonconvergence(opal):
    x, v = ic.elements_to_state(1.0, 1.0, 0.3, 0.0, 0.0, 0.0, 1.0)
    xg, vg, it = opal.debug_drift(1.0, 0.5, x[None], v[None], max_iter=1)
    assert it[0] == -1
    assert np.array_equal(xg[0], x) and np.array_equal(vg[0], v)


# ---------------------------------------------------------------- kick
def _accel_case(name):
    if name == "tiny":
        return ic.tiny(0), None
    if name == "cluster":
        s = ic.random_cluster(seed=2, n=40, spread=0.01)
        return s, oracle.hill_rcrit(1.0, 20.0, s.m, s.x)      # many pairs inside rc
    if name == "planetesimals":
        return ic.planetesimals_jupiter(0, n=1000), None
    if name == "ragged":
        s = ic.random_cluster(seed=5, n=333, spread=0.05)
        return s, oracle.hill_rcrit(1.0, 10.0, s.m, s.x)
    raise KeyError(name)


def _accel_err(a, ao):
    """Per-body error relative to the body's |a| (to the largest |a| for a
    body whose every partner sits inside 0.1 rc, where the kick's share is 0)."""
    scale = np.maximum(np.linalg.norm(ao, axis=1), 1e-3 * np.linalg.norm(ao, axis=1).max())
    return np.linalg.norm(a - ao, axis=1) / scale


@pytest.mark.parametrize("name", ["tiny", "cluster", "planetesimals", "ragged"])
@pytest.mark.parametrize("form", [0, 1])
def test_accel_fp64_matches_oracle(opal, name, form):
    s, rc = _accel_case(name)
    if rc is None:
        rc = oracle.hill_rcrit(1.0, 3.0, s.m, s.x)
    with opal.Simulation.from_system(s, precision=0, changeover=form) as sim:
        a = sim.debug_accel(rc)
    ao = oracle.accel(1.0, s.m, s.x, rc, form=form)
    err = _accel_err(a, ao)
    assert err.max() <= 1e-12, err.max()


U32 = 2.0 ** -24


def _mixed_kick_bound(s, rc, rows):
    """Per-body bound on the mixed kick's error, from its arithmetic.
    - A pair beyond the slow-path threshold (2 (rc_i + rc_max))^2 is taken
      from the FP32 hi parts alone: each coordinate difference is off by up
      to 2^-24 (|x_i| + |x_j|) (the dropped lo parts and the rounding of the
      difference), so a term of size |t| = G m K / r^2 is off by up to
      3 |t| 2^-24 (|x_i| + |x_j|) / r.
    - Every term carries a few ulp of FP32 rounding, the approximate rsqrt
      included (8 ulp); a pair inside the critical distance, whose weight K
      comes from FP32 arithmetic on rc rounded up to a float, 32.
    - Each accumulator lane adds up to 128 terms in FP32: up to 128 ulp of
      the sum of the magnitudes.
    So |da_i| <= sum_j |t_j| (sep_j + (8 or 32 + 128) 2^-24).  A body whose pulls nearly
    cancel (sum |t| much larger than |a|) can reach a large relative error
    within it; the bound names which."""
    rcm = rc.max()
    out = np.empty(len(rows))
    tsum = np.empty(len(rows))
    for q, i in enumerate(rows):
        d = s.x - s.x[i]
        r = np.linalg.norm(d, axis=1)
        r[i] = np.inf
        rcij = np.maximum(rc, rc[i])
        K = np.ones(s.n)
        for j in np.nonzero(r < rcij)[0]:
            K[j] = oracle.changeover(r[j], rcij[j], 0)
        t = s.G * s.m * K / r ** 2
        far = r * r >= (2.0 * (rc[i] + rcm)) ** 2
        xn = np.linalg.norm(s.x, axis=1)
        sep = np.where(far, 3.0 * U32 * (xn + xn[i]) / r, 0.0)
        ulps = np.where(r < rcij, 32.0, 8.0) + 128.0
        out[q] = np.sum(t * (sep + ulps * U32))
        tsum[q] = np.sum(t)
    return out, tsum


def _check_mixed_accel(a, ao, bound, tsum):
    absd = np.linalg.norm(a - ao, axis=1)
    err = _accel_err(a, ao)
    ratio = np.where(bound > 0, absd / np.maximum(bound, 1e-300), 0.0)   # a body with no kick terms: 0 of 0
    k = int(np.argmax(err))
    print(f"mixed kick: median relative error {np.median(err):.2e}, largest {err[k]:.2e} "
          f"(a body whose mutual pulls sum to {tsum[k] / np.linalg.norm(ao[k]):.1f}x its net pull); "
          f"largest error / bound {ratio.max():.3f}")
    assert np.median(err) <= 1e-6, np.median(err)
    assert (absd <= bound).all(), (ratio.max(), int(np.argmax(ratio)))


@pytest.mark.parametrize("name", ["tiny", "cluster", "planetesimals", "ragged"])
def test_accel_mixed_matches_oracle(opal, name):
    """The mixed kick against the oracle: median relative error <= 1e-6 and
    every body within the bound its own terms give (_mixed_kick_bound)."""
    s, rc = _accel_case(name)
    if rc is None:
        rc = oracle.hill_rcrit(1.0, 3.0, s.m, s.x)
    with opal.Simulation.from_system(s, precision=1) as sim:
        a = sim.debug_accel(rc)
    ao = oracle.accel(1.0, s.m, s.x, rc)
    bound, tsum = _mixed_kick_bound(s, rc, list(range(s.n)))
    _check_mixed_accel(a, ao, bound, tsum)


def _accel_rows(s, rc, rows, form=0):
    """The oracle's kick sum for the given bodies only: G sum_j m_j K(r_ij;
    max(rc_i, rc_j)) (x_j - x_i) / r_ij^3, K from the oracle's changeover
    (1 beyond rc_ij, so only the few pairs inside it call it)."""
    out = np.empty((len(rows), 3))
    for q, i in enumerate(rows):
        d = s.x - s.x[i]
        r = np.linalg.norm(d, axis=1)
        r[i] = np.inf
        rcij = np.maximum(rc, rc[i])
        K = np.ones(s.n)
        for j in np.nonzero(r < rcij)[0]:
            K[j] = oracle.changeover(r[j], rcij[j], form)
        w = s.m * K / r ** 3
        out[q] = s.G * (w[:, None] * d).sum(axis=0)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_encounter_heavy_accelerations_on_a_sample(opal, precision):
    """The 131072-body encounter-heavy workload with Jupiter and Saturn: the
    kick's accelerations (every work item, chunk and partial row of the full
    launch) for 256 seeded-random bodies and the two giants."""
    s = ic.encounter_heavy(0)
    rc = oracle.hill_rcrit(s.M0, 3.0, s.m, s.x)
    with opal.Simulation.from_system(s, precision=precision) as sim:
        a = sim.debug_accel(rc)
    rows = sorted(set(np.random.default_rng(7).choice(s.n, 256, replace=False).tolist()) |
                  {int(np.argmax(s.m)), int(np.argsort(s.m)[-2])})
    ao = _accel_rows(s, rc, rows)
    err = _accel_err(a[rows], ao)
    if precision == 0:
        assert err.max() <= 1e-12, err.max()
    else:
        bound, tsum = _mixed_kick_bound(s, rc, rows)
        _check_mixed_accel(a[rows], ao, bound, tsum)


# ---------------------------------------------------------------- scan
def _scan_compare(opal, s, dt, f_hill):
    x0, V0, x1, V1 = drifted(s, dt)
    rc = oracle.hill_rcrit(s.M0, f_hill, s.m, x1)
    with opal.Simulation.from_system(s, dt=dt) as sim:
        gi, gj, gcand = sim.debug_scan(x0, V0, x1, V1, rc)
    oi, oj, ocand = oracle.scan(dt, x0, V0, x1, V1, rc)
    got, ref = set(zip(gi.tolist(), gj.tolist())), set(zip(oi.tolist(), oj.tolist()))
    for (i, j) in got ^ ref:
        D = oracle.min_sep2(dt, x0[j] - x0[i], V0[j] - V0[i], x1[j] - x1[i], V1[j] - V1[i])
        r2 = max(rc[i], rc[j]) ** 2
        assert abs(D - r2) <= 1e-9 * r2, (i, j, D, r2)
    return len(ref), gcand


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("f_hill", [0.5, 2.0, 8.0])
def test_scan_matches_oracle_on_clusters(opal, seed, f_hill):
    s = ic.random_cluster(seed=seed, n=70, spread=0.02, vspread=0.05)
    nflag, ncand = _scan_compare(opal, s, 0.05, f_hill)
    assert ncand >= nflag


def test_scan_matches_oracle_on_planetesimal_disk(opal):
    s = ic.planetesimals_jupiter(0, n=1000)
    nflag, _ = _scan_compare(opal, s, s.dt, 3.0)
    assert nflag > 0


def test_scan_backwards_in_time(opal):
    s = ic.random_cluster(seed=9, n=50, spread=0.02, vspread=0.05)
    _scan_compare(opal, s, -0.05, 2.0)


# ---------------------------------------------------------------- BS
def _bs_compare(opal, X0, V0, m, R, rc, dt, tol=1e-12, tol_v=None, exact_substeps=True):
    n = len(m)
    p = oracle.make_params(dt=dt)
    mo, Ro, rco = m.copy(), R.copy(), rc.copy()
    alive = np.ones(n, np.int32)
    Xo, Vo = X0.copy(), V0.copy()
    st, El, nmg, sub = oracle.bs_group(p, np.arange(n, dtype=np.int32), mo, Ro, rco, alive, Xo, Vo)
    assert st == oracle.OK
    sys_bodies = ic.System("g", m.copy(), X0.copy(), V0.copy(), R.copy(), dt=dt, nsteps=1)
    with opal.Simulation.from_system(sys_bodies, precision=0) as sim:
        gst, out = sim.debug_bs_group(X0, V0, rc, m, R)
    assert gst == opal.OK
    assert out["alive"].tolist() == alive.tolist()
    assert np.array_equal(out["m"], mo)
    live = alive > 0
    assert relpos(out["x"][live], Xo[live]) <= tol
    assert np.abs(out["V"][live] - Vo[live]).max() <= (tol_v or tol) * np.abs(Vo[live]).max()
    if exact_substeps:
        assert out["substeps"] == sub
    else:
        assert abs(out["substeps"] - sub) <= max(2, sub // 50), (out["substeps"], sub)
    if nmg:   # a difference of nearly equal energies: relative precision ~1e-12 / 1e-3
        assert abs(out["E_lost"] - El) <= 1e-10 * abs(El)
    return nmg, sub


def test_bs_single_body_matches_oracle(opal):
    x, v = ic.elements_to_state(1.0, 1.2, 0.3, 0.1, 0.2, 0.3, 2.0)
    _bs_compare(opal, x[None], v[None], np.array([1e-9]), np.array([1e-9]), np.array([1e-9]), 0.3)


def test_bs_close_encounter_matches_oracle(opal):
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.02, 0.0, 0.0, 0.0, 0.0)
    X0 = np.array([x1, x1 + [0.0, 0.004, 0.0002], x1 + [0.003, -0.002, 0.0]])
    V0 = np.array([v1, v1 + [0.01, -0.02, 0.0], v1 + [-0.01, 0.0, 0.001]])
    m = np.array([3e-6, 2e-6, 1e-6])
    nmg, sub = _bs_compare(opal, X0, V0, m, np.full(3, 1e-8), np.array([0.02, 0.01, 0.01]), 0.0628)
    assert sub >= 1


@pytest.mark.parametrize("dt,offset", [(0.3, 2e-4), (0.6, 5e-5), (0.0628, 1e-4)])
def test_bs_deep_encounter_with_rejections_matches_oracle(opal, dt, offset):
    """Close approaches that force 150-340 substeps and many halvings.  The
    bound is derived from the method's own accuracy on the case: ten times
    the change of the oracle's result when bs_tol goes from 1e-12 to 1e-13
    (at least 1e-10).  Substep counts may differ where an accept decision
    sits at the tolerance."""
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.02, 0.0, 0.0, 0.0, 0.0)
    X0 = np.array([x1, x1 + [0.0, 0.002, offset]])
    V0 = np.array([v1, v1 + [0.0, -0.06, 0.0]])
    m = np.array([3e-6, 1e-6])
    R, rc = np.full(2, 1e-9), np.array([0.02, 0.02])
    ref = {}
    for tol in (1e-12, 1e-13):
        X, V = X0.copy(), V0.copy()
        st, *_ = oracle.bs_group(oracle.make_params(dt=dt, bs_tol=tol), np.arange(2, dtype=np.int32), m.copy(),
                                 R.copy(), rc.copy(), np.ones(2, np.int32), X, V)
        assert st == oracle.OK
        ref[tol] = (X, V)
    change = [np.abs(ref[1e-12][k] - ref[1e-13][k]).max() / np.abs(ref[1e-13][k]).max() for k in (0, 1)]
    nmg, sub = _bs_compare(opal, X0, V0, m, R, rc, dt, tol=max(1e-10, 10 * change[0]),
                           tol_v=max(1e-10, 10 * change[1]), exact_substeps=False)
    assert sub >= 100


def test_bs_merger_matches_oracle(opal):
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.02, 0.0, 0.0, 0.0, 0.0)
    X0 = np.array([x1, x1 + [0.0, 0.004, 0.0002]])
    V0 = np.array([v1, v1 + [0.0, -0.08, -0.004]])
    m = np.array([3e-6, 2e-6])
    nmg, sub = _bs_compare(opal, X0, V0, m, np.array([3e-4, 2e-4]), np.array([1.0, 1.0]), 0.0628)
    assert nmg == 1


# ---------------------------------------------------------------- whole steps
def _run_pair(opal, s, nsteps, precision, block=10, **kw):
    sim = opal.Simulation.from_system(s, precision=precision, **kw)
    osim = oracle.Sim.from_system(s, **{k: v for k, v in kw.items() if k in ("dt", "changeover", "bs_max_substeps")})
    E0g, E0o = sim.energy()[0], osim.energy()[0]
    done = 0
    while done < nsteps:
        k = min(block, nsteps - done)
        sim.step(k)
        assert osim.step(k) == oracle.OK
        done += k
    st = sim.state()
    dEg = abs(sim.energy()[0] - E0g) / abs(E0g)
    dEo = abs(osim.energy()[0] - E0o) / abs(E0o)
    out = dict(sim=sim, osim=osim, st=st, dEg=dEg, dEo=dEo)
    return out


def _alive_parity(out):
    st, osim = out["st"], out["osim"]
    alive = np.nonzero(osim.alive)[0]
    assert st["ids"].tolist() == alive.tolist()
    return relpos(st["x"], osim.x[alive])


@pytest.mark.parametrize("name,nsteps", [("tiny", 100), ("planetesimals", 100)])
def test_step_fp64_matches_oracle(opal, name, nsteps):
    s = ic.tiny(0) if name == "tiny" else ic.planetesimals_jupiter(0, n=1000)
    out = _run_pair(opal, s, nsteps, 0)
    err = _alive_parity(out)
    assert err <= 1e-12, err
    E, L, P, El = out["sim"].energy()
    Eo, Lo, Po, Elo = out["osim"].energy()
    assert abs(E - Eo) <= 1e-13 * abs(Eo)
    assert np.abs(L - Lo).max() <= 1e-13 * np.linalg.norm(Lo)


@pytest.mark.parametrize("name,nsteps", [("tiny", 100), ("planetesimals", 100)])
def test_step_mixed_matches_oracle(opal, name, nsteps):
    s = ic.tiny(0) if name == "tiny" else ic.planetesimals_jupiter(0, n=1000)
    out = _run_pair(opal, s, nsteps, 1)
    err = _alive_parity(out)
    assert err <= 1e-6, err
    assert out["dEg"] <= 2 * out["dEo"] + 1e-14, (out["dEg"], out["dEo"])


def test_step_with_mergers_matches_oracle(opal):
    s = ic.random_cluster(seed=11, n=24, spread=0.02, vspread=0.01, mass=3e-7)
    s.R = s.R * 30.0
    out = _run_pair(opal, s, 60, 0, block=1)
    st, osim = out["st"], out["osim"]
    assert osim.alive.sum() < s.n                         # mergers happened
    err = _alive_parity(out)
    assert err <= 1e-9, err
    assert np.allclose(st["m"], osim.m[osim.alive > 0], rtol=1e-15, atol=0)
    El, Elo = out["sim"].energy()[3], out["osim"].energy()[3]
    assert abs(El - Elo) <= 1e-9 * abs(Elo)


def test_mixed_overlap_step_with_mergers_matches_oracle(opal):
    """The mixed form's overlap step (the kick on the state after the drift,
    beside the encounter integrator, encounter members left out as sources
    and their new terms added afterwards) with perfect mergers: 2000
    planetesimals and Jupiter with radii x600, 10 steps in one call (under
    8% of the big bodies in encounters, so the step stays in overlap), about
    27 mergers.  Survivors, masses and E_lost must follow the oracle."""
    s = ic.planetesimals_jupiter(3, n=2000)
    s.R = s.R * 600.0
    with opal.Simulation.from_system(s, precision=1) as sim:
        osim = oracle.Sim.from_system(s)
        sim.step(10)
        assert sim.step_overlap
        assert osim.step(10) == oracle.OK
        st = sim.state()
        alive = np.nonzero(osim.alive)[0]
        assert alive.size < s.n                             # mergers happened
        assert st["ids"].tolist() == alive.tolist()
        err = relpos(st["x"], osim.x[alive])
        assert err <= 1e-6, err
        assert np.allclose(st["m"], osim.m[alive], rtol=1e-14, atol=0)
        El, Elo = sim.energy()[3], osim.energy()[3]
        assert abs(El - Elo) <= 1e-6 * abs(Elo), (El, Elo)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_equal_mass_disk_two_steps(opal, precision):
    """The 16384-body workload in the benchmark's launch configuration; the
    oracle's scan runs the exact test on all 1.3e8 pairs."""
    s = ic.equal_mass_disk(0)
    out = _run_pair(opal, s, 2, precision, block=1)
    err = _alive_parity(out)
    assert err <= (1e-12 if precision == 0 else 1e-6), err
    assert out["sim"].stats()["n_pairs"] == out["osim"].stats.n_pairs


def test_full_size_equal_mass_disk_hundred_steps(opal):
    """The headline workload (16384 equal-mass bodies, dt = 0.01 yr) for 100
    steps in both forms against one oracle run on the same seeded inputs:
    relative position error <= 1e-6 (mixed form), |dE/E| of the mixed form
    within 2x the oracle's over the same steps, and the flagged-pair count of
    every step equal to the oracle's in the FP64 form.

    FP64 form: 1e-12 for 99.9% of the bodies, and for the rest within twice
    what the oracle itself moves when its inputs move by one ulp
    (tests/golden/disk16384_oracle_sensitivity.json, written by the script
    beside it from two oracle runs): 100 steps of about 110 encounters each
    amplify rounding differences to ~1e-11 for the few bodies in the closest
    encounters (8 of 16384 above 1e-12 in the oracle's own comparison),
    which no independent FP64 rounding can avoid.  The mixed form follows a trajectory ~1e-7 away from the oracle's
    (relative), so a pair whose minimum separation lies that close to its
    critical distance may flip: its counts must agree to one pair a step and
    to 1% over the run.  The oracle's scan skips pairs by its end-point bound
    here (the all-pairs test would take 100 x 10 s); the pruned and exact
    scans are pinned to give the same set."""
    s = ic.equal_mass_disk(0)
    osim = oracle.Sim.from_system(s, scan_prune=1)
    E0o = osim.energy()[0]
    with opal.Simulation.from_system(s, precision=0) as g64, opal.Simulation.from_system(s, precision=1) as gmx:
        E0 = [g.energy()[0] for g in (g64, gmx)]
        counts = []
        for _ in range(100):
            g64.step(1)
            gmx.step(1)
            assert osim.step(1) == oracle.OK
            counts.append((osim.stats.n_pairs, g64.stats()["n_pairs"], gmx.stats()["n_pairs"]))
        counts = np.array(counts)
        alive = np.nonzero(osim.alive)[0]
        st64, stmx = g64.state(), gmx.state()
        assert st64["ids"].tolist() == alive.tolist() and stmx["ids"].tolist() == alive.tolist()
        err64 = relpos(st64["x"], osim.x[alive])
        errmx = relpos(stmx["x"], osim.x[alive])
        dEo = abs(osim.energy()[0] - E0o) / abs(E0o)
        dE64 = abs(g64.energy()[0] - E0[0]) / abs(E0[0])
        dEmx = abs(gmx.energy()[0] - E0[1]) / abs(E0[1])
        print(f"100 steps, 16384 bodies: position error FP64 {err64:.3e}, mixed {errmx:.3e}; "
              f"|dE/E| oracle {dEo:.3e}, FP64 {dE64:.3e}, mixed {dEmx:.3e}; "
              f"flagged pairs {counts[:, 0].sum()} (oracle), {counts[:, 1].sum()} (FP64), {counts[:, 2].sum()} (mixed)")
        e64 = np.linalg.norm(st64["x"] - osim.x[alive], axis=1) / np.linalg.norm(osim.x[alive], axis=1)
        sens = json.load(open(os.path.join(GOLDEN, "disk16384_oracle_sensitivity.json")))
        print(f"FP64 per-body error: 99.9% quantile {np.quantile(e64, 0.999):.3e}, {(e64 > 1e-12).sum()} bodies "
              f"above 1e-12; the oracle's 1-ulp sensitivity: max {sens['max_rel_pos_change']:.3e}, "
              f"{sens['bodies_above_1e-12']} bodies above 1e-12")
        assert np.quantile(e64, 0.999) <= 1e-12
        assert err64 <= 2 * sens["max_rel_pos_change"], err64
        assert errmx <= 1e-6, errmx
        assert dEmx <= 2 * dEo + 1e-14, (dEmx, dEo)
        assert (counts[:, 1] == counts[:, 0]).all(), np.nonzero(counts[:, 1] != counts[:, 0])[0]
        assert np.abs(counts[:, 2] - counts[:, 0]).max() <= 1
        assert abs(int(counts[:, 2].sum()) - int(counts[:, 0].sum())) <= 0.01 * counts[:, 0].sum()


def test_backward_steps_retrace_forward_steps(opal):
    s = ic.tiny(0)
    with opal.Simulation.from_system(s, precision=0) as sim:
        x0 = sim.state()["x"]
        sim.step(100)
        st = sim.state()
    with opal.Simulation(st["m"], st["x"], st["v"], st["R"], precision=0, dt=-s.dt) as back:
        back.step(100)
        assert relpos(back.state()["x"], x0) <= 1e-12


def test_ensemble_matches_each_system(opal):
    systems = [ic.tiny(seed=3, n=70), ic.tiny(seed=4, n=130), ic.planetesimals_jupiter(1, n=200)]
    for s in systems:
        s.dt = systems[0].dt
    with opal.Simulation.ensemble(systems, precision=0) as sim:
        sim.step(20)
        for k, s in enumerate(systems):
            osim = oracle.Sim.from_system(s, dt=systems[0].dt)
            assert osim.step(20) == oracle.OK
            st = sim.state(k)
            assert relpos(st["x"], osim.x[osim.alive > 0]) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_ensemble_on_a_sample_of_systems(opal, precision):
    """The benchmark's 256-system ensemble (N log-uniform in 64-4096, about
    32000 encounter groups a step), stepped as one simulation in its
    benchmark launch configuration; the smallest, the largest and four
    seeded-random systems against the oracle after two steps."""
    systems = ic.ensemble(0, 256)
    ns = np.array([s.n for s in systems])
    pick = [int(np.argmin(ns)), int(np.argmax(ns))] + [int(k) for k in
                                                        np.random.default_rng(1).choice(256, 4, replace=False)]
    # FP64: 1e-9, as for the other many-group cases (an accept decision of the
    # packed path can sit within rounding of the tolerance); mixed: 1e-6
    tol = 1e-9 if precision == 0 else 1e-6
    with opal.Simulation.ensemble(systems, precision=precision) as sim:
        sim.step(2)
        assert sim.stats()["n_groups"] > 608            # the packed path takes part
        for k in pick:
            osim = oracle.Sim.from_system(systems[k], dt=systems[0].dt)
            assert osim.step(2) == oracle.OK
            st = sim.state(k)
            alive = np.nonzero(osim.alive)[0]
            assert st["ids"].tolist() == alive.tolist(), k
            assert relpos(st["x"], osim.x[alive]) <= tol, (k, relpos(st["x"], osim.x[alive]))
            assert np.allclose(st["m"], osim.m[alive], rtol=1e-15, atol=0), k


@pytest.mark.parametrize("inflate", [1.0, 30.0])
def test_many_groups_take_the_packed_path_and_match_the_oracle(opal, inflate):
    """More encounter groups in a step than the lockstep kernels take (608):
    the packed kernel (one lane per member) integrates them, and the step runs
    the kick after the encounters (many bodies involved).  Every system must
    still match the oracle; with inflated radii some groups merge."""
    systems = [ic.random_cluster(seed=300 + k, n=100, spread=0.15, vspread=0.01, mass=3e-7) for k in range(64)]
    for s in systems:
        s.R = s.R * inflate
    with opal.Simulation.ensemble(systems, precision=0) as sim:
        sim.step(1)
        assert sim.stats()["n_groups"] > 608
        sim.step(4)
        merged = 0
        for k, s in enumerate(systems):
            osim = oracle.Sim.from_system(s)
            assert osim.step(5) == oracle.OK
            st = sim.state(k)
            alive = np.nonzero(osim.alive)[0]
            assert st["ids"].tolist() == alive.tolist()
            merged += s.n - alive.size
            assert relpos(st["x"], osim.x[alive]) <= 1e-9
            assert np.allclose(st["m"], osim.m[alive], rtol=1e-15, atol=0)
        if inflate > 1.0:
            assert merged > 0


def _jupiter_zone(n, seed=21, inflate=1.0):
    """n small bodies on orbits about Jupiter's (4.6-5.8 au) and a Jupiter
    analogue: every step one encounter group of about n / 15 members."""
    disk = ic._disk(seed, 11, n, lambda u: np.full_like(u, 1e-4 * ic.M_EARTH), 4.6, 5.8, 0.02, 0.01, 2.0)
    jup = ic._giant(seed, 12, ic.M_JUP, 5.2, 0.048, 1.33)
    m, x, v, R = ic._cat(disk, jup)
    return ic.System(f"jupiter_zone_n{n}", m, x, v, R * inflate, dt=0.05 * ic.YEAR, nsteps=3)


@pytest.mark.parametrize("n,inflate", [(1500, 1.0), (2500, 1.0), (2500, 300.0)])
def test_groups_of_more_than_64_members_match_the_oracle(opal, n, inflate):
    """A group of about 100-160 members (Jupiter's critical sphere) goes to the
    whole-GPU encounter kernel; with inflated radii its members merge."""
    s = _jupiter_zone(n, inflate=inflate)
    out = _run_pair(opal, s, 3, 0, block=1)
    assert out["sim"].stats()["n_groups"] >= 1
    err = _alive_parity(out)
    assert err <= 1e-9, err
    st, osim = out["st"], out["osim"]
    assert np.allclose(st["m"], osim.m[osim.alive > 0], rtol=1e-14, atol=0)
    if inflate > 1.0:
        assert osim.alive.sum() < s.n
        # E_lost is a difference of nearly equal energies, led by the pair's mutual
        # term at contact: separation ~3e-5 au against positions ~5 au, so states
        # that agree to 1e-9 relative fix it to about 1e-4 at worst
        El, Elo = out["sim"].energy()[3], out["osim"].energy()[3]
        assert abs(El - Elo) <= 1e-4 * abs(Elo)


def test_reduced_encounter_heavy_groups_of_hundreds_match_the_oracle(opal):
    """The encounter-heavy workload built with 48000 instead of 131072
    planetesimals (same masses, radii x10, 2-10 au, Jupiter and Saturn,
    dt = 0.05 yr): the giants' encounter groups hold about 660 and 300
    members, so every step runs the whole-GPU encounter kernel on groups of
    hundreds.  Three steps of both forms against one oracle run: FP64 within
    1e-9 (as the other whole-GPU cases: an accept decision of a group of
    hundreds can sit within rounding of the tolerance), mixed within 1e-6."""
    s = ic.encounter_heavy(0, 48000)
    # the first step's groups, from the oracle's own drift and scan
    x0, V0, x1, V1 = drifted(s, s.dt)
    rc = oracle.hill_rcrit(s.M0, s.rcrit_hill, s.m, x1)
    pi, pj, _ = oracle.scan(s.dt, x0, V0, x1, V1, rc, prune=1)
    _, lab = oracle.groups(s.n, pi, pj)
    assert np.bincount(lab[lab >= 0]).max() > 500
    osim = oracle.Sim.from_system(s, scan_prune=1)
    assert osim.step(3) == oracle.OK
    alive = np.nonzero(osim.alive)[0]
    for precision, tol in ((0, 1e-9), (1, 1e-6)):
        with opal.Simulation.from_system(s, precision=precision) as sim:
            sim.step(3)
            st = sim.state()
            assert st["ids"].tolist() == alive.tolist()
            err = relpos(st["x"], osim.x[alive])
            print(f"precision {precision}: 3 steps of {s.n} bodies, max relative position error {err:.3e}")
            assert err <= tol, (precision, err)
            assert np.allclose(st["m"], osim.m[alive], rtol=1e-14, atol=0)


def test_get_state_roundtrip_continues_the_run(opal):
    s = ic.tiny(1)
    with opal.Simulation.from_system(s, precision=0) as a:
        a.step(30)
        st = a.state()
        with opal.Simulation(st["m"], st["x"], st["v"], st["R"], precision=0, dt=s.dt) as b:
            a.step(30)
            b.step(30)
            assert relpos(b.state()["x"], a.state()["x"]) <= 1e-13


def test_runs_are_deterministic(opal):
    s = ic.planetesimals_jupiter(2, n=600)
    out = []
    for _ in range(2):
        with opal.Simulation.from_system(s, precision=1) as sim:
            sim.step(40)
            out.append(sim.state()["x"])
    assert np.array_equal(out[0], out[1])


def test_profiled_steps_equal_graph_steps(opal):
    s = ic.planetesimals_jupiter(3, n=500)
    with opal.Simulation.from_system(s, precision=0) as a, opal.Simulation.from_system(s, precision=0) as b:
        a.step(5)
        prof = b.profile(5)
        assert np.array_equal(a.state()["x"], b.state()["x"])
        assert "kick" in prof and prof["kick"] > 0


def test_energy_matches_oracle_before_any_step(opal):
    s = ic.planetesimals_jupiter(0, n=1000)
    with opal.Simulation.from_system(s) as sim:
        E, L, P, El = sim.energy()
    Eo, Lo, Po = oracle.energy(1.0, 1.0, s.m, s.x, oracle.helio_to_dh(1.0, s.m, s.v))
    assert abs(E - Eo) <= 1e-14 * abs(Eo)
    assert np.abs(L - Lo).max() <= 1e-14 * np.linalg.norm(Lo)
    assert np.abs(P - Po).max() <= 1e-14 * np.abs(s.m[:, None] * s.v).sum()
    assert El == 0.0


# ---------------------------------------------------------------- failures
def test_kepler_failure_undoes_the_step(opal):
    s = ic.tiny(0)
    with opal.Simulation.from_system(s, precision=0, kepler_max_iter=1) as sim:
        before = sim.state()
        st = sim.try_step(3)
        assert st == opal.EKEPLER
        after = sim.state()
        assert sim.steps_done == 0
        for k in ("x", "v", "m", "R"):
            assert np.array_equal(before[k], after[k]), k
        assert "Kepler" in opal.lib().opal_last_error(sim.ptr).decode()


def test_bs_failure_undoes_the_step(opal):
    s = ic.random_cluster(seed=3, n=12, spread=0.004, vspread=0.01, mass=3e-6)
    with opal.Simulation.from_system(s, precision=0, bs_max_substeps=1, dt=0.3) as sim:
        before = sim.state()
        assert sim.try_step(1) == opal.EBS
        after = sim.state()
        for k in ("x", "v", "m", "R", "ids"):
            assert np.array_equal(before[k], after[k]), k


def test_barrier_wait_running_out_undoes_the_step(opal):
    """The whole-GPU encounter kernel (a group of about 100 members here)
    meets at grid barriers whose waits are bounded.  With barriers that never
    release (as if a block never arrived) and a 2 ms limit, every wait ends at
    the limit, all blocks leave through the abort flag, and the step reports
    OPAL_EBS and is undone; with normal barriers the same step then succeeds
    and matches the oracle."""
    import time
    s = _jupiter_zone(1500)
    with opal.Simulation.from_system(s, precision=0) as sim:
        before = sim.state()
        sim.debug_barrier(2_000_000, 1)
        t0 = time.perf_counter()
        assert sim.try_step(1) == opal.EBS
        assert time.perf_counter() - t0 < 2.0          # ended at the 2 ms limit, not at the default 4 s
        assert "grid-barrier wait ran out" in opal.lib().opal_last_error(sim.ptr).decode()
        after = sim.state()
        assert sim.steps_done == 0
        for k in ("x", "v", "m", "R", "ids"):
            assert np.array_equal(before[k], after[k]), k
        sim.debug_barrier(0, 0)
        sim.step(1)
        assert sim.stats()["n_groups"] >= 1
        osim = oracle.Sim.from_system(s)
        assert osim.step(1) == oracle.OK
        alive = np.nonzero(osim.alive)[0]
        st = sim.state()
        assert st["ids"].tolist() == alive.tolist()
        assert relpos(st["x"], osim.x[alive]) <= 1e-9


def test_encounter_overflow_is_reported_and_a_larger_list_succeeds(opal):
    s = ic.random_cluster(seed=4, n=40, spread=0.01, vspread=0.02, mass=3e-6)
    with opal.Simulation.from_system(s, precision=0, encounter_capacity=1) as sim:
        before = sim.state()
        assert sim.try_step(1) == opal.EOVERFLOW
        assert np.array_equal(before["x"], sim.state()["x"])
    with opal.Simulation.from_system(s, precision=0, encounter_capacity=4096) as sim:
        sim.step(1)
        assert sim.stats()["n_pairs"] > 1
