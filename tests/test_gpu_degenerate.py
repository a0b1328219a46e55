"""GPU parity on the degenerate systems of the method: one body (no pair at
all: the step is the jump and the Kepler drift), two bodies (one pair, in
and out of the changeover zone), a pair that merges on its first encounter
and leaves a one-body system that keeps stepping, and an ensemble that mixes
these with an ordinary system, so that j-ranges, tiles and groups of one and
two bodies sit beside full ones in one launch.  Tolerances as in
test_gpu_parity: 1e-12 relative position error in the FP64 form, 1e-6 in
the mixed form.
"""
import numpy as np
import pytest

import oracle
import opal_ic as ic

pytestmark = pytest.mark.gpu

DT = 0.01 * ic.YEAR


@pytest.fixture(scope="module")
def opal():
    from paper_2601_19654_gb300.build import build
    build()
    oracle.build()
    from paper_2601_19654_gb300 import opal as o
    return o


def relpos(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def _system(name, m, x, v, R):
    return ic.System(name, np.asarray(m, float), np.atleast_2d(np.asarray(x, float)).copy(),
                     np.atleast_2d(np.asarray(v, float)).copy(), np.asarray(R, float), dt=DT, nsteps=1)


def _one_body():
    x, v = ic.elements_to_state(1.0 + 3e-6, 1.0, 0.2, 0.05, 0.3, 0.4, 1.0)
    return _system("one", [3e-6], x, v, [4e-5])


def _two_bodies(sep_au):
    """Two Earth-mass bodies on neighbouring orbits, sep_au apart at the start."""
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.01, 0.0, 0.0, 0.0, 0.0)
    x2, v2 = ic.elements_to_state(1.0, 1.0 + sep_au, 0.01, 0.001, 0.0, 0.0, 0.002)
    return _system("two", [3e-6, 3e-6], [x1, x2], [v1, v2], [4e-5, 4e-5])


def _head_on():
    """Two bodies falling onto each other: they touch within the first step."""
    x1, v1 = ic.elements_to_state(1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    return _system("merge", [3e-6, 2e-6], [x1, x1 + [0.0, 1e-4, 0.0]], [v1, v1 + [0.0, -0.05, 0.0]],
                   [4e-5, 3e-5])


def _compare(opal, s, nsteps, precision, tol):
    with opal.Simulation.from_system(s, precision=precision) as sim:
        osim = oracle.Sim.from_system(s)
        first = None
        for _ in range(nsteps // 10):
            sim.step(10)
            assert osim.step(10) == oracle.OK
            first = first or sim.stats()
        st = sim.state()
        alive = np.nonzero(osim.alive)[0]
        assert st["ids"].tolist() == alive.tolist()
        assert relpos(st["x"], osim.x[alive]) <= tol
        assert np.allclose(st["m"], osim.m[alive], rtol=1e-15, atol=0)
        E, L, P, El = sim.energy()
        Eo, Lo, Po, Elo = osim.energy()
        assert abs(E - Eo) <= (1e-13 if precision == 0 else 1e-9) * abs(Eo)
        return first, osim


@pytest.mark.parametrize("precision", [0, 1])
def test_a_single_body_matches_the_oracle(opal, precision):
    _compare(opal, _one_body(), 100, precision, 1e-12 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("sep", [0.5, 0.02])
def test_two_bodies_match_the_oracle(opal, precision, sep):
    """sep = 0.5 au: no encounter, the pair is a plain Newtonian term; 0.02 au
    (inside the critical radius of 0.03 au): an encounter on each of the
    first 23 steps, then apart.  (A pair that stays bound inside its Hill
    sphere is chaotic: rounding grows past 1e-12 within 50 steps.)"""
    s = _two_bodies(sep)
    stats, osim = _compare(opal, s, 50, precision, 1e-12 if precision == 0 else 1e-6)
    if sep < 0.1:   # the 10th step
        assert stats["n_groups"] == 1 and stats["bs_substeps"] >= 1
    else:
        assert stats["n_groups"] == 0


def test_a_merger_that_leaves_one_body_matches_the_oracle(opal):
    s = _head_on()
    with opal.Simulation.from_system(s, precision=0) as sim:
        osim = oracle.Sim.from_system(s)
        sim.step(1)
        assert osim.step(1) == oracle.OK
        assert osim.alive.tolist() == [1, 0]
        assert sim.stats()["n_mergers"] == 1
        sim.step(20)                                    # a one-body system from here on
        assert osim.step(20) == oracle.OK
        st = sim.state()
        assert st["ids"].tolist() == [0]
        assert st["m"][0] == osim.m[0] == 3e-6 + 2e-6   # mass conserved, summed once
        assert relpos(st["x"], osim.x[:1]) <= 1e-9
        El, Elo = sim.energy()[3], osim.energy()[3]
        assert abs(El - Elo) <= 1e-9 * abs(Elo)


@pytest.mark.parametrize("precision", [0, 1])
def test_an_ensemble_of_uneven_and_degenerate_systems(opal, precision):
    systems = [_one_body(), _two_bodies(0.02), ic.tiny(seed=5, n=90), _two_bodies(0.5), _one_body()]
    for s in systems:
        s.dt = DT
    tol = 1e-12 if precision == 0 else 1e-6
    with opal.Simulation.ensemble(systems, precision=precision) as sim:
        sim.step(30)
        for k, s in enumerate(systems):
            osim = oracle.Sim.from_system(s)
            assert osim.step(30) == oracle.OK
            st = sim.state(k)
            alive = np.nonzero(osim.alive)[0]
            assert st["ids"].tolist() == alive.tolist()
            assert relpos(st["x"], osim.x[alive]) <= tol, k
