"""GPU parity of star collisions and ejections (Sec. 2.1.2: mce_cent, and
bodies beyond 400 au removed every 200 yr) against the oracle, through the
C ABI.  The removal step, the star's mass, the survivors' states and the
energy the removals take out must agree; positions to the usual bounds
(1e-12 FP64, 1e-6 mixed), E_lost to 1e-10 relative."""
import math

import numpy as np
import pytest

import oracle
import opal_ic as ic
from test_gpu_parity import relpos
from test_oracle_removal import _plunge

pytestmark = pytest.mark.gpu

DT = 0.01 * ic.YEAR


@pytest.fixture(scope="module")
def opal():
    from paper_2601_19654_gb300.build import build
    build()
    oracle.build()
    from paper_2601_19654_gb300 import opal as o
    return o


def _compare(sim, osim, tol, sys=0):
    st = sim.state(sys)
    alive = np.nonzero(osim.alive)[0]
    assert st["ids"].tolist() == alive.tolist()
    assert relpos(st["x"], osim.x[alive]) <= tol
    assert sim.central_mass(sys) == osim.M0
    El, Elo = sim.energy(sys)[3], osim.energy()[3]
    assert abs(El - Elo) <= 1e-10 * max(abs(Elo), 1e-30) + 1e-25


def _accretion_system():
    mp = 1e-3
    xp, vp = ic.elements_to_state(1.0 + mp, 1.5, 0.02, 0.0, 0.0, 0.0, 1.0)
    xb, vb = _plunge(q=0.002)
    xs, vs = _plunge(q=0.001, r_start=0.7)                 # a small body that plunges too
    m = np.array([mp, 2e-6, 0.0])
    return ic.System("accretion", m, np.array([xp, xb, xs]), np.array([vp, vb, vs]),
                     np.array([1e-4, 1e-5, 1e-6]), dt=DT, nsteps=400)


@pytest.mark.parametrize("precision", [0, 1])
def test_accretion_matches_the_oracle(opal, precision):
    s = _accretion_system()
    sim = opal.Simulation.from_system(s, precision=precision, r_star=0.005)
    osim = oracle.Sim.from_system(s, r_star=0.005)
    accreted = 0
    for _ in range(400):
        sim.step(1)
        assert osim.step(1) == oracle.OK
        st = sim.stats()
        assert st["n_accreted"] == osim.stats.n_accreted
        accreted += st["n_accreted"]
        if accreted == 2:
            break
    assert accreted == 2                                  # the embryo-mass body and the small one
    _compare(sim, osim, 1e-12 if precision == 0 else 1e-6)
    assert sim.central_mass() == 1.0 + 2e-6
    sim.step(20)                                          # and the run goes on
    assert osim.step(20) == oracle.OK
    _compare(sim, osim, 1e-12 if precision == 0 else 1e-6)


def test_ejection_matches_the_oracle(opal):
    mp = 1e-3
    xp, vp = ic.elements_to_state(1.0 + mp, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    s = ic.System("escape", np.array([mp, 1e-6, 1e-6]),
                  np.array([xp, [3.0, 0.0, 0.0], [0.0, -3.5, 0.1]]),
                  np.array([vp, [0.0, 1.2, 0.0], [1.1, 0.0, 0.0]]), np.array([1e-4, 1e-5, 1e-5]),
                  dt=DT, nsteps=400)
    kw = dict(r_eject=5.0, eject_every=25)
    sim = opal.Simulation.from_system(s, precision=0, **kw)
    osim = oracle.Sim.from_system(s, **kw)
    ejected = []
    for k in range(1, 400):
        sim.step(1)
        assert osim.step(1) == oracle.OK
        assert sim.stats()["n_ejected"] == osim.stats.n_ejected
        if osim.stats.n_ejected:
            ejected.append(k)
        if osim.alive.sum() == 1:
            break
    assert ejected and all(k % 25 == 0 for k in ejected)
    _compare(sim, osim, 1e-12)
    assert sim.central_mass() == 1.0


def test_removals_in_an_ensemble_keep_each_system_apart(opal):
    """Three systems: one with an accretion, one with ejections, one with
    neither; each system's star and state follow the oracle on its own."""
    acc = _accretion_system()
    esc = ic.System("escape", np.array([1e-3, 1e-6]), np.array([[1.0, 0.0, 0.0], [3.0, 0.0, 0.0]]),
                    np.array([[0.0, 1.0, 0.0], [0.0, 1.2, 0.0]]), np.array([1e-4, 1e-5]), dt=DT, nsteps=400)
    quiet = ic.tiny(seed=2, n=10)
    quiet.dt = DT
    systems = [acc, esc, quiet]
    kw = dict(r_star=0.005, r_eject=5.0, eject_every=25)
    with opal.Simulation.ensemble(systems, precision=0, **kw) as sim:
        osims = [oracle.Sim.from_system(s, **kw) for s in systems]
        for _ in range(6):
            sim.step(50)
            for o in osims:
                assert o.step(50) == oracle.OK
        for k, o in enumerate(osims):
            _compare(sim, o, 1e-12, sys=k)
        assert osims[0].alive.sum() < 3 and osims[1].alive.sum() < 2 and osims[2].alive.all()
