"""GPU parity with small bodies (Sec. 2.1: massless particles that feel the
star and the big bodies; only big bodies are gravity sources).

Every system lists its big bodies first, then its small ones.  Tolerances are
those of the all-big parity tests: 1e-12 (FP64) and 1e-6 (mixed) relative
position error on encounter-light runs, 1e-9 where Bulirsch-Stoer groups with
mergers decide the result.
"""
import numpy as np
import pytest

import oracle
import opal_ic as ic
from test_gpu_parity import _alive_parity, _jupiter_zone, _run_pair, relpos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def opal():
    from paper_2601_19654_gb300.build import build
    build()
    oracle.build()
    from paper_2601_19654_gb300 import opal as o
    return o


def _big_first(s):
    """The same system with its big bodies moved in front of its small ones
    (a stable reorder; ids then follow the new order)."""
    order = np.concatenate([np.nonzero(s.m > 0)[0], np.nonzero(s.m == 0)[0]])
    return ic.System(s.name + "_bigfirst", s.m[order], s.x[order], s.v[order], s.R[order], dt=s.dt,
                     nsteps=s.nsteps)


def _half_small_cluster(seed, n=48, inflate=30.0):
    s = ic.random_cluster(seed=seed, n=n, spread=0.02, vspread=0.01, mass=3e-7)
    s.m[n // 2:] = 0.0
    s.R = s.R * inflate
    return s


@pytest.mark.parametrize("precision", [0, 1])
def test_embryo_disk_with_planetesimals_matches_oracle(opal, precision):
    """63 embryos and Jupiter with 8000 massless planetesimals, 50 steps."""
    s = ic.embryos_planetesimals(1, n_big=64, n_small=8000)
    out = _run_pair(opal, s, 50, precision)
    err = _alive_parity(out)
    if precision == 0:
        assert err <= 1e-12, err
    else:
        assert err <= 1e-6, err
        assert out["dEg"] <= 2 * out["dEo"] + 1e-14, (out["dEg"], out["dEo"])


def test_small_bodies_merge_only_into_big_ones(opal):
    """Half of a dense cluster is massless and radii are inflated: small
    bodies that touch a big one are absorbed, two small ones never merge."""
    s = _half_small_cluster(11)
    out = _run_pair(opal, s, 60, 0, block=1)
    st, osim = out["st"], out["osim"]
    assert osim.alive[:24].sum() < 24 and osim.alive[24:].sum() < 24   # both kinds of merger
    err = _alive_parity(out)
    assert err <= 1e-9, err
    assert np.allclose(st["m"], osim.m[osim.alive > 0], rtol=1e-15, atol=0)
    assert (st["m"][st["ids"] >= 24] == 0).all()
    El, Elo = out["sim"].energy()[3], out["osim"].energy()[3]
    assert abs(El - Elo) <= 1e-9 * abs(Elo)


def test_many_groups_with_small_members_take_the_packed_path(opal):
    """More than 608 groups, each a mix of big and small members, through the
    packed encounter kernel; every system must match the oracle."""
    systems = []
    for k in range(64):
        s = ic.random_cluster(seed=500 + k, n=100, spread=0.15, vspread=0.01, mass=3e-7)
        s.m[60:] = 0.0
        s.R = s.R * 30.0
        systems.append(s)
    with opal.Simulation.ensemble(systems, precision=0) as sim:
        sim.step(1)
        assert sim.stats()["n_groups"] > 608
        sim.step(3)
        for k, s in enumerate(systems):
            osim = oracle.Sim.from_system(s)
            assert osim.step(4) == oracle.OK
            st = sim.state(k)
            alive = np.nonzero(osim.alive)[0]
            assert st["ids"].tolist() == alive.tolist()
            assert relpos(st["x"], osim.x[alive]) <= 1e-9
            assert np.allclose(st["m"], osim.m[alive], rtol=1e-15, atol=0)


@pytest.mark.parametrize("inflate", [1.0, 300.0])
def test_jupiter_with_a_swarm_of_small_bodies(opal, inflate):
    """Jupiter and 2500 massless bodies about its orbit: one group of more than
    64 members (the whole-GPU encounter kernel) that is almost all small
    bodies; with inflated radii they overlap one another and Jupiter, and
    only Jupiter absorbs them."""
    s = _jupiter_zone(2500, inflate=inflate)
    s.m[:-1] = 0.0
    s = _big_first(s)
    out = _run_pair(opal, s, 3, 0, block=1)
    assert out["sim"].stats()["n_groups"] >= 1
    err = _alive_parity(out)
    assert err <= 1e-9, err
    st, osim = out["st"], out["osim"]
    if inflate > 1.0:
        assert osim.alive.sum() < s.n
        assert st["m"][0] == s.m[0]                   # Jupiter keeps its mass


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_planetesimal_workload_on_a_sample(opal, precision):
    """The benchmark's small-body workload (1024 big, 262144 small bodies), one
    step in its launch configuration.  A small body acts on nothing, so the
    oracle run on the big bodies plus a sample of small ones gives the same
    states for those bodies (up to where a big body's encounter with a small
    one not in the sample sends it through Bulirsch-Stoer instead of the
    drift: within the BS tolerance)."""
    s = ic.embryos_planetesimals(0)
    nb = s.meta["n_big"]
    with opal.Simulation.from_system(s, precision=precision) as sim:
        sim.step(1)
        st = sim.state()
        assert sim.stats()["n_pairs"] > 0
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(np.arange(nb, s.n), 96, replace=False))
    keep = np.concatenate([np.arange(nb), sample])
    sub = ic.System("sample", s.m[keep], s.x[keep], s.v[keep], s.R[keep], dt=s.dt, nsteps=1)
    osim = oracle.Sim.from_system(sub)
    assert osim.step(1) == oracle.OK
    pos = {int(i): k for k, i in enumerate(st["ids"])}
    # the same bodies of the sample are alive on both sides
    assert [int(i) in pos for i in keep] == (osim.alive > 0).tolist()
    live = np.nonzero(osim.alive)[0]
    got = np.array([st["x"][pos[int(keep[k])]] for k in live])
    tol = 1e-10 if precision == 0 else 1e-6
    big = live < nb
    assert relpos(got[big], osim.x[live[big]]) <= tol
    assert relpos(got[~big], osim.x[live[~big]]) <= tol
