"""The allocation-free energy diagnostic against the simulation's own.

opal_energy_momentum_noalloc (device arrays in, nothing allocated, fixed
scratch in device memory) must give the E, L and P that
opal_energy_momentum gives for the same state, on two calls in a row, and
the oracle's energy and momenta of one state.  Both library calls go
through the C ABI.  The file name sorts last so that the test also runs
after every other GPU test has used the device.

Tolerances: the two sides sum the same FP64 terms in different orders (and
the diagnostic counts each pair from both ends), so E and L agree to 1e-12
relative; P, a sum with cancellation, to 1e-12 of sum m |v|.
"""
import numpy as np
import pytest

import opal_ic as ic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def opal():
    from paper_2601_19654_gb300.build import build
    build()
    from paper_2601_19654_gb300 import opal as o
    return o


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _noalloc(o, n, G, M0, m, x, v):
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    o.energy_momentum_noalloc(n, G, M0, m.data_ptr(), x.data_ptr(), v.data_ptr(), out.data_ptr(),
                              stream.cuda_stream)
    stream.synchronize()
    return out.cpu().numpy()


def _check(out, E, L, P, st):
    assert np.all(np.isfinite(out))
    assert abs(out[0] - E) <= 1e-12 * abs(E), (out[0], E)
    np.testing.assert_allclose(out[1:4], L, rtol=1e-12, atol=1e-12 * np.linalg.norm(L))
    pscale = float(np.sum(st["m"] * np.linalg.norm(st["v"], axis=1)))
    np.testing.assert_allclose(out[4:7], P, rtol=0, atol=1e-12 * pscale)


@pytest.mark.parametrize("name,make,steps", [
    ("1001 bodies (ragged last block), after 20 steps", lambda: ic.planetesimals_jupiter(5, 1000), 20),
    ("16384-body disk, after 3 steps", lambda: ic.equal_mass_disk(2, 16384), 3),
    ("131072-body disk (the size limit), initial state", lambda: ic.equal_mass_disk(4, 131072), 0),
])
def test_noalloc_matches_energy_momentum(opal, name, make, steps):
    s = make()
    sim = opal.Simulation.from_system(s, precision=0)
    if steps:
        sim.step(steps)
    E, L, P, _ = sim.energy()
    st = sim.state()
    sim.close()
    n = st["m"].size
    m, x, v = _dev(st["m"]), _dev(st["x"]), _dev(st["v"])
    first = _noalloc(opal, n, s.G, s.M0, m, x, v)
    second = _noalloc(opal, n, s.G, s.M0, m, x, v)
    _check(first, E, L, P, st)
    _check(second, E, L, P, st)
    # same inputs, same fixed-order sums: the second call repeats the first exactly
    assert np.array_equal(first, second)


def test_noalloc_matches_the_oracle_energy(opal):
    """Once against the oracle itself: the oracle's energy and momenta (its
    own DH conversion and compensated sums) of the same 1001-body state."""
    import oracle
    oracle.build()
    s = ic.planetesimals_jupiter(6, 1000)
    with opal.Simulation.from_system(s, precision=0) as sim:
        sim.step(10)
        st = sim.state()
    n = st["m"].size
    out = _noalloc(opal, n, s.G, s.M0, _dev(st["m"]), _dev(st["x"]), _dev(st["v"]))
    V = oracle.helio_to_dh(s.M0, st["m"], st["v"])
    E, L, P = oracle.energy(s.G, s.M0, st["m"], st["x"], V)
    _check(out, E, L, P, st)


def test_noalloc_empty_and_rejections(opal):
    m = _dev(np.ones(4))
    x = _dev(np.arange(12.0) + 1.0)
    v = _dev(np.zeros(12))
    # n = 0: nothing to sum, every output is zero
    assert np.array_equal(_noalloc(opal, 0, 1.0, 1.0, m, x, v), np.zeros(7))
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    host = np.zeros(12)
    bad = [
        ((131073, 1.0, 1.0, m.data_ptr(), x.data_ptr(), v.data_ptr(), out.data_ptr()), "131072"),
        ((-1, 1.0, 1.0, m.data_ptr(), x.data_ptr(), v.data_ptr(), out.data_ptr()), "< 0"),
        ((4, 0.0, 1.0, m.data_ptr(), x.data_ptr(), v.data_ptr(), out.data_ptr()), "G and M0"),
        ((4, 1.0, 1.0, m.data_ptr(), host.ctypes.data, v.data_ptr(), out.data_ptr()), "not device memory"),
        ((4, 1.0, 1.0, m.data_ptr(), x.data_ptr() + 4, v.data_ptr(), out.data_ptr()), "aligned"),
        ((4, 1.0, 1.0, m.data_ptr(), x.data_ptr(), v.data_ptr(), 0), "NULL"),
    ]
    for args, why in bad:
        with pytest.raises(opal.OpalError) as e:
            opal.energy_momentum_noalloc(*args, torch.cuda.current_stream().cuda_stream)
        assert e.value.status == opal.EINVAL and why in str(e.value), (why, str(e.value))
    torch.cuda.synchronize()
    # nothing was launched for a rejected call: out still holds its NaNs
    assert torch.isnan(out).all().item()
