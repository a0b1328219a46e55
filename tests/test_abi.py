"""The C-ABI library builds, loads and exports every symbol its headers declare;
argument validation happens on the host, before any device call."""
import os
import re

import numpy as np
import pytest

from paper_2601_19654_gb300.build import build as build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    from paper_2601_19654_gb300 import opal
    return opal


def declared_functions():
    names = set()
    for h in ("opal.h", "opal_testing.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(opal_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    L = lib.lib()
    names = declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing


def test_defaults(lib):
    p = lib.default_params()
    assert p.G == 1.0 and p.M0 == 1.0 and p.rcrit_hill == 3.0 and p.bs_tol == 1e-12
    assert abs(p.dt - 0.02 * np.pi) < 1e-15
    assert p.precision == 1 and p.changeover == 0


def _bodies(n=3):
    m = np.full(n, 1e-6)
    x = np.array([[1.0 + 0.1 * k, 0.0, 0.0] for k in range(n)])
    v = np.array([[0.0, 1.0, 0.0] for _ in range(n)])
    return m, x, v, np.full(n, 1e-5)


@pytest.mark.parametrize("mutate,needle", [
    (lambda b, p: b[0].__setitem__(1, -1.0), "negative mass"),
    (lambda b, p: b[3].__setitem__(0, -1.0), "negative radius"),
    (lambda b, p: b[1].__setitem__((2, 0), np.nan), "non-finite"),
    (lambda b, p: b[2].__setitem__((0, 1), np.inf), "non-finite"),
    (lambda b, p: b[1].__setitem__(0, [0.0, 0.0, 0.0]), "on the star"),
    (lambda b, p: b[0].__setitem__(0, 0.0), "follows a small"),   # small bodies come after the big ones
    (lambda b, p: setattr(p, "dt", 0.0), "dt"),
    (lambda b, p: setattr(p, "dt", float("nan")), "dt"),
    (lambda b, p: setattr(p, "M0", -1.0), "M0"),
    (lambda b, p: setattr(p, "G", 0.0), "G"),
    (lambda b, p: setattr(p, "bs_tol", 0.0), "bs_tol"),
    (lambda b, p: setattr(p, "precision", 2), "precision"),
    (lambda b, p: setattr(p, "changeover", 5), "changeover"),
    (lambda b, p: setattr(p, "r_star", -1.0), "r_star"),
    (lambda b, p: setattr(p, "r_eject", float("inf")), "r_eject"),
    (lambda b, p: setattr(p, "r_eject", 400.0), "eject_every"),          # no interval given
])
def test_invalid_inputs_are_rejected_before_any_device_call(lib, mutate, needle):
    b = list(_bodies())
    p = lib.default_params()
    mutate(b, p)
    with pytest.raises(lib.OpalError) as e:
        lib.Simulation(*b, params=p)
    assert e.value.status == lib.EINVAL
    assert needle in str(e.value)


def test_empty_system_is_rejected(lib):
    with pytest.raises(lib.OpalError) as e:
        lib.Simulation(np.zeros(0), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    assert e.value.status == lib.EINVAL
    with pytest.raises(lib.OpalError) as e:
        m, x, v, R = _bodies(4)
        lib.Simulation(m, x, v, R, n_per_sys=[4, 0])
    assert e.value.status == lib.EINVAL


@pytest.mark.parametrize("nps,needle", [
    ([2, -1], "n ="),
    ([], "at least one system"),
])
def test_bad_ensemble_layouts_are_rejected(lib, nps, needle):
    m, x, v, R = _bodies(2)
    with pytest.raises(lib.OpalError) as e:
        lib.Simulation(m, x, v, R, n_per_sys=nps)
    assert e.value.status == lib.EINVAL
    assert needle in str(e.value)


def test_small_before_big_in_a_later_system_is_rejected(lib):
    """The big-first order holds within each system: the second system may
    not put a big body after its own small one."""
    m, x, v, R = _bodies(4)
    m[:] = [1e-6, 0.0, 0.0, 1e-6]                 # system 1 = bodies 2, 3: small then big
    with pytest.raises(lib.OpalError) as e:
        lib.Simulation(m, x, v, R, n_per_sys=[2, 2])
    assert e.value.status == lib.EINVAL and "follows a small" in str(e.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """With no built library there is no fallback: loading raises."""
    import importlib
    from paper_2601_19654_gb300 import opal
    monkeypatch.setattr(opal, "_lib", None)
    monkeypatch.setattr(opal, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(opal.OpalError):
        opal.lib()
    importlib.reload(opal)


def test_barrier_hook_rejects_a_null_simulation(lib):
    """The barrier test hook validates on the host: no simulation, no call."""
    assert lib.lib().opal_debug_barrier(None, 1000, 1) == lib.EINVAL


def test_normal_build_has_no_device_timeline(lib):
    """The device timeline is compiled only into the measurement build: the
    normal library reports no kernel slots and refuses the readout, while the
    slot names (shared by both builds) cover the step's kernels."""
    L = lib.lib()
    assert L.opal_timeline_kernels() == 0
    assert L.opal_timeline(None, 1, None) == lib.EINVAL
    names = []
    k = 0
    while L.opal_timeline_name(k) is not None:
        names.append(L.opal_timeline_name(k).decode())
        k += 1
    assert {"k_open", "k_kick", "k_bs_ws", "k_kick_rows", "k_close", "k_finish"} <= set(names)
    assert L.opal_timeline_name(-1) is None
