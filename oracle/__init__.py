"""Python view of the FP64 oracle (test infrastructure only).

The oracle is plain serial C (``opal_oracle.c``) compiled with gcc into
``oracle/_build/liboracle.so`` and called through ctypes.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA library in ``paper_2601_19654_gb300``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opal_oracle.c")
_HDR = os.path.join(_HERE, "opal_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EKEPLER, EBS = 0, 1, 4, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("M0", C.c_double), ("dt", C.c_double),
                ("rcrit_hill", C.c_double), ("bs_tol", C.c_double),
                ("changeover", C.c_int32), ("kepler_max_iter", C.c_int32),
                ("bs_max_substeps", C.c_int32), ("scan_prune", C.c_int32),
                ("r_star", C.c_double), ("r_eject", C.c_double), ("eject_every", C.c_int64),
                ("steps_done", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_groups", C.c_int64), ("n_mergers", C.c_int64),
                ("bs_substeps", C.c_int64), ("kepler_iter_max", C.c_int64),
                ("n_candidates", C.c_int64), ("n_accreted", C.c_int64), ("n_ejected", C.c_int64)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = C.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_helio_to_dh.argtypes = [_i64, C.c_double, _D, _D, _D]
            L.orc_dh_to_helio.argtypes = [_i64, C.c_double, _D, _D, _D]
            L.orc_changeover.argtypes = [C.c_double, C.c_double, C.c_int32]
            L.orc_changeover.restype = C.c_double
            L.orc_hill_rcrit.argtypes = [_i64, C.c_double, C.c_double, _D, _D, _I, _D]
            L.orc_accel.argtypes = [_i64, C.c_double, C.c_int32, _D, _D, _D, _I, _D]
            L.orc_stumpff.argtypes = [C.c_double, _D]
            L.orc_kepler_drift.argtypes = [C.c_double, C.c_double, _D, _D, C.c_int32,
                                           C.POINTER(C.c_int32)]
            L.orc_kepler_drift.restype = C.c_int32
            L.orc_drift_min_r.argtypes = [C.c_double, C.c_double, _D, _D, _D, _D]
            L.orc_drift_min_r.restype = C.c_double
            L.orc_min_sep2.argtypes = [C.c_double, _D, _D, _D, _D]
            L.orc_min_sep2.restype = C.c_double
            L.orc_scan.argtypes = [_i64, C.c_double, _D, _D, _D, _D, _D, _I, C.c_void_p, C.c_int32, _i64, _I, _I,
                                   C.POINTER(C.c_int64)]
            L.orc_scan.restype = C.c_int64
            L.orc_groups.argtypes = [_i64, _i64, _I, _I, _I]
            L.orc_groups.restype = C.c_int64
            L.orc_bs_group.argtypes = [C.POINTER(Params), _i64, _I, _D, _D, _D, _I, _D, _D,
                                       C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int64)]
            L.orc_bs_group.restype = C.c_int32
            L.orc_energy.argtypes = [_i64, C.c_double, C.c_double, _D, _D, _D, _I,
                                     C.POINTER(C.c_double), _D, _D]
            L.orc_step.argtypes = [C.POINTER(Params), _i64, _D, _D, _D, _D, _D, _D, _I,
                                   C.POINTER(C.c_int32), C.POINTER(C.c_double), _i64,
                                   C.POINTER(Stats)]
            L.orc_step.restype = C.c_int32
            _lib = L
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _alive(n, alive=None):
    return np.ones(n, np.int32) if alive is None else np.ascontiguousarray(alive, dtype=np.int32)


def make_params(G=1.0, M0=1.0, dt=0.01 * 2 * np.pi, rcrit_hill=3.0, bs_tol=1e-12, changeover=0,
                kepler_max_iter=0, bs_max_substeps=0, r_star=0.0, r_eject=0.0, eject_every=0,
                scan_prune=0) -> Params:
    """scan_prune=0: the encounter scan runs the exact test on every pair (the
    plain definition); 1: it first skips the pairs the end-point bound rules
    out (same flagged set, for systems too large for the all-pairs test)."""
    return Params(G, M0, dt, rcrit_hill, bs_tol, changeover, kepler_max_iter, bs_max_substeps, int(scan_prune),
                  r_star, r_eject, eject_every, 0)


# --- function-level views ---------------------------------------------------
def helio_to_dh(M0, m, v):
    m = _d(m)
    V = np.empty((m.size, 3))
    lib().orc_helio_to_dh(m.size, M0, m, _d(v, (m.size, 3)), V)
    return V


def dh_to_helio(M0, m, V):
    m = _d(m)
    v = np.empty((m.size, 3))
    lib().orc_dh_to_helio(m.size, M0, m, _d(V, (m.size, 3)), v)
    return v


def changeover(r, rc, form=0):
    return lib().orc_changeover(float(r), float(rc), int(form))


def hill_rcrit(M0, f_hill, m, x, alive=None):
    m = _d(m)
    rc = np.empty(m.size)
    lib().orc_hill_rcrit(m.size, M0, f_hill, m, _d(x, (m.size, 3)), _alive(m.size, alive), rc)
    return rc


def accel(G, m, x, rc, alive=None, form=0):
    m = _d(m)
    a = np.empty((m.size, 3))
    lib().orc_accel(m.size, G, form, m, _d(x, (m.size, 3)), _d(rc), _alive(m.size, alive), a)
    return a


def stumpff(z):
    c = np.empty(4)
    lib().orc_stumpff(float(z), c)
    return c


def kepler_drift(mu, dt, x, v, max_iter=0):
    x = _d(x).copy()
    v = _d(v).copy()
    it = C.c_int32(0)
    st = lib().orc_kepler_drift(mu, dt, x, v, max_iter, C.byref(it))
    return st, x, v, it.value


def drift_min_r(mu, dt, x0, V0, x1, V1):
    """Closest approach to the star during a drift from (x0, V0) to (x1, V1)."""
    return lib().orc_drift_min_r(mu, dt, _d(x0), _d(V0), _d(x1), _d(V1))


def min_sep2(dt, d0, u0, d1, u1):
    return lib().orc_min_sep2(dt, _d(d0), _d(u0), _d(d1), _d(u1))


def scan(dt, x0, V0, x1, V1, rc, alive=None, m=None, prune=0):
    """Flagged pairs; m (optional) marks the small bodies (m == 0), no two of
    which are ever a pair.  Without m every body counts as big.  prune=0 tests
    every pair exactly; prune=1 skips the pairs the end-point bound rules out."""
    n = np.asarray(rc).size
    cap = max(16, 4 * n)
    mm = None if m is None else _d(m)
    while True:
        pi = np.empty(cap, np.int32)
        pj = np.empty(cap, np.int32)
        nc = C.c_int64(0)
        cnt = lib().orc_scan(n, dt, _d(x0, (n, 3)), _d(V0, (n, 3)), _d(x1, (n, 3)), _d(V1, (n, 3)),
                             _d(rc), _alive(n, alive),
                             None if mm is None else mm.ctypes.data_as(C.c_void_p), int(prune), cap, pi, pj,
                             C.byref(nc))
        if cnt <= cap:
            return pi[:cnt].copy(), pj[:cnt].copy(), nc.value
        cap = int(cnt)


def groups(n, pi, pj):
    label = np.empty(n, np.int32)
    ng = lib().orc_groups(n, len(pi), np.ascontiguousarray(pi, np.int32),
                          np.ascontiguousarray(pj, np.int32), label)
    return ng, label


def bs_group(params: Params, members, m, R, rc, alive, x, V):
    """BS over one step for the listed members; arrays are updated in place."""
    El = C.c_double(0.0)
    nmg = C.c_int64(0)
    sub = C.c_int64(0)
    st = lib().orc_bs_group(C.byref(params), len(members), np.ascontiguousarray(members, np.int32),
                            m, R, rc, alive, x, V, C.byref(El), C.byref(nmg), C.byref(sub))
    return st, El.value, nmg.value, sub.value


def energy(G, M0, m, x, V, alive=None):
    m = _d(m)
    E = C.c_double(0)
    L = np.empty(3)
    P = np.empty(3)
    lib().orc_energy(m.size, G, M0, m, _d(x, (m.size, 3)), _d(V, (m.size, 3)), _alive(m.size, alive),
                     C.byref(E), L, P)
    return E.value, L, P


class Sim:
    """Whole-step oracle state (heliocentric input, DH state inside)."""

    def __init__(self, m, x, v_helio, R, G=1.0, M0=1.0, dt=0.01 * 2 * np.pi, rcrit_hill=3.0,
                 bs_tol=1e-12, changeover=0, kepler_max_iter=0, bs_max_substeps=0, r_star=0.0,
                 r_eject=0.0, eject_every=0, scan_prune=0):
        self.p = make_params(G, M0, dt, rcrit_hill, bs_tol, changeover, kepler_max_iter,
                             bs_max_substeps, r_star, r_eject, eject_every, scan_prune)
        self.n = int(np.asarray(m).size)
        self.m = _d(m).copy()
        self.R = _d(R).copy()
        self.x = _d(x, (self.n, 3)).copy()
        self.V = helio_to_dh(M0, self.m, _d(v_helio, (self.n, 3)))
        self.a = np.zeros((self.n, 3))
        self.rc = np.zeros(self.n)
        self.alive = np.ones(self.n, np.int32)
        self.have_a = C.c_int32(0)
        self.E_lost = C.c_double(0.0)
        self.stats = Stats()
        self.steps_done = 0

    @classmethod
    def from_system(cls, s, **kw):
        args = dict(G=s.G, M0=s.M0, dt=s.dt, rcrit_hill=s.rcrit_hill)
        args.update(kw)
        return cls(s.m, s.x, s.v, s.R, **args)

    def step(self, nsteps=1) -> int:
        st = lib().orc_step(C.byref(self.p), self.n, self.m, self.R, self.x, self.V, self.a, self.rc,
                            self.alive, C.byref(self.have_a), C.byref(self.E_lost), int(nsteps),
                            C.byref(self.stats))
        self.steps_done = int(self.p.steps_done)
        return st

    @property
    def M0(self) -> float:
        """The star's mass (grows by the mass of every body it accretes)."""
        return float(self.p.M0)

    def energy(self):
        E, L, P = energy(self.p.G, self.p.M0, self.m, self.x, self.V, self.alive)
        return E, L, P, self.E_lost.value

    def helio_velocities(self):
        return dh_to_helio(self.p.M0, np.where(self.alive > 0, self.m, 0.0), self.V)

    def state(self):
        return dict(m=self.m.copy(), x=self.x.copy(), V=self.V.copy(), R=self.R.copy(),
                    alive=self.alive.copy(), a=self.a.copy(), rc=self.rc.copy())
