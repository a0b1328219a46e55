"""Thin ctypes binding of the C ABI in include/opal.h and include/opal_testing.h.

Argument marshalling only: every stage of the step runs in the CUDA library
``_build/libopal_gb300.so``.  There is no CPU fallback: if the library is
missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB, LIB_TIMELINE, build

OK, EINVAL, ENOMEM, ECUDA, EKEPLER, EBS, EOVERFLOW, ENONFINITE = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EKEPLER", 5: "EBS", 6: "EOVERFLOW",
                7: "ENONFINITE"}


class OpalError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("M0", C.c_double), ("dt", C.c_double), ("rcrit_hill", C.c_double),
                ("bs_tol", C.c_double), ("precision", C.c_int32), ("changeover", C.c_int32),
                ("kepler_max_iter", C.c_int32), ("bs_max_substeps", C.c_int32),
                ("encounter_capacity", C.c_int64), ("r_star", C.c_double), ("r_eject", C.c_double),
                ("eject_every", C.c_int64)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_P = C.c_void_p
_lib = None
_lock = threading.Lock()


def _declare(L):
    L.opal_default_params.argtypes = [C.POINTER(Params)]
    L.opal_create.argtypes = [C.POINTER(Params), C.c_int64, _D, _D, _D, _D, C.POINTER(_P)]
    L.opal_ensemble_create.argtypes = [C.POINTER(Params), C.c_int32, _I64, _D, _D, _D, _D, C.POINTER(_P)]
    L.opal_step.argtypes = [_P, C.c_int64]
    L.opal_step_async.argtypes = [_P, C.c_int64]
    L.opal_wait.argtypes = [_P]
    L.opal_num_systems.argtypes = [_P]
    L.opal_num_systems.restype = C.c_int32
    L.opal_num_bodies.argtypes = [_P]
    L.opal_num_bodies.restype = C.c_int64
    L.opal_steps_done.argtypes = [_P]
    L.opal_steps_done.restype = C.c_int64
    L.opal_get_state.argtypes = [_P, C.c_int32, C.POINTER(C.c_int64), _I64, _D, _D, _D, _D]
    L.opal_energy_momentum.argtypes = [_P, C.c_int32, C.POINTER(C.c_double), _D, _D, C.POINTER(C.c_double)]
    L.opal_last_step_stats.argtypes = [_P, _I64]
    L.opal_central_mass.argtypes = [_P, C.c_int32, C.POINTER(C.c_double)]
    L.opal_stream.argtypes = [_P]
    L.opal_stream.restype = C.c_void_p
    L.opal_profile_steps.argtypes = [_P, C.c_int64, C.c_int32, C.POINTER(C.c_int32), _D,
                                     C.POINTER(C.c_char_p)]
    L.opal_time_kick.argtypes = [_P, C.c_int32]
    L.opal_time_kick.restype = C.c_int
    L.opal_last_kick_ms.argtypes = [_P]
    L.opal_last_kick_ms.restype = C.c_double
    L.opal_time_kick_alone.argtypes = [_P, C.c_int32, C.POINTER(C.c_double)]
    L.opal_time_kick_alone.restype = C.c_int
    L.opal_graph_kernels.argtypes = [_P]
    L.opal_graph_kernels.restype = C.c_int32
    L.opal_step_overlap.argtypes = [_P]
    L.opal_step_overlap.restype = C.c_int32
    L.opal_kick_config.argtypes = [_P]
    L.opal_kick_config.restype = C.c_char_p
    L.opal_last_error.argtypes = [_P]
    L.opal_last_error.restype = C.c_char_p
    L.opal_destroy.argtypes = [_P]
    L.opal_destroy.restype = None
    L.opal_debug_accel.argtypes = [_P, C.c_void_p, _D]
    L.opal_debug_drift.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_int32, _D, _D, _I32]
    L.opal_debug_scan.argtypes = [_P, _D, _D, _D, _D, _D, C.c_int64, _I32, _I32, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)]
    L.opal_debug_bs_group.argtypes = [_P, _D, _D, _D, _D, _D, _D, _D, _I32, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64)]
    L.opal_debug_barrier.argtypes = [_P, C.c_int64, C.c_int32]
    L.opal_energy_momentum_noalloc.argtypes = [C.c_int64, C.c_double, C.c_double, _P, _P, _P, _P, _P]
    L.opal_probe_alu_peaks.argtypes = [_D]
    L.opal_timeline_kernels.argtypes = []
    L.opal_timeline_kernels.restype = C.c_int32
    L.opal_timeline_name.argtypes = [C.c_int32]
    L.opal_timeline_name.restype = C.c_char_p
    L.opal_timeline.argtypes = [_P, C.c_int32, _P]
    L.opal_timeline.restype = C.c_int
    for name in ("opal_probe_alu_peaks", "opal_create", "opal_ensemble_create", "opal_step", "opal_step_async", "opal_wait", "opal_get_state", "opal_energy_momentum",
                 "opal_last_step_stats", "opal_profile_steps", "opal_debug_accel", "opal_debug_drift",
                 "opal_debug_scan", "opal_debug_bs_group", "opal_debug_barrier", "opal_energy_momentum_noalloc",
                 "opal_central_mass"):
        getattr(L, name).restype = C.c_int


def lib(auto_build: bool = False):
    """The loaded CUDA library (builds it first when asked and out of date).
    With OPAL_TIMELINE_BUILD=1 in the environment when it is first loaded,
    the measurement build with the device timeline is loaded instead."""
    global _lib
    with _lock:
        if _lib is None:
            timeline = os.environ.get("OPAL_TIMELINE_BUILD") == "1"
            path = LIB_TIMELINE if timeline else LIB
            if auto_build:
                build(timeline=timeline)
            if not os.path.exists(path):
                raise OpalError(ECUDA, f"CUDA library not built ({path}); run paper_2601_19654_gb300.build.build()")
            L = C.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _check(st, sim_ptr=None):
    if st != OK:
        msg = lib().opal_last_error(sim_ptr)
        raise OpalError(st, msg.decode() if msg else "")


def energy_momentum_noalloc(n: int, G: float, M0: float, m_ptr: int, x_ptr: int, v_ptr: int, out_ptr: int,
                            stream: int = 0) -> None:
    """opal_energy_momentum_noalloc on device pointers (raw addresses): E, L, P
    of one system into out_ptr[7], enqueued on stream; nothing is allocated."""
    _check(lib().opal_energy_momentum_noalloc(int(n), float(G), float(M0), m_ptr, x_ptr, v_ptr, out_ptr,
                                              stream or None))


def probe_alu_peaks() -> dict:
    """opal_probe_alu_peaks: measured FP32 and FP64 FMA TFLOP/s and MUFU rsqrt
    Tops/s of the current device."""
    out = np.zeros(3)
    _check(lib().opal_probe_alu_peaks(out))
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "mufu_rsqrt_tops": float(out[2])}


def default_params(**kw) -> Params:
    p = Params()
    lib().opal_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class Simulation:
    """One system, or an ensemble of systems, resident on the GPU."""

    def __init__(self, m, x, v, radius, params: Params | None = None, n_per_sys=None, **kw):
        self.params = params if params is not None else default_params(**kw)
        m = _d(m)
        n = m.size
        x = _d(x, (n, 3))
        v = _d(v, (n, 3))
        radius = _d(radius)
        ptr = _P()
        if n_per_sys is None:
            self.n_per_sys = np.array([n], np.int64)
            st = lib().opal_create(C.byref(self.params), n, m, x, v, radius, C.byref(ptr))
        else:
            self.n_per_sys = np.ascontiguousarray(n_per_sys, dtype=np.int64)
            st = lib().opal_ensemble_create(C.byref(self.params), len(self.n_per_sys), self.n_per_sys, m, x, v,
                                            radius, C.byref(ptr))
        _check(st)
        self._ptr = ptr

    @classmethod
    def from_system(cls, s, **kw):
        args = dict(G=s.G, M0=s.M0, dt=s.dt, rcrit_hill=s.rcrit_hill)
        args.update(kw)
        return cls(s.m, s.x, s.v, s.R, **args)

    @classmethod
    def ensemble(cls, systems, **kw):
        args = dict(G=systems[0].G, M0=systems[0].M0, dt=systems[0].dt, rcrit_hill=systems[0].rcrit_hill)
        args.update(kw)
        return cls(np.concatenate([s.m for s in systems]), np.concatenate([s.x for s in systems]),
                   np.concatenate([s.v for s in systems]), np.concatenate([s.R for s in systems]),
                   n_per_sys=[s.n for s in systems], **args)

    @property
    def ptr(self):
        if self._ptr is None:
            raise OpalError(EINVAL, "simulation destroyed")
        return self._ptr

    def step(self, nsteps: int = 1) -> int:
        st = lib().opal_step(self.ptr, int(nsteps))
        _check(st, self.ptr)
        return st

    def step_async(self, nsteps: int = 1):
        _check(lib().opal_step_async(self.ptr, int(nsteps)), self.ptr)

    def wait(self) -> int:
        st = lib().opal_wait(self.ptr)
        _check(st, self.ptr)
        return st

    def try_step(self, nsteps: int = 1) -> int:
        """Like step() but returns the status instead of raising."""
        return lib().opal_step(self.ptr, int(nsteps))

    @property
    def steps_done(self) -> int:
        return lib().opal_steps_done(self.ptr)

    @property
    def stream(self) -> int:
        return lib().opal_stream(self.ptr)

    def state(self, sys: int = 0) -> dict:
        n = int(self.n_per_sys[sys])
        na = C.c_int64(0)
        ids = np.empty(n, np.int64)
        m = np.empty(n)
        x = np.empty((n, 3))
        v = np.empty((n, 3))
        R = np.empty(n)
        _check(lib().opal_get_state(self.ptr, sys, C.byref(na), ids, m, x, v, R), self.ptr)
        k = na.value
        return dict(ids=ids[:k], m=m[:k], x=x[:k], v=v[:k], R=R[:k])

    def energy(self, sys: int = 0):
        E = C.c_double(0)
        L = np.empty(3)
        P = np.empty(3)
        El = C.c_double(0)
        _check(lib().opal_energy_momentum(self.ptr, sys, C.byref(E), L, P, C.byref(El)), self.ptr)
        return E.value, L, P, El.value

    def stats(self) -> dict:
        out = np.zeros(8, np.int64)
        _check(lib().opal_last_step_stats(self.ptr, out), self.ptr)
        return dict(n_pairs=int(out[0]), n_groups=int(out[1]), n_mergers=int(out[2]), bs_substeps=int(out[3]),
                    n_candidates=int(out[4]), kepler_iter_max=int(out[5]), n_accreted=int(out[6]),
                    n_ejected=int(out[7]))

    def central_mass(self, sys: int = 0) -> float:
        """The star's mass of system sys (grows by every body it accretes)."""
        M0 = C.c_double(0.0)
        _check(lib().opal_central_mass(self.ptr, sys, C.byref(M0)), self.ptr)
        return M0.value

    @property
    def graph_kernels(self) -> int:
        return lib().opal_graph_kernels(self.ptr)

    @property
    def step_overlap(self) -> bool:
        """True when the last step call ran the kick beside the encounter integrator."""
        return lib().opal_step_overlap(self.ptr) == 1

    @property
    def kick_config(self) -> str:
        return lib().opal_kick_config(self.ptr).decode()

    def time_kick(self, enable: bool = True):
        _check(lib().opal_time_kick(self.ptr, 1 if enable else 0), self.ptr)

    def last_kick_ms(self) -> float:
        return lib().opal_last_kick_ms(self.ptr)

    def kick_alone_ms(self, reps: int = 10) -> float:
        """Mean device time of the step's kick kernel launched alone."""
        ms = C.c_double(0.0)
        _check(lib().opal_time_kick_alone(self.ptr, int(reps), C.byref(ms)), self.ptr)
        return ms.value

    def timeline_reset(self):
        """Clear the device timeline (a timeline build: OPAL_TIMELINE_BUILD=1)."""
        _check(lib().opal_timeline(self.ptr, 1, None), self.ptr)

    def timeline(self) -> dict:
        """Kernel name -> (first block start, last block end) in ns of the
        global timer, for the kernels that ran since timeline_reset()."""
        n = int(lib().opal_timeline_kernels())
        buf = np.zeros(2 * max(n, 1), dtype=np.uint64)
        _check(lib().opal_timeline(self.ptr, 0, buf.ctypes.data), self.ptr)
        out = {}
        for k in range(n):
            if buf[2 * k] != np.uint64(0xFFFFFFFFFFFFFFFF):
                out[lib().opal_timeline_name(k).decode()] = (int(buf[2 * k]), int(buf[2 * k + 1]))
        return out

    def profile(self, nsteps: int) -> dict:
        cap = 64
        nk = C.c_int32(0)
        ms = np.zeros(cap)
        names = (C.c_char_p * cap)()
        _check(lib().opal_profile_steps(self.ptr, int(nsteps), cap, C.byref(nk), ms, names), self.ptr)
        return {names[k].decode(): float(ms[k]) for k in range(nk.value)}

    # --- test hooks ---------------------------------------------------------
    def debug_accel(self, rc=None):
        n = int(self.n_per_sys.sum())
        a = np.empty((n, 3))
        rcp = None if rc is None else _d(rc).ctypes.data_as(C.c_void_p)
        keep = None if rc is None else _d(rc)
        if keep is not None:
            rcp = keep.ctypes.data_as(C.c_void_p)
        _check(lib().opal_debug_accel(self.ptr, rcp, a), self.ptr)
        return a

    def debug_scan(self, x0, V0, x1, V1, rc):
        n = int(self.n_per_sys.sum())
        cap = max(64, 8 * n)
        while True:
            pi = np.empty(cap, np.int32)
            pj = np.empty(cap, np.int32)
            cnt = C.c_int64(0)
            nc = C.c_int64(0)
            _check(lib().opal_debug_scan(self.ptr, _d(x0, (n, 3)), _d(V0, (n, 3)), _d(x1, (n, 3)),
                                         _d(V1, (n, 3)), _d(rc), cap, pi, pj, C.byref(cnt), C.byref(nc)), self.ptr)
            if cnt.value <= cap:
                return pi[:cnt.value].copy(), pj[:cnt.value].copy(), nc.value
            cap = int(cnt.value)

    def debug_bs_group(self, x0, V0, rc, m, radius, alive=None):
        n = int(self.n_per_sys.sum())
        x = np.empty((n, 3))
        V = np.empty((n, 3))
        m = _d(m).copy()
        radius = _d(radius).copy()
        alive = np.ones(n, np.int32) if alive is None else np.ascontiguousarray(alive, np.int32).copy()
        El = C.c_double(0)
        sub = C.c_int64(0)
        st = lib().opal_debug_bs_group(self.ptr, _d(x0, (n, 3)), _d(V0, (n, 3)), _d(rc), x, V, m, radius, alive,
                                       C.byref(El), C.byref(sub))
        return st, dict(x=x, V=V, m=m, R=radius, alive=alive, E_lost=El.value, substeps=sub.value)

    def debug_barrier(self, wait_ns: int = 0, hold: int = 0):
        """Limit of the whole-GPU encounter kernel's barrier waits (0: the
        default); hold=1 makes the barriers never release (test hook)."""
        _check(lib().opal_debug_barrier(self.ptr, int(wait_ns), int(hold)), self.ptr)

    def close(self):
        if getattr(self, "_ptr", None) is not None:
            lib().opal_destroy(self._ptr)
            self._ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_drift(mu, dt, x, v, max_iter=0):
    x = _d(x).copy()
    v = _d(v).copy()
    n = x.size // 3
    x = x.reshape(n, 3)
    v = v.reshape(n, 3)
    it = np.zeros(n, np.int32)
    _check(lib().opal_debug_drift(n, mu, dt, max_iter, x, v, it))
    return x, v, it
