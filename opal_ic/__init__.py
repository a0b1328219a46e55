"""Seeded synthetic initial conditions for planetary N-body systems.

This module is the only code shared by the oracle side and the CUDA side, and
it holds none of the integrator's arithmetic: it draws orbital elements from a
counter-based generator and turns them into heliocentric Cartesian states by
the textbook element-to-state formulas (no Kepler-equation solve: the angle
drawn for the orbital phase is the true anomaly).

Random numbers come from splitmix64 (Steele, Lea & Flood 2014), used in
counter mode: draw k of stream s is mix(key(s) + (k + 1) * GAMMA), where mix is
the splitmix64 finaliser.  Every draw is therefore reproducible from
(seed, stream, k) alone, on any machine.

Units: G = 1, lengths in au, masses in solar masses, time in yr / (2 pi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --- physical constants (IAU nominal values) -------------------------------
M_EARTH = 3.00349e-6      # Earth mass in solar masses
M_JUP = 9.54588e-4        # Jupiter mass in solar masses
M_SAT = 2.85886e-4        # Saturn mass in solar masses
AU_CM = 1.495978707e13    # 1 au in cm
MSUN_G = 1.98841e33       # solar mass in g
TWOPI = 2.0 * math.pi
YEAR = TWOPI              # one year in code time units (G = M_sun = au = 1)

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    """64-bit key of (seed, stream): one splitmix64 output of a packed word."""
    word = np.array([(int(seed) * 0x10001 + int(stream) * 0x9E37 + 0x5EED) & 0xFFFFFFFFFFFFFFFF],
                    dtype=np.uint64)
    return _mix(word)[0]


def uniform(seed: int, stream: int, k) -> np.ndarray:
    """Uniform doubles in [0, 1) for counters k (array-like of ints)."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + (k + np.uint64(1)) * _GAMMA
    return (_mix(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Stream:
    """Sequential view of one counter-based stream."""

    def __init__(self, seed: int, stream: int):
        self.seed, self.stream, self.k = int(seed), int(stream), 0

    def take(self, n: int) -> np.ndarray:
        u = uniform(self.seed, self.stream, np.arange(self.k, self.k + n))
        self.k += n
        return u


def rayleigh(u: np.ndarray, sigma: float) -> np.ndarray:
    return sigma * np.sqrt(-2.0 * np.log1p(-u))


def log_uniform(u: np.ndarray, lo: float, hi: float) -> np.ndarray:
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def radius_from_density(m: np.ndarray, rho_cgs: float) -> np.ndarray:
    """Physical radius in au of a sphere of mass m (M_sun) and density rho (g/cm^3)."""
    grams = np.asarray(m, dtype=np.float64) * MSUN_G
    return np.cbrt(3.0 * grams / (4.0 * math.pi * rho_cgs)) / AU_CM


def elements_to_state(mu, a, e, inc, Omega, omega, f):
    """Heliocentric position and velocity from elements (true anomaly f).

    Perifocal frame: r = p / (1 + e cos f), position r (cos f, sin f, 0),
    velocity sqrt(mu / p) (-sin f, e + cos f, 0), with p = a (1 - e^2);
    then the rotation Rz(Omega) Rx(inc) Rz(omega).
    """
    mu, a, e, inc, Omega, omega, f = (np.asarray(t, dtype=np.float64)
                                      for t in (mu, a, e, inc, Omega, omega, f))
    p = a * (1.0 - e * e)
    r = p / (1.0 + e * np.cos(f))
    pf = np.stack([r * np.cos(f), r * np.sin(f), np.zeros_like(r)], axis=-1)
    s = np.sqrt(mu / p)
    vf = np.stack([-s * np.sin(f), s * (e + np.cos(f)), np.zeros_like(r)], axis=-1)
    cO, sO, ci, si, cw, sw = (np.cos(Omega), np.sin(Omega), np.cos(inc), np.sin(inc),
                              np.cos(omega), np.sin(omega))
    # rows of Rz(Omega) Rx(inc) Rz(omega)
    R = np.empty(np.shape(r) + (3, 3))
    R[..., 0, 0] = cO * cw - sO * sw * ci
    R[..., 0, 1] = -cO * sw - sO * cw * ci
    R[..., 0, 2] = sO * si
    R[..., 1, 0] = sO * cw + cO * sw * ci
    R[..., 1, 1] = -sO * sw + cO * cw * ci
    R[..., 1, 2] = -cO * si
    R[..., 2, 0] = sw * si
    R[..., 2, 1] = cw * si
    R[..., 2, 2] = ci
    x = np.einsum("...ij,...j->...i", R, pf)
    v = np.einsum("...ij,...j->...i", R, vf)
    return x, v


@dataclass
class System:
    """One planetary system: heliocentric state of the bodies around a star."""
    name: str
    m: np.ndarray            # (n,) masses, M_sun
    x: np.ndarray            # (n, 3) heliocentric positions, au
    v: np.ndarray            # (n, 3) heliocentric velocities, au / (yr / 2 pi)
    R: np.ndarray            # (n,) physical radii, au
    dt: float                # step in code time units
    nsteps: int              # length of the run the workload is quoted on
    G: float = 1.0
    M0: float = 1.0
    rcrit_hill: float = 3.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def _disk(seed, stream, n, mass_fn, a_lo, a_hi, sig_e, sig_i, rho, G=1.0, M0=1.0):
    s = Stream(seed, stream)
    u = s.take(7 * n).reshape(n, 7)
    m = mass_fn(u[:, 0])
    a = a_lo + u[:, 1] * (a_hi - a_lo)
    e = np.minimum(rayleigh(u[:, 2], sig_e), 0.9)
    inc = rayleigh(u[:, 3], sig_i)
    Om, om, f = TWOPI * u[:, 4], TWOPI * u[:, 5], TWOPI * u[:, 6]
    x, v = elements_to_state(G * (M0 + m), a, e, inc, Om, om, f)
    return m, x, v, radius_from_density(m, rho)


def _giant(seed, stream, mass, a, e, rho, G=1.0, M0=1.0):
    u = Stream(seed, stream).take(3)
    x, v = elements_to_state(G * (M0 + mass), a, e, 0.0, TWOPI * u[0], TWOPI * u[1], TWOPI * u[2])
    return np.array([mass]), x[None, :], v[None, :], radius_from_density(np.array([mass]), rho)


def _cat(*parts):
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(4))


def tiny(seed: int = 0, n: int = 10) -> System:
    """10 bodies of 0.05-1 Earth masses at 0.7-2 au, e/i Rayleigh 0.01/0.005, rho 3."""
    m, x, v, R = _disk(seed, 1, n, lambda u: log_uniform(u, 0.05 * M_EARTH, 1.0 * M_EARTH),
                       0.7, 2.0, 0.01, 0.005, 3.0)
    return System(f"tiny_n{n}_seed{seed}", m, x, v, R, dt=0.01 * YEAR, nsteps=1000)


def planetesimals_jupiter(seed: int = 0, n: int = 1000) -> System:
    """n planetesimals of 1e-3-1e-1 Earth masses at 1-4 au (rho 2) plus Jupiter at 5.2 au."""
    disk = _disk(seed, 2, n, lambda u: log_uniform(u, 1e-3 * M_EARTH, 1e-1 * M_EARTH),
                 1.0, 4.0, 0.02, 0.01, 2.0)
    jup = _giant(seed, 3, M_JUP, 5.2, 0.048, 1.33)
    m, x, v, R = _cat(disk, jup)
    return System(f"planetesimals{n}_jupiter_seed{seed}", m, x, v, R, dt=0.02 * YEAR, nsteps=10000)


def equal_mass_disk(seed: int = 0, n: int = 16384) -> System:
    """n equal bodies of 1e-3 Earth masses at 0.5-3 au, e/i Rayleigh 0.01/0.005, rho 2."""
    m, x, v, R = _disk(seed, 4, n, lambda u: np.full_like(u, 1e-3 * M_EARTH),
                       0.5, 3.0, 0.01, 0.005, 2.0)
    return System(f"equal_mass_disk_n{n}_seed{seed}", m, x, v, R, dt=0.01 * YEAR, nsteps=1000)


def encounter_heavy(seed: int = 0, n: int = 131072) -> System:
    """n bodies of 1e-4 Earth masses at 2-10 au, e/i 0.05/0.025, radii x10, plus Jupiter and Saturn."""
    m, x, v, R = _disk(seed, 5, n, lambda u: np.full_like(u, 1e-4 * M_EARTH),
                       2.0, 10.0, 0.05, 0.025, 2.0)
    R = R * 10.0
    jup = _giant(seed, 6, M_JUP, 5.2, 0.048, 1.33)
    sat = _giant(seed, 7, M_SAT, 9.5, 0.056, 0.69)
    m, x, v, R = _cat((m, x, v, R), jup, sat)
    return System(f"encounter_heavy_n{n}_seed{seed}", m, x, v, R, dt=0.05 * YEAR, nsteps=500)


def embryos_planetesimals(seed: int = 0, n_big: int = 1024, n_small: int = 262144) -> System:
    """Big bodies first, then small ones (Mercury's big and small lists):
    n_big - 1 embryos of 0.01-0.1 Earth masses at 0.7-3 au (rho 3) and Jupiter
    at 5.2 au, then n_small massless planetesimals at 0.7-3 au with the radius
    of a 1e-4 Earth-mass body of density 2; e/i Rayleigh 0.02/0.01."""
    big = _disk(seed, 10, n_big - 1, lambda u: log_uniform(u, 0.01 * M_EARTH, 0.1 * M_EARTH),
                0.7, 3.0, 0.02, 0.01, 3.0)
    jup = _giant(seed, 11, M_JUP, 5.2, 0.048, 1.33)
    small = _disk(seed, 12, n_small, lambda u: np.zeros_like(u), 0.7, 3.0, 0.02, 0.01, 2.0)
    r_small = radius_from_density(np.array([1e-4 * M_EARTH]), 2.0)[0]
    small = (small[0], small[1], small[2], np.full(n_small, r_small))
    m, x, v, R = _cat(big, jup, small)
    return System(f"embryos{n_big}_planetesimals{n_small}_seed{seed}", m, x, v, R, dt=0.01 * YEAR,
                  nsteps=1000, meta={"n_big": n_big, "n_small": n_small})


def ensemble_sizes(seed: int = 0, nsys: int = 256, lo: int = 64, hi: int = 4096) -> np.ndarray:
    """Body counts of an ensemble, log-uniform in [lo, hi]."""
    u = Stream(seed, 8).take(nsys)
    return np.floor(log_uniform(u, lo, hi + 1.0)).astype(np.int64).clip(lo, hi)


def ensemble(seed: int = 0, nsys: int = 256, lo: int = 64, hi: int = 4096) -> list[System]:
    """nsys independent systems drawn like `tiny`, each with its own seed and size."""
    sizes = ensemble_sizes(seed, nsys, lo, hi)
    return [tiny(seed=1000 + 7919 * seed + k, n=int(nk)) for k, nk in enumerate(sizes)]


def jupiter_eccentric(e: float = 0.22, a: float = 5.2, mass: float = M_JUP) -> System:
    """One Jupiter-mass planet on an e = 0.22 orbit (energy test (i) of Sec. 4.2)."""
    x, v = elements_to_state(mass + 1.0, a, e, 0.0, 0.0, 0.0, 0.0)
    m = np.array([mass])
    return System("jupiter_e022", m, x[None, :], v[None, :], radius_from_density(m, 1.33),
                  dt=0.01 * YEAR, nsteps=10_000_000)


def random_cluster(seed: int, n: int, spread: float = 0.02, vspread: float = 0.02,
                   mass: float = 1e-6, center_a: float = 1.0) -> System:
    """n bodies packed near a circular orbit at center_a: a small, encounter-rich test system."""
    s = Stream(seed, 9)
    u = s.take(7 * n).reshape(n, 7)
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    x[:, 0] = center_a + spread * (2 * u[:, 0] - 1)
    x[:, 1] = spread * (2 * u[:, 1] - 1)
    x[:, 2] = 0.1 * spread * (2 * u[:, 2] - 1)
    vc = 1.0 / np.sqrt(center_a)
    v[:, 0] = vspread * (2 * u[:, 3] - 1)
    v[:, 1] = vc + vspread * (2 * u[:, 4] - 1)
    v[:, 2] = 0.1 * vspread * (2 * u[:, 5] - 1)
    m = mass * (0.5 + u[:, 6])
    return System(f"cluster_n{n}_seed{seed}", m, x, v, radius_from_density(m, 2.0),
                  dt=0.01 * YEAR, nsteps=100)


CONFIGS = {
    "tiny": tiny,
    "planetesimals_jupiter": planetesimals_jupiter,
    "equal_mass_disk": equal_mass_disk,
    "encounter_heavy": encounter_heavy,
    "embryos_planetesimals": embryos_planetesimals,
}
