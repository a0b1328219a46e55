"""The closest-approach search of the encounter confirmation, restated in
numpy in the precisions the kernel uses (bracket tests and Newton search in
FP32, the path and its derivatives at the root in FP64, the minimum taken as
the local quadratic's |d|^2 - g^2 / g'), against the oracle's FP64
minimum (bisection of g on the same 16 intervals): the two must agree far inside the 1e-9 relative band the GPU's and
the oracle's flagged sets are compared at, also for near head-on passes
whose minimum is tiny.  The GPU parity tests check the kernel itself; this
pins the accuracy of the method it uses.
"""
import numpy as np
import pytest

import oracle

F32 = np.float32


def _hermite(s, d0, tu0, d1, tu1, ft):
    """Relative position on the cubic Hermite path and its first and second
    s-derivatives, in floating type ft (tu = T u, the scaled tangents)."""
    s = ft(s)
    s2 = s * s
    s3 = s2 * s
    h = (ft(2) * s3 - ft(3) * s2 + ft(1), s3 - ft(2) * s2 + s, ft(-2) * s3 + ft(3) * s2, s3 - s2)
    p = (ft(6) * s2 - ft(6) * s, ft(3) * s2 - ft(4) * s + ft(1), ft(-6) * s2 + ft(6) * s, ft(3) * s2 - ft(2) * s)
    q = (ft(12) * s - ft(6), ft(6) * s - ft(4), ft(-12) * s + ft(6), ft(6) * s - ft(2))
    comb = lambda c: c[0] * d0 + c[1] * tu0 + c[2] * d1 + c[3] * tu1
    return comb(h), comb(p), comb(q)


def _interval_min2(T, k, d0, u0, d1, u1):
    f0, f1 = d0.astype(F32), d1.astype(F32)
    tu0, tu1 = (T * u0).astype(F32), (T * u1).astype(F32)
    lo, hi = F32(k / 16.0), F32((k + 1) / 16.0)
    dd, dp, _ = _hermite(lo, f0, tu0, f1, tu1, F32)
    ga = F32(dd @ dp)
    dd, dp, _ = _hermite(hi, f0, tu0, f1, tu1, F32)
    gb = F32(dd @ dp)
    if not (ga < 0 and gb >= 0):
        return np.inf
    s = F32(lo + (hi - lo) * (ga / (ga - gb)))
    if not (lo < s < hi):
        s = F32(0.5) * (lo + hi)
    for _ in range(60):
        dd, dp, d2 = _hermite(s, f0, tu0, f1, tu1, F32)
        g, gp = F32(dd @ dp), F32(dp @ dp + dd @ d2)
        if g < 0:
            lo = s
        else:
            hi = s
        sn = F32(s - g / gp) if gp > 0 else F32(np.nan)
        if not (gp > 0 and lo < sn < hi):
            sn = F32(0.5) * (lo + hi)
        step = F32(sn - s)
        s = sn
        if abs(step) <= F32(1e-7) or hi - lo <= F32(2e-7):
            break
    dd, dp, d2 = _hermite(float(s), d0, T * u0, d1, T * u1, np.float64)
    g, gp = dd @ dp, dp @ dp + dd @ d2
    D = dd @ dd
    if gp > 0:
        D -= g * g / gp
    return max(float(D), 0.0)


def _min_over_path(T, d0, u0, d1, u1):
    D = min(d0 @ d0, d1 @ d1)
    for k in range(16):
        D = min(D, _interval_min2(T, k, d0, u0, d1, u1))
    return D


@pytest.mark.parametrize("kind", ["random", "head_on"])
def test_fp32_search_with_fp64_polish_matches_the_oracle(kind):
    oracle.build()
    rng = np.random.default_rng(3 if kind == "random" else 4)
    T = 0.0628
    worst = 0.0
    for _ in range(400):
        d0 = rng.normal(size=3) * 0.02
        if kind == "random":
            u0 = rng.normal(size=3) * 0.3
            d1 = -d0 * rng.uniform(0.2, 1.5) + rng.normal(size=3) * 0.005
            u1 = u0 + rng.normal(size=3) * 0.05
        else:
            u0 = -d0 / T * rng.uniform(0.5, 3.0) + rng.normal(size=3) * 1e-4
            d1 = d0 + T * u0 + rng.normal(size=3) * 1e-6
            u1 = u0 + rng.normal(size=3) * 1e-5
        ref = oracle.min_sep2(T, d0, u0, d1, u1)
        got = _min_over_path(T, d0, u0, d1, u1)
        worst = max(worst, abs(got - ref) / ref)
    assert worst <= 1e-10, worst
