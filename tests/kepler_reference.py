"""High-precision two-body propagation by the classical eccentric-anomaly route.

An independent reference for the universal-variable drift: it never uses
Stumpff functions.  For an ellipse (a > 0) it solves the difference form of
Kepler's equation for dE,
    n dt = dE - (1 - r0/a) sin dE + (x.v / sqrt(mu a)) (1 - cos dE),
and for a hyperbola (a < 0) the analogue in dF,
    n dt = (x.v / sqrt(-mu a)) (cosh dF - 1) + (1 - r0/a) sinh dF - dF,
by bisection in mpmath at 50 digits, then applies the Gauss f and g
functions written with the anomaly difference (Danby, Fundamentals of
Celestial Mechanics, ch. 6).
"""
import mpmath as mp


def _bisect(fun, lo, hi, iters=400):
    flo = fun(lo)
    if (flo < 0) == (fun(hi) < 0):
        raise ValueError("root not bracketed")
    for _ in range(iters):
        mid = (lo + hi) / 2
        fm = fun(mid)
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return (lo + hi) / 2


def propagate(mu, dt, x, v, dps=50):
    with mp.workdps(dps):
        mu, dt = mp.mpf(mu), mp.mpf(dt)
        x = [mp.mpf(t) for t in x]
        v = [mp.mpf(t) for t in v]
        r0 = mp.sqrt(sum(t * t for t in x))
        v2 = sum(t * t for t in v)
        eta = sum(a * b for a, b in zip(x, v))
        a = 1 / (2 / r0 - v2 / mu)
        if a > 0:
            n = mp.sqrt(mu / a ** 3)
            s0 = eta / mp.sqrt(mu * a)
            c0 = 1 - r0 / a

            def kep(dE):
                return dE - c0 * mp.sin(dE) + s0 * (1 - mp.cos(dE)) - n * dt

            span = abs(n * dt) + 4
            dE = _bisect(kep, -span, span)
            f = 1 - a / r0 * (1 - mp.cos(dE))
            g = dt - (dE - mp.sin(dE)) / n
            x1 = [f * p + g * q for p, q in zip(x, v)]
            r1 = mp.sqrt(sum(t * t for t in x1))
            fd = -mp.sqrt(mu * a) * mp.sin(dE) / (r1 * r0)
            gd = 1 - a / r1 * (1 - mp.cos(dE))
        else:
            n = mp.sqrt(mu / (-a) ** 3)
            s0 = eta / mp.sqrt(-mu * a)
            c0 = 1 - r0 / a

            def kep(dF):
                return s0 * (mp.cosh(dF) - 1) + c0 * mp.sinh(dF) - dF - n * dt

            span = mp.asinh(abs(n * dt) + 1) + 4
            dF = _bisect(kep, -span, span)
            f = 1 - a / r0 * (1 - mp.cosh(dF))
            g = dt - (mp.sinh(dF) - dF) / n
            x1 = [f * p + g * q for p, q in zip(x, v)]
            r1 = mp.sqrt(sum(t * t for t in x1))
            fd = -mp.sqrt(-mu * a) * mp.sinh(dF) / (r1 * r0)
            gd = 1 - a / r1 * (1 - mp.cosh(dF))
        v1 = [fd * p + gd * q for p, q in zip(x, v)]
        return [float(t) for t in x1], [float(t) for t in v1]
