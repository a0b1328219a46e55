/*
 * Oracle for the hybrid symplectic N-body step -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain serial FP64 C, written for a reader to check against the method by
 * eye.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
 * load it; the CUDA library never links or calls it, and the two share no
 * code.  Each function names the passage of the paper it follows.  Where the
 * paper is silent (it defers the mathematics of the integrator to Chambers
 * 1999), the reading taken is stated beside the code.
 *
 * Paper map (Simonetti et al., "Mercury-Opal", Sec. 2.1.1 and Sec. 3.1):
 *   - democratic heliocentric coordinates: Sec. 2.1.1, footnote 1;
 *   - kick with the changeover-weighted mutual forces: Sec. 3.1, force block,
 *     LOOP 2, and the critical-radius footnote of Sec. 2.1.1;
 *   - jump (stellar Hamiltonian) and the momentum reduction: Sec. 3.1,
 *     Hamiltonian block, LOOPs 1-4;
 *   - Keplerian drift of every body: Sec. 3.1, third block (WHFast lineage,
 *     universal variables);
 *   - Hill and critical radii: Sec. 2.1.1, items (4) and footnote 2;
 *   - close-encounter scan (minimum separation over the step against the
 *     critical distance): Sec. 3.1, mce_snif block, LOOPs 1-3;
 *   - Bulirsch-Stoer integration of the bodies in close encounter from the
 *     saved start-of-drift state, with collisions: Sec. 2.1.1 footnote 2,
 *     Sec. 3.2 data-management listing, Sec. 2.1.2 (mce_coll);
 *   - energy and momentum: Sec. 2.1.1 item (7);
 *   - star collisions and ejections (Sec. 2.1.2: mce_cent, and bodies beyond
 *     400 au removed every 200 yr): a body whose Kepler drift passes within
 *     the star's radius is accreted at the end of the step (M0 grows by its
 *     mass, the heliocentric frame moves to the merged star); every
 *     eject_every steps, bodies beyond r_eject are removed.  The energy each
 *     removal takes out of the Hamiltonian is added to E_lost;
 *   - small bodies (Sec. 2.1): bodies of zero mass are massless particles
 *     that feel the star and the big bodies (mass > 0) but are the source of
 *     no force; two small bodies never interact, so a pair of them is never
 *     flagged, never integrated together and never merged.
 *
 * Pins: every function here is checked by tests/test_oracle_*.py against
 * closed forms, brute force at high precision, conservation laws and the
 * numbers the paper prints; none is "parity unpinned".
 */
#include "opal_oracle.h"

#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* Neumaier's compensated summation (a plain accumulator with a carry). */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double nval(const nsum* a) { return a->s + a->c; }

/* ---------------------------------------------------------------------- */
/* Coordinates (Sec. 2.1.1, footnote 1): democratic heliocentric = heliocentric
 * positions with barycentric velocities.  With heliocentric velocities v_i,
 * the barycentric velocity of body i is V_i = v_i - sum_j m_j v_j / (M0 + sum m),
 * and the inverse is v_i = V_i + sum_j m_j V_j / M0. */
void orc_helio_to_dh(int64_t n, double M0, const double* m, const double* v, double* V) {
    double Mtot = M0, S[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        Mtot += m[i];
        for (int k = 0; k < 3; k++) S[k] += m[i] * v[3 * i + k];
    }
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) V[3 * i + k] = v[3 * i + k] - S[k] / Mtot;
}

void orc_dh_to_helio(int64_t n, double M0, const double* m, const double* V, double* v) {
    double P[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) P[k] += m[i] * V[3 * i + k];
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) v[3 * i + k] = V[3 * i + k] + P[k] / M0;
}

/* ---------------------------------------------------------------------- */
/* Changeover function K(r; rc) splitting each pair's force between the kick
 * (weight K) and the encounter integrator (weight 1 - K).  The paper names
 * the critical radius only (Sec. 2.1.1, footnote 2); the form is the one of
 * the hybrid integrator it cites (Chambers 1999): y = (r - 0.1 rc)/(0.9 rc),
 * K = 0 for y <= 0, K = 1 for r >= rc, and in between the rational
 * y^2 / (2y^2 - 2y + 1) (form 0) or the quintic 10y^3 - 15y^4 + 6y^5 (form 1). */
double orc_changeover(double r, double rc, int32_t form) {
    if (r >= rc) return 1.0;
    double y = (r - 0.1 * rc) / (0.9 * rc);
    if (y <= 0.0) return 0.0;
    if (form == 0) return y * y / (2.0 * y * y - 2.0 * y + 1.0);
    return y * y * y * (10.0 - 15.0 * y + 6.0 * y * y);
}

/* Hill radius from the instantaneous heliocentric distance, and the critical
 * radius as a multiple of it (Sec. 2.1.1, item 4 and footnotes 2-3):
 * R_H = |x| (m / 3 M0)^(1/3), rc = f_hill R_H. */
void orc_hill_rcrit(int64_t n, double M0, double f_hill, const double* m, const double* x,
                    const int32_t* alive, double* rc) {
    for (int64_t i = 0; i < n; i++)
        rc[i] = alive[i] ? f_hill * norm3(x + 3 * i) * cbrt(m[i] / (3.0 * M0)) : 0.0;
}

/* Mutual accelerations of the kick (Sec. 3.1, force block, LOOP 2):
 * a_i = sum_{j != i} G m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3, with
 * rc_ij = max(rc_i, rc_j).  Each a_i is summed over j in increasing order;
 * small bodies (m_j = 0) are no source and are left out of the sum (Sec. 2.1:
 * only the big bodies are gravity sources). */
void orc_accel(int64_t n, double G, int32_t form, const double* m, const double* x,
               const double* rc, const int32_t* alive, double* a) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        double ai[3] = {0, 0, 0};
        if (alive[i]) {
            for (int64_t j = 0; j < n; j++) {
                if (j == i || !alive[j] || m[j] == 0.0) continue;
                double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
                double r2 = dot3(d, d);
                double r = sqrt(r2);
                double rcij = rc[i] > rc[j] ? rc[i] : rc[j];
                double K = orc_changeover(r, rcij, form);
                double s = G * m[j] * K / (r2 * r);
                for (int k = 0; k < 3; k++) ai[k] += s * d[k];
            }
        }
        for (int k = 0; k < 3; k++) a[3 * i + k] = ai[k];
    }
}

/* ---------------------------------------------------------------------- */
/* Stumpff functions c_0..c_3 of the universal-variable Kepler solution used
 * by the drift (Sec. 3.1, third block; WHFast lineage).  c_k(z) is the series
 * sum_j (-z)^j / (k + 2j)!.  Arguments with |z| > 0.1 are first divided by 4
 * until small; each c_k is summed there as the series itself, ten terms
 * nested from the innermost, c_k = (1 - z/((k+1)(k+2)) (1 - z/((k+3)(k+4)) (...))) / k!,
 * and the quartering is undone with the double-angle relations
 *   c0(4z) = 2 c0^2 - 1,  c1(4z) = c0 c1,  c2(4z) = c1^2 / 2,
 *   c3(4z) = (c2 + c0 c3) / 4. */
void orc_stumpff(double z, double c[4]) {
    int nq = 0;
    while (fabs(z) > 0.1) {
        z *= 0.25;
        nq++;
    }
    static const double fact[4] = {1.0, 1.0, 2.0, 6.0};
    for (int k = 0; k < 4; k++) {
        double s = 1.0;
        for (int j = 10; j >= 1; j--) s = 1.0 - z * s / (double)((k + 2 * j - 1) * (k + 2 * j));
        c[k] = s / fact[k];
    }
    for (; nq > 0; nq--) {
        c[3] = (c[2] + c[0] * c[3]) * 0.25;
        c[2] = c[1] * c[1] * 0.5;
        c[1] = c[0] * c[1];
        c[0] = 2.0 * c[0] * c[0] - 1.0;
    }
}

/* Keplerian drift of one body over dt about a central mass with mu = G M0
 * (Sec. 3.1, third block; arxes_drift reports failure through iflag).
 * Universal variable chi with G_k = chi^k c_k(beta chi^2):
 *   r0 = |x|, eta = x.v, beta = 2 mu / r0 - v^2,
 *   F(chi) = r0 G1 + eta G2 + mu G3 - dt = 0,  F' = r = r0 G0 + eta G1 + mu G2.
 * F is increasing (F' = r > 0) and F' >= q, the pericentre distance, so the
 * root lies in [0, dt/q] (dt > 0; mirrored for dt < 0).  Newton from
 * chi = dt / r0 (bound orbits) or the logarithmic start of Vallado's
 * Algorithm 8 (unbound orbits) keeps that bracket up to date and bisects whenever a Newton
 * step would leave it; converged when |dchi| <= 1e-15 |chi|, or when |dchi|
 * is below 1e-12 |chi| and no smaller than the step before.  A bound orbit
 * first drops whole periods P = 2 pi mu / beta^1.5 from dt (the state repeats).
 * The Gauss functions f = 1 - mu G2 / r0, g = dt - mu G3,
 * fdot = -mu G1 / (r r0), gdot = 1 - mu G2 / r give x' = f x + g v,
 * v' = fdot x + gdot v.  Returns ORC_EKEPLER (state untouched) if max_iter
 * iterations do not converge. */
int32_t orc_kepler_drift(double mu, double dt, double x[3], double v[3], int32_t max_iter,
                         int32_t* iters) {
    if (max_iter <= 0) max_iter = 50;
    double r0 = norm3(x), v2 = dot3(v, v), eta = dot3(x, v);
    double beta = 2.0 * mu / r0 - v2;
    if (beta > 0.0) {
        double period = 2.0 * M_PI * mu / (beta * sqrt(beta));
        if (fabs(dt) > period) dt = fmod(dt, period);
    }
    double h[3] = {x[1] * v[2] - x[2] * v[1], x[2] * v[0] - x[0] * v[2], x[0] * v[1] - x[1] * v[0]};
    double p = dot3(h, h) / mu;
    double ecc2 = 1.0 - p * beta / mu;
    double q = p / (1.0 + sqrt(ecc2 > 0.0 ? ecc2 : 0.0));
    double lo, hi;
    if (dt >= 0.0) {
        lo = 0.0;
        hi = q > 0.0 ? dt / q : HUGE_VAL;
    } else {
        lo = q > 0.0 ? dt / q : -HUGE_VAL;
        hi = 0.0;
    }
    double chi = dt / r0, c[4];
    if (beta < 0.0) {
        /* unbound orbit: the logarithmic starting value of the universal
         * variable (Vallado, Fundamentals of Astrodynamics, Algorithm 8),
         * with a = mu / beta < 0; kept only when its logarithm is defined */
        double a = mu / beta, sg = dt >= 0.0 ? 1.0 : -1.0;
        double den = eta + sg * sqrt(-mu * a) * (1.0 - r0 / a);
        double arg = -2.0 * beta * dt / den;
        if (den != 0.0 && arg > 0.0 && isfinite(arg)) chi = sg * sqrt(-a / mu) * log(arg);
    }
    if (chi < lo) chi = lo;
    if (chi > hi) chi = hi;
    int conv = 0, it;
    double dchi_prev = HUGE_VAL;
    for (it = 1; it <= max_iter; it++) {
        orc_stumpff(beta * chi * chi, c);
        double G0 = c[0], G1 = chi * c[1], G2 = chi * chi * c[2], G3 = chi * chi * chi * c[3];
        double F = r0 * G1 + eta * G2 + mu * G3 - dt;
        double dF = r0 * G0 + eta * G1 + mu * G2;
        if (F < 0.0) lo = chi;
        else hi = chi;
        double chin = chi - F / dF;
        if (!(chin >= lo && chin <= hi)) chin = 0.5 * (lo + hi);
        double dchi = chin - chi;
        chi = chin;
        /* done when the step is at the 1e-15 level, or when it has stopped
         * shrinking while below 1e-12 (F is then at its rounding floor) */
        if (fabs(dchi) <= 1e-15 * fabs(chi) ||
            (fabs(dchi) <= 1e-12 * fabs(chi) && fabs(dchi) >= dchi_prev)) {
            conv = 1;
            break;
        }
        dchi_prev = fabs(dchi);
    }
    if (iters) *iters = conv ? it : max_iter;
    if (!conv) return ORC_EKEPLER;
    orc_stumpff(beta * chi * chi, c);
    double G0 = c[0], G1 = chi * c[1], G2 = chi * chi * c[2], G3 = chi * chi * chi * c[3];
    double r = r0 * G0 + eta * G1 + mu * G2;
    double f = 1.0 - mu * G2 / r0, g = dt - mu * G3;
    double fd = -mu * G1 / (r * r0), gd = 1.0 - mu * G2 / r;
    double xn[3], vn[3];
    for (int k = 0; k < 3; k++) {
        xn[k] = f * x[k] + g * v[k];
        vn[k] = fd * x[k] + gd * v[k];
    }
    for (int k = 0; k < 3; k++) {
        x[k] = xn[k];
        v[k] = vn[k];
    }
    return ORC_OK;
}

/* Closest approach to the star during a body's drift from (x0, V0) to
 * (x1, V1) over dt on its Kepler orbit about mu (the star-collision test,
 * Sec. 2.1.2 mce_cent): the pericentre distance q = p / (1 + e) when the
 * pericentre is passed within the drift, else the nearer end.  The passage
 * is read off the mean anomaly, which advances uniformly: on an ellipse
 * (beta = 2 mu / r - v^2 > 0, a = mu / beta) M = E - e sin E with
 * e cos E = 1 - r / a and e sin E = x.V / sqrt(mu a), and the pericentre is at
 * M = 2 pi k; on a hyperbola M = e sinh F - F with e sinh F = x.V / sqrt(-mu a),
 * and the pericentre is at M = 0.  The swept interval is [M0, M0 + n dt]. */
double orc_drift_min_r(double mu, double dt, const double x0[3], const double V0[3], const double x1[3],
                       const double V1[3]) {
    const double r0 = norm3(x0), r1 = norm3(x1);
    double rmin = r0 < r1 ? r0 : r1;
    const double eta0 = dot3(x0, V0);
    const double beta = 2.0 * mu / r0 - dot3(V0, V0);
    const double h[3] = {x0[1] * V0[2] - x0[2] * V0[1], x0[2] * V0[0] - x0[0] * V0[2],
                         x0[0] * V0[1] - x0[1] * V0[0]};
    const double p = dot3(h, h) / mu;
    const double e2 = 1.0 - p * beta / mu;
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    const double q = p / (1.0 + e);
    int passed = 0;
    (void)V1;
    if (beta > 0.0) {
        const double a = mu / beta, n = sqrt(mu / (a * a * a));
        const double ecE = 1.0 - r0 / a, esE = eta0 / sqrt(mu * a);
        const double M0 = atan2(esE, ecE) - esE, M1 = M0 + n * dt;
        const double lo = M0 < M1 ? M0 : M1, hi = M0 < M1 ? M1 : M0;
        passed = 2.0 * M_PI * ceil(lo / (2.0 * M_PI)) <= hi;
    } else if (beta < 0.0) {
        const double a = mu / beta, n = sqrt(mu / (-a * a * a));
        const double esF = eta0 / sqrt(-mu * a);
        const double F0 = e > 0.0 ? asinh(esF / e) : 0.0;
        const double M0 = esF - F0, M1 = M0 + n * dt;
        passed = (M0 <= 0.0 && M1 >= 0.0) || (M0 >= 0.0 && M1 <= 0.0);
    } else {
        passed = (dt * eta0 < 0.0) && (dt * dot3(x1, V1) >= 0.0);   /* parabolic: x.V turns outward */
    }
    if (passed && q < rmin) rmin = q;
    return rmin;
}

/* ---------------------------------------------------------------------- */
/* Minimum separation of a pair over the step (Sec. 3.1, mce_snif LOOP 3,
 * "minimal separation between each couple of bodies"; the routine is mce_min).
 * Reading: the relative path over the step is the cubic Hermite interpolant
 * of the relative position d and velocity u at its two ends,
 *   d(s) = h00 d0 + h10 T u0 + h01 d1 + h11 T u1,  s in [0, 1], T = dt,
 * written here in powers of s (collecting the basis polynomials
 * h00 = 2s^3 - 3s^2 + 1, h10 = s^3 - 2s^2 + s, h01 = -2s^3 + 3s^2, h11 = s^3 - s^2):
 *   d(s) = A + B s + C s^2 + D s^3,  A = d0,  B = T u0,
 *   C = 3 (d1 - d0) - T (2 u0 + u1),  D = 2 (d0 - d1) + T (u0 + u1).
 * The result is min over s of |d(s)|^2: the two ends, and every local minimum
 * inside.  Those lie where g(s) = d.d' = (1/2) d|d|^2/ds, the quintic
 *   g = A.B + (2 A.C + B.B) s + 3 (A.D + B.C) s^2 + (4 B.D + 2 C.C) s^3
 *       + 5 C.D s^4 + 3 D.D s^5,
 * changes sign from - to + ; the sign is read on a grid of 16 equal intervals
 * and each such interval is halved 48 times (bisection: the root is then
 * known to 2^-52 of the step). */
static double poly_g(const double g[6], double s) {
    return g[0] + s * (g[1] + s * (g[2] + s * (g[3] + s * (g[4] + s * g[5]))));
}

double orc_min_sep2(double T, const double d0[3], const double u0[3], const double d1[3],
                    const double u1[3]) {
    double A[3], B[3], Cc[3], D[3];
    for (int k = 0; k < 3; k++) {
        A[k] = d0[k];
        B[k] = T * u0[k];
        Cc[k] = 3.0 * (d1[k] - d0[k]) - T * (2.0 * u0[k] + u1[k]);
        D[k] = 2.0 * (d0[k] - d1[k]) + T * (u0[k] + u1[k]);
    }
    const double g[6] = {dot3(A, B), 2.0 * dot3(A, Cc) + dot3(B, B), 3.0 * (dot3(A, D) + dot3(B, Cc)),
                         4.0 * dot3(B, D) + 2.0 * dot3(Cc, Cc), 5.0 * dot3(Cc, D), 3.0 * dot3(D, D)};
    double Dmin = dot3(d0, d0), D1 = dot3(d1, d1);
    if (D1 < Dmin) Dmin = D1;
    double ga = poly_g(g, 0.0);
    for (int k = 0; k < 16; k++) {
        const double sa = k / 16.0, sb = (k + 1) / 16.0;
        const double gb = poly_g(g, sb);
        if (ga < 0.0 && gb >= 0.0) {
            double lo = sa, hi = sb;
            for (int it = 0; it < 48; it++) {
                const double mid = 0.5 * (lo + hi);
                if (poly_g(g, mid) < 0.0) lo = mid;
                else hi = mid;
            }
            const double s = 0.5 * (lo + hi);
            double d[3];
            for (int q = 0; q < 3; q++) d[q] = A[q] + s * (B[q] + s * (Cc[q] + s * D[q]));
            const double Dm = dot3(d, d);
            if (Dm < Dmin) Dmin = Dm;
        }
        ga = gb;
    }
    return Dmin;
}

/* Close-encounter scan (Sec. 3.1, mce_snif LOOPs 1-3): for every pair i < j
 * of live bodies, flag it when the minimum separation over the step is <=
 * the critical distance rc_ij = max(rc_i, rc_j) (the comparison is ".le.").
 * x0, V0 are the saved start-of-drift state (Sec. 3.1, third block), x1, V1
 * the state after the drift.  Pairs are listed with i ascending, then j.
 * Two small bodies (m = 0 both; m may be NULL: no small bodies) are never a
 * pair: they do not interact (Sec. 2.1).
 *
 * prune = 0 runs the exact test on every pair.  prune = 1 first skips the
 * pairs that one bound rules out; it only saves time, the flagged set is the
 * exact test's (the tests check the two modes give the same set):
 * during the drift dx/dt = V, and the interpolant of body i's own path
 * p(s) = h00 x0 + h10 T V0 + h01 x1 + h11 T V1 satisfies
 * p(s) - x1 = h00 (x0 - x1) + h10 T V0 + h11 T V1 (h00 + h01 = 1), with
 * |h00| <= 1 and |h10|, |h11| <= 4/27 on [0, 1]; so p stays within
 * rho = |x0 - x1| + (4/27)|T|(|V0| + |V1|) of x1, and
 * |d(s)| >= |x1_j - x1_i| - rho_i - rho_j.
 * Returns the number of flagged pairs (the first min(count, cap) are written);
 * n_candidates gets the number of pairs given the exact test. */
int64_t orc_scan(int64_t n, double T, const double* x0, const double* V0, const double* x1,
                 const double* V1, const double* rc, const int32_t* alive, const double* m, int32_t prune,
                 int64_t cap, int32_t* pi, int32_t* pj, int64_t* n_candidates) {
    double* rho = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        double w[3] = {x0[3 * i] - x1[3 * i], x0[3 * i + 1] - x1[3 * i + 1], x0[3 * i + 2] - x1[3 * i + 2]};
        rho[i] = norm3(w) + (4.0 / 27.0) * fabs(T) * (norm3(V0 + 3 * i) + norm3(V1 + 3 * i));
    }
    int64_t count = 0, ncand = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!alive[i]) continue;
        for (int64_t j = i + 1; j < n; j++) {
            if (!alive[j]) continue;
            if (m && m[i] == 0.0 && m[j] == 0.0) continue; /* two small bodies */
            double rcij = rc[i] > rc[j] ? rc[i] : rc[j];
            double d0[3], u0[3], d1[3], u1[3];
            for (int k = 0; k < 3; k++) {
                d0[k] = x0[3 * j + k] - x0[3 * i + k];
                u0[k] = V0[3 * j + k] - V0[3 * i + k];
                d1[k] = x1[3 * j + k] - x1[3 * i + k];
                u1[k] = V1[3 * j + k] - V1[3 * i + k];
            }
            if (prune) {
                double r1 = norm3(d1);
                if (r1 - rho[i] - rho[j] > rcij + 1e-12 * (r1 + rho[i] + rho[j])) continue;
            }
            ncand++;
            double D = orc_min_sep2(T, d0, u0, d1, u1);
            if (D <= rcij * rcij) {
                if (count < cap) {
                    pi[count] = (int32_t)i;
                    pj[count] = (int32_t)j;
                }
                count++;
            }
        }
    }
    free(rho);
    if (n_candidates) *n_candidates = ncand;
    return count;
}

/* Encounter groups: connected components of the graph of flagged pairs (the
 * paper hands all pairs to one BS call, Sec. 3.2 listing; integrating each
 * component on its own is the same ODE, since bodies in different components
 * have no (1 - K) coupling).  label[i] = lowest body index of i's component,
 * or -1 if i is in no pair.  Returns the number of groups. */
static int64_t uf_find(int32_t* parent, int64_t i) {
    while (parent[i] != i) {
        parent[i] = parent[parent[i]];
        i = parent[i];
    }
    return i;
}

int64_t orc_groups(int64_t n, int64_t npairs, const int32_t* pi, const int32_t* pj, int32_t* label) {
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        parent[i] = (int32_t)i;
        label[i] = -1;
    }
    for (int64_t p = 0; p < npairs; p++) {
        int64_t a = uf_find(parent, pi[p]), b = uf_find(parent, pj[p]);
        if (a == b) continue;
        if (a < b) parent[b] = (int32_t)a;
        else parent[a] = (int32_t)b;
    }
    for (int64_t p = 0; p < npairs; p++) {
        label[pi[p]] = (int32_t)uf_find(parent, pi[p]);
        label[pj[p]] = (int32_t)uf_find(parent, pj[p]);
    }
    int64_t ng = 0;
    for (int64_t i = 0; i < n; i++)
        if (label[i] == i) ng++;
    free(parent);
    return ng;
}

/* ---------------------------------------------------------------------- */
/* Bulirsch-Stoer integration of one encounter group over the step (Sec. 2.1.1
 * footnote 2: the interaction and Keplerian Hamiltonians of the bodies in the
 * encounter are advanced by BS; Sec. 3.2: from the saved x0, v0).
 * Equations: dx_b/dt = V_b,
 *   dV_b/dt = -G M0 x_b/|x_b|^3 + sum_{c in group, c != b} G m_c (1 - K) (x_c - x_b)/r^3.
 * Substep: modified midpoint with n_k = 2, 4, ..., 16 steps, Neville
 * extrapolation in h^2; row k is accepted when
 *   max_b max(|dX_b|/|X_b|, |dV_b|/|V_b|) <= bs_tol,
 * with d = T[k][k] - T[k][k-1].  Step control: the first substep is the whole
 * step; after acceptance at row k <= 2 the next substep doubles, at k >= 6 it
 * halves; a substep not accepted by row 7 is retried at half length.
 * Collisions (mce_coll, Sec. 2.1.2) are tested after each accepted substep:
 * |x_b - x_c| <= R_b + R_c merges the pair perfectly (mass, momentum and
 * centre of mass kept; R = cbrt(R_b^3 + R_c^3); survivor = heavier body, the
 * lower index on a tie).  E_lost gets the change of the pair's kinetic,
 * central and mutual energy. */
typedef struct {
    int64_t nm;
    const orc_params* p;
    double *mm, *Rm, *rcm;
    int32_t* am;
    const int32_t* gid;
} bs_ctx;

static void bs_deriv(const bs_ctx* c, const double* y, double* f) {
    const int64_t nm = c->nm;
    const double* X = y;
    const double* V = y + 3 * nm;
    double* fX = f;
    double* fV = f + 3 * nm;
    const double G = c->p->G, M0 = c->p->M0;
    for (int64_t b = 0; b < nm; b++) {
        if (!c->am[b]) {
            for (int k = 0; k < 3; k++) fX[3 * b + k] = fV[3 * b + k] = 0.0;
            continue;
        }
        const double* xb = X + 3 * b;
        double r2 = dot3(xb, xb), r = sqrt(r2);
        double s = -G * M0 / (r2 * r);
        double acc[3] = {s * xb[0], s * xb[1], s * xb[2]};
        for (int64_t q = 0; q < nm; q++) {
            if (q == b || !c->am[q] || c->mm[q] == 0.0) continue; /* a small body pulls nothing */
            double d[3] = {X[3 * q] - xb[0], X[3 * q + 1] - xb[1], X[3 * q + 2] - xb[2]};
            double dr2 = dot3(d, d), dr = sqrt(dr2);
            double rcbq = c->rcm[b] > c->rcm[q] ? c->rcm[b] : c->rcm[q];
            double wgt = 1.0 - orc_changeover(dr, rcbq, c->p->changeover);
            if (wgt == 0.0) continue;
            double t = G * c->mm[q] * wgt / (dr2 * dr);
            for (int k = 0; k < 3; k++) acc[k] += t * d[k];
        }
        for (int k = 0; k < 3; k++) {
            fX[3 * b + k] = V[3 * b + k];
            fV[3 * b + k] = acc[k];
        }
    }
}

/* modified midpoint: n steps of h = H/n from y0 */
static void bs_mmid(const bs_ctx* c, const double* y0, double H, int n, double* out, double* za,
                    double* zb, double* f) {
    const int64_t q = 6 * c->nm;
    double h = H / n;
    bs_deriv(c, y0, f);
    for (int64_t i = 0; i < q; i++) {
        za[i] = y0[i];
        zb[i] = y0[i] + h * f[i];
    }
    for (int s = 1; s < n; s++) {
        bs_deriv(c, zb, f);
        for (int64_t i = 0; i < q; i++) {
            double znew = za[i] + 2.0 * h * f[i];
            za[i] = zb[i];
            zb[i] = znew;
        }
    }
    bs_deriv(c, zb, f);
    for (int64_t i = 0; i < q; i++) out[i] = 0.5 * (zb[i] + za[i] + h * f[i]);
}

static void bs_merge(bs_ctx* c, double* y, int64_t b, int64_t q, double* E_lost) {
    const double G = c->p->G, M0 = c->p->M0;
    const int64_t nm = c->nm;
    double* X = y;
    double* V = y + 3 * nm;
    double mb = c->mm[b], mq = c->mm[q], M = mb + mq;
    double d[3] = {X[3 * q] - X[3 * b], X[3 * q + 1] - X[3 * b + 1], X[3 * q + 2] - X[3 * b + 2]};
    double xn[3], vn[3];
    for (int k = 0; k < 3; k++) {
        xn[k] = (mb * X[3 * b + k] + mq * X[3 * q + k]) / M;
        vn[k] = (mb * V[3 * b + k] + mq * V[3 * q + k]) / M;
    }
    double e_before = 0.5 * mb * dot3(V + 3 * b, V + 3 * b) + 0.5 * mq * dot3(V + 3 * q, V + 3 * q)
                      - G * M0 * mb / norm3(X + 3 * b) - G * M0 * mq / norm3(X + 3 * q)
                      - G * mb * mq / norm3(d);
    double e_after = 0.5 * M * dot3(vn, vn) - G * M0 * M / norm3(xn);
    *E_lost += e_before - e_after;
    int64_t keep, gone;
    if (mb > mq) keep = b, gone = q;
    else if (mq > mb) keep = q, gone = b;
    else keep = (c->gid[b] < c->gid[q]) ? b : q, gone = (keep == b) ? q : b;
    double Rn = cbrt(c->Rm[b] * c->Rm[b] * c->Rm[b] + c->Rm[q] * c->Rm[q] * c->Rm[q]);
    for (int k = 0; k < 3; k++) {
        X[3 * keep + k] = xn[k];
        V[3 * keep + k] = vn[k];
    }
    c->mm[keep] = M;
    c->Rm[keep] = Rn;
    c->mm[gone] = 0.0;
    c->am[gone] = 0;
}

int32_t orc_bs_group(const orc_params* p, int64_t nm, const int32_t* members, double* m, double* R,
                     const double* rc, int32_t* alive, double* x, double* V, double* E_lost,
                     int64_t* n_mergers, int64_t* substeps) {
    const int KMAX = 8;
    const int64_t q = 6 * nm;
    double* mem = (double*)malloc(sizeof(double) * (size_t)(q * (KMAX * KMAX + 4) + 3 * nm));
    double* y = mem;                       /* current state: X (3 nm) then V (3 nm) */
    double* Tb = y + q;                    /* tableau, T[k][j] at Tb + (k*KMAX + j)*q */
    double* za = Tb + (int64_t)KMAX * KMAX * q;
    double* zb = za + q;
    double* f = zb + q;
    double* mm = f + q;
    double* Rm = mm + nm;
    double* rcm = Rm + nm;
    int32_t* am = (int32_t*)malloc(sizeof(int32_t) * (size_t)nm);
    for (int64_t b = 0; b < nm; b++) {
        int64_t g = members[b];
        for (int k = 0; k < 3; k++) {
            y[3 * b + k] = x[3 * g + k];
            y[3 * nm + 3 * b + k] = V[3 * g + k];
        }
        mm[b] = m[g];
        Rm[b] = R[g];
        rcm[b] = rc[g];
        am[b] = alive[g];
    }
    bs_ctx c = {nm, p, mm, Rm, rcm, am, members};
    const double dt = p->dt, tol = p->bs_tol;
    const int64_t cap = p->bs_max_substeps > 0 ? p->bs_max_substeps : (1 << 20);
    double t = 0.0, H = dt;
    int64_t nsub = 0;
    int32_t status = ORC_OK;
    for (;;) {
        double rem = dt - t;
        int last = 0;
        if (fabs(H) >= fabs(rem)) {
            H = rem;
            last = 1;
        }
        int kacc = -1;
        for (int k = 0; k < KMAX; k++) {
            double* Tk0 = Tb + (int64_t)(k * KMAX) * q;
            bs_mmid(&c, y, H, 2 * (k + 1), Tk0, za, zb, f);
            for (int j = 1; j <= k; j++) {
                double* Tkj = Tb + (int64_t)(k * KMAX + j) * q;
                double* Tkj1 = Tb + (int64_t)(k * KMAX + j - 1) * q;
                double* Tpj1 = Tb + (int64_t)((k - 1) * KMAX + j - 1) * q;
                /* Neville's recurrence in h^2: T_kj = T_k,j-1 + (T_k,j-1 - T_k-1,j-1) / ((n_k / n_k-j)^2 - 1) */
                double ratio = (double)(k + 1) / (double)(k - j + 1);
                double den = ratio * ratio - 1.0;
                for (int64_t i = 0; i < q; i++) Tkj[i] = Tkj1[i] + (Tkj1[i] - Tpj1[i]) / den;
            }
            if (k >= 1) {
                double* Tkk = Tb + (int64_t)(k * KMAX + k) * q;
                double* Tkm = Tb + (int64_t)(k * KMAX + k - 1) * q;
                double err = 0.0;
                for (int64_t b = 0; b < nm; b++) {
                    if (!am[b]) continue;
                    for (int part = 0; part < 2; part++) {
                        int64_t o = part * 3 * nm + 3 * b;
                        double dv[3] = {Tkk[o] - Tkm[o], Tkk[o + 1] - Tkm[o + 1], Tkk[o + 2] - Tkm[o + 2]};
                        double sc = norm3(Tkk + o);
                        if (sc < 1e-300) sc = 1e-300;
                        double e = norm3(dv) / sc;
                        if (!(e <= err)) err = e; /* NaN propagates as "not converged" */
                    }
                }
                if (err <= tol) {
                    kacc = k;
                    break;
                }
            }
        }
        nsub++;
        if (substeps) (*substeps)++;
        if (kacc >= 0) {
            memcpy(y, Tb + (int64_t)(kacc * KMAX + kacc) * q, sizeof(double) * (size_t)q);
            t = last ? dt : t + H;
            for (int64_t b = 0; b < nm; b++) {
                for (int64_t e = b + 1; e < nm && am[b]; e++) {
                    if (!am[e] || (mm[b] == 0.0 && mm[e] == 0.0)) continue; /* two small bodies never touch */
                    double d[3] = {y[3 * e] - y[3 * b], y[3 * e + 1] - y[3 * b + 1], y[3 * e + 2] - y[3 * b + 2]};
                    if (norm3(d) <= Rm[b] + Rm[e]) {
                        bs_merge(&c, y, b, e, E_lost);
                        if (n_mergers) (*n_mergers)++;
                    }
                }
            }
            if (last) break;
            if (kacc <= 2) H *= 2.0;
            else if (kacc >= 6) H *= 0.5;
        } else {
            H *= 0.5;
        }
        if (nsub >= cap) {
            status = ORC_EBS;
            break;
        }
    }
    if (status == ORC_OK) {
        for (int64_t b = 0; b < nm; b++) {
            int64_t g = members[b];
            for (int k = 0; k < 3; k++) {
                x[3 * g + k] = y[3 * b + k];
                V[3 * g + k] = y[3 * nm + 3 * b + k];
            }
            m[g] = mm[b];
            R[g] = Rm[b];
            alive[g] = am[b];
        }
    }
    free(am);
    free(mem);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Energy and momenta in democratic heliocentric variables (Sec. 2.1.1 item 7;
 * the split of the Hamiltonian is footnote 1 of Sec. 2.1.1):
 *   E = sum 1/2 m|V|^2 - sum G M0 m/|x| + |P|^2/(2 M0) - sum_{i<j} G m_i m_j / r_ij,
 *   P = sum m V,  L = sum m x x V. */
void orc_energy(int64_t n, double G, double M0, const double* m, const double* x, const double* V,
                const int32_t* alive, double* E, double L[3], double P[3]) {
    nsum e = {0, 0}, pp[3] = {{0, 0}, {0, 0}, {0, 0}}, ll[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = 0; i < n; i++) {
        if (!alive[i]) continue;
        const double* xi = x + 3 * i;
        const double* vi = V + 3 * i;
        nadd(&e, 0.5 * m[i] * dot3(vi, vi));
        nadd(&e, -G * M0 * m[i] / norm3(xi));
        for (int k = 0; k < 3; k++) nadd(&pp[k], m[i] * vi[k]);
        nadd(&ll[0], m[i] * (xi[1] * vi[2] - xi[2] * vi[1]));
        nadd(&ll[1], m[i] * (xi[2] * vi[0] - xi[0] * vi[2]));
        nadd(&ll[2], m[i] * (xi[0] * vi[1] - xi[1] * vi[0]));
    }
    for (int64_t i = 0; i < n; i++) {
        if (!alive[i]) continue;
        nsum row = {0, 0};
        for (int64_t j = i + 1; j < n; j++) {
            /* a small body has no mutual potential energy with anything */
            if (!alive[j] || m[i] == 0.0 || m[j] == 0.0) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            nadd(&row, -G * m[i] * m[j] / norm3(d));
        }
        nadd(&e, nval(&row));
    }
    double Pv[3] = {nval(&pp[0]), nval(&pp[1]), nval(&pp[2])};
    nadd(&e, dot3(Pv, Pv) / (2.0 * M0));
    *E = nval(&e);
    for (int k = 0; k < 3; k++) {
        P[k] = Pv[k];
        L[k] = nval(&ll[k]);
    }
}

/* ---------------------------------------------------------------------- */
/* One or more steps of the hybrid integrator (Sec. 3.1 blocks in order; the
 * encounter part as in the Sec. 3.2 listing).  Per step:
 *   (first call only) rc and a at the current positions;
 *   kick V += dt/2 a;  jump x += dt/2 P/M0 with P = sum m V;  save x0, V0;
 *   drift every body over dt;  rc from the positions after the drift;
 *   scan;  BS for each group of flagged pairs from (x0, V0);
 *   jump x += dt/2 P/M0;  a at the new positions;  kick V += dt/2 a.
 * The closing a is kept for the next step's opening kick (both are
 * evaluated at the same positions and masses).  On error the state is put
 * back to the start of the failed step and the status is returned. */
/* Removal of body i at the end of a step: accreted by the star (the merged
 * star, at the centre of mass of the star and the body, becomes the origin of
 * the heliocentric frame, so every other position moves by -m_i x_i / M0';
 * barycentric velocities are unchanged) or ejected.  E_lost gets the
 * Hamiltonian's drop, from the energy before and after. */
static void remove_body(orc_params* p, int64_t n, double* m, double* x, double* V, int32_t* alive, int64_t i,
                        int accrete, double* E_lost) {
    double Eb, Ea, L[3], P[3];
    orc_energy(n, p->G, p->M0, m, x, V, alive, &Eb, L, P);
    if (accrete) {
        const double M0n = p->M0 + m[i];
        const double Xc[3] = {m[i] * x[3 * i] / M0n, m[i] * x[3 * i + 1] / M0n, m[i] * x[3 * i + 2] / M0n};
        for (int64_t j = 0; j < n; j++)
            if (alive[j] && j != i)
                for (int k = 0; k < 3; k++) x[3 * j + k] -= Xc[k];
        p->M0 = M0n;
    }
    alive[i] = 0;
    m[i] = 0.0;
    orc_energy(n, p->G, p->M0, m, x, V, alive, &Ea, L, P);
    *E_lost += Eb - Ea;
}

int32_t orc_step(orc_params* p, int64_t n, double* m, double* R, double* x, double* V, double* a,
                 double* rc, int32_t* alive, int32_t* have_accel, double* E_lost, int64_t nsteps,
                 orc_stats* st) {
    const double G = p->G, dt = p->dt, half = 0.5 * p->dt;
    size_t n3 = sizeof(double) * (size_t)(3 * n + 1), n1 = sizeof(double) * (size_t)(n + 1);
    double *x0 = malloc(n3), *V0 = malloc(n3), *xs = malloc(n3), *Vs = malloc(n3), *as = malloc(n3);
    double *ms = malloc(n1), *Rs = malloc(n1), *rcs = malloc(n1);
    int32_t* als = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t* label = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t* members = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t* accf = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t cap = 4 * n + 64;
    int32_t* pi = malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* pj = malloc(sizeof(int32_t) * (size_t)cap);
    int32_t status = ORC_OK;
    for (int64_t step = 0; step < nsteps && status == ORC_OK; step++) {
        orc_stats s = {0, 0, 0, 0, 0, 0, 0, 0};
        const double M0 = p->M0;   /* the star's mass this step (accretions change it at the end) */
        if (!*have_accel) {
            orc_hill_rcrit(n, M0, p->rcrit_hill, m, x, alive, rc);
            orc_accel(n, G, p->changeover, m, x, rc, alive, a);
            *have_accel = 1;
        }
        memcpy(xs, x, n3 - sizeof(double));
        memcpy(Vs, V, n3 - sizeof(double));
        memcpy(as, a, n3 - sizeof(double));
        memcpy(ms, m, n1 - sizeof(double));
        memcpy(Rs, R, n1 - sizeof(double));
        memcpy(rcs, rc, n1 - sizeof(double));
        memcpy(als, alive, sizeof(int32_t) * (size_t)n);
        double E_lost_s = *E_lost;
        /* opening kick (Hamiltonian block, LOOP 1) */
        for (int64_t i = 0; i < n; i++)
            if (alive[i])
                for (int k = 0; k < 3; k++) V[3 * i + k] += half * a[3 * i + k];
        /* jump: momentum reduction (LOOP 2), positions (LOOP 3), copy (LOOP 4) */
        double P[3] = {0, 0, 0};
        for (int64_t i = 0; i < n; i++)
            if (alive[i])
                for (int k = 0; k < 3; k++) P[k] += m[i] * V[3 * i + k];
        for (int64_t i = 0; i < n; i++)
            if (alive[i])
                for (int k = 0; k < 3; k++) x[3 * i + k] += half * P[k] / M0;
        memcpy(x0, x, n3 - sizeof(double));
        memcpy(V0, V, n3 - sizeof(double));
        /* drift; a drift passing within the star's radius marks the body for accretion */
        for (int64_t i = 0; i < n && status == ORC_OK; i++) {
            accf[i] = 0;
            if (!alive[i]) continue;
            int32_t it = 0;
            if (orc_kepler_drift(G * M0, dt, x + 3 * i, V + 3 * i, p->kepler_max_iter, &it) != ORC_OK)
                status = ORC_EKEPLER;
            if (it > s.kepler_iter_max) s.kepler_iter_max = it;
            if (p->r_star > 0.0 && orc_drift_min_r(G * M0, dt, x0 + 3 * i, V0 + 3 * i, x + 3 * i, V + 3 * i) <= p->r_star)
                accf[i] = 1;
        }
        if (status == ORC_OK) {
            orc_hill_rcrit(n, M0, p->rcrit_hill, m, x, alive, rc);
            int64_t np = orc_scan(n, dt, x0, V0, x, V, rc, alive, m, p->scan_prune, cap, pi, pj, &s.n_candidates);
            if (np > cap) {
                cap = np;
                pi = realloc(pi, sizeof(int32_t) * (size_t)cap);
                pj = realloc(pj, sizeof(int32_t) * (size_t)cap);
                np = orc_scan(n, dt, x0, V0, x, V, rc, alive, m, p->scan_prune, cap, pi, pj, &s.n_candidates);
            }
            s.n_pairs = np;
            if (np > 0) {
                s.n_groups = orc_groups(n, np, pi, pj, label);
                for (int64_t g = 0; g < n && status == ORC_OK; g++) {
                    if (label[g] != g) continue;
                    int64_t nm = 0;
                    for (int64_t i = g; i < n; i++)
                        if (label[i] == g) members[nm++] = (int32_t)i;
                    for (int64_t b = 0; b < nm; b++)
                        for (int k = 0; k < 3; k++) {
                            x[3 * members[b] + k] = x0[3 * members[b] + k];
                            V[3 * members[b] + k] = V0[3 * members[b] + k];
                        }
                    status = orc_bs_group(p, nm, members, m, R, rc, alive, x, V, E_lost, &s.n_mergers,
                                          &s.bs_substeps);
                }
            }
        }
        if (status == ORC_OK) {
            /* closing jump, forces at the new positions, closing kick */
            P[0] = P[1] = P[2] = 0.0;
            for (int64_t i = 0; i < n; i++)
                if (alive[i])
                    for (int k = 0; k < 3; k++) P[k] += m[i] * V[3 * i + k];
            for (int64_t i = 0; i < n; i++)
                if (alive[i])
                    for (int k = 0; k < 3; k++) x[3 * i + k] += half * P[k] / M0;
            orc_accel(n, G, p->changeover, m, x, rc, alive, a);
            for (int64_t i = 0; i < n; i++)
                if (alive[i])
                    for (int k = 0; k < 3; k++) V[3 * i + k] += half * a[3 * i + k];
            /* end of the step: accretions in ascending index (a body merged away
             * in its encounter is gone already), then ejections when due */
            for (int64_t i = 0; i < n; i++)
                if (accf[i] && alive[i]) {
                    remove_body(p, n, m, x, V, alive, i, 1, E_lost);
                    s.n_accreted++;
                }
            if (p->r_eject > 0.0 && p->eject_every > 0 && (p->steps_done + 1) % p->eject_every == 0)
                for (int64_t i = 0; i < n; i++)
                    if (alive[i] && norm3(x + 3 * i) > p->r_eject) {
                        remove_body(p, n, m, x, V, alive, i, 0, E_lost);
                        s.n_ejected++;
                    }
            if (s.n_accreted + s.n_ejected > 0) *have_accel = 0;   /* the next step evaluates a afresh */
            p->steps_done++;
        } else {
            memcpy(x, xs, n3 - sizeof(double));
            memcpy(V, Vs, n3 - sizeof(double));
            memcpy(a, as, n3 - sizeof(double));
            memcpy(m, ms, n1 - sizeof(double));
            memcpy(R, Rs, n1 - sizeof(double));
            memcpy(rc, rcs, n1 - sizeof(double));
            memcpy(alive, als, sizeof(int32_t) * (size_t)n);
            *E_lost = E_lost_s;
        }
        if (st) *st = s;
    }
    free(x0); free(V0); free(xs); free(Vs); free(as); free(ms); free(Rs); free(rcs);
    free(als); free(label); free(members); free(accf); free(pi); free(pj);
    return status;
}
