/*
 * Oracle for the hybrid symplectic N-body step (test infrastructure).
 *
 * A plain, serial, FP64 statement of one step of the second-order
 * mixed-variable symplectic integrator with close-encounter handling that
 * Mercury-Opal runs (Sec. 2.1.1; Sec. 3.1 gives the loops of the step).  It
 * exists to check the CUDA path and is used only by the tests, by the smoke
 * check and by the benchmark's CPU-baseline leg; the product never links it.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Units: any consistent set; the tests use G = 1, au, M_sun, yr / (2 pi).
 * Arrays are row-major: x[3*i + k] is coordinate k of body i.
 * Velocities are democratic-heliocentric (barycentric) unless a function
 * says "helio".
 */
#ifndef OPAL_ORACLE_H
#define OPAL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status values (same numbering as the library's, by convention only) */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EKEPLER = 4, ORC_EBS = 5 };

typedef struct {
    double G, M0, dt;
    double rcrit_hill;      /* critical radius in Hill radii (3 in the workloads) */
    double bs_tol;          /* Bulirsch-Stoer relative tolerance (1e-12) */
    int32_t changeover;     /* 0: rational y^2/(2y^2-2y+1); 1: quintic 10y^3-15y^4+6y^5 */
    int32_t kepler_max_iter;/* cap on universal-variable iterations (0: default 50) */
    int32_t bs_max_substeps;/* cap on BS substeps per group per step (0: default 1<<20) */
    int32_t scan_prune;     /* 0: the exact test on every pair; 1: skip pairs a bound rules out first */
    double r_star;          /* radius of the star: a drift passing within it is accreted (0: off) */
    double r_eject;         /* ejection distance from the star (0: off) */
    int64_t eject_every;    /* steps between ejection checks (Sec. 2.1.2: every 200 yr) */
    int64_t steps_done;     /* state: steps completed (the ejection check counts them) */
} orc_params;

typedef struct {
    int64_t n_pairs;        /* flagged pairs in the last step */
    int64_t n_groups;       /* encounter groups in the last step */
    int64_t n_mergers;      /* mergers in the last step */
    int64_t bs_substeps;    /* accepted + rejected BS substeps in the last step */
    int64_t kepler_iter_max;/* largest iteration count of the drift in the last step */
    int64_t n_candidates;   /* pairs that reached the exact minimum-separation test */
    int64_t n_accreted;     /* bodies accreted by the star in the last step */
    int64_t n_ejected;      /* bodies ejected at the end of the last step */
} orc_stats;

/* helio <-> democratic-heliocentric velocities (Sec. 2.1.1, footnote on coordinates) */
void orc_helio_to_dh(int64_t n, double M0, const double* m, const double* v_helio, double* V);
void orc_dh_to_helio(int64_t n, double M0, const double* m, const double* V, double* v_helio);

double orc_changeover(double r, double rc, int32_t form);
void orc_hill_rcrit(int64_t n, double M0, double f_hill, const double* m, const double* x,
                    const int32_t* alive, double* rc);
void orc_accel(int64_t n, double G, int32_t form, const double* m, const double* x,
               const double* rc, const int32_t* alive, double* a);

void orc_stumpff(double z, double c[4]);
int32_t orc_kepler_drift(double mu, double dt, double x[3], double v[3], int32_t max_iter,
                         int32_t* iters);
double orc_drift_min_r(double mu, double dt, const double x0[3], const double V0[3], const double x1[3],
                       const double V1[3]);

double orc_min_sep2(double dt, const double d0[3], const double u0[3], const double d1[3],
                    const double u1[3]);
int64_t orc_scan(int64_t n, double dt, const double* x0, const double* V0, const double* x1,
                 const double* V1, const double* rc, const int32_t* alive, const double* m,
                 int32_t prune, int64_t cap, int32_t* pi, int32_t* pj, int64_t* n_candidates);
int64_t orc_groups(int64_t n, int64_t npairs, const int32_t* pi, const int32_t* pj,
                   int32_t* label);

int32_t orc_bs_group(const orc_params* p, int64_t nmem, const int32_t* members, double* m,
                     double* R, const double* rc, int32_t* alive, double* x, double* V,
                     double* E_lost, int64_t* n_mergers, int64_t* substeps);

void orc_energy(int64_t n, double G, double M0, const double* m, const double* x,
                const double* V, const int32_t* alive, double* E, double L[3], double P[3]);

int32_t orc_step(orc_params* p, int64_t n, double* m, double* R, double* x, double* V,
                 double* a, double* rc, int32_t* alive, int32_t* have_accel, double* E_lost,
                 int64_t nsteps, orc_stats* st);

#ifdef __cplusplus
}
#endif
#endif
