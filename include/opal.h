/*
 * opal.h -- C ABI of the GB300 hybrid symplectic N-body step.
 *
 * The library advances N fully interacting bodies around a central star
 * (the problem of Simonetti et al., "Mercury-Opal", Sec. 2.1: a star plus big
 * bodies with mass, position, velocity and physical radius) with one full
 * step of the second-order mixed-variable symplectic integrator with close-
 * encounter handling (Sec. 2.1.1; the step's loops are listed in Sec. 3.1):
 *   changeover-weighted O(N^2) kick (Sec. 3.1, force block, LOOP 2),
 *   jump by the stellar Hamiltonian (Sec. 3.1, Hamiltonian block),
 *   Keplerian drift of every body (Sec. 3.1, third block),
 *   close-encounter scan (Sec. 3.1, mce_snif block),
 *   Bulirsch-Stoer integration of the bodies in encounter, with perfect
 *   mergers (Sec. 2.1.1 footnote 2; Sec. 3.2 listing; mce_coll, Sec. 2.1.2).
 * Every step runs in CUDA kernels on the current device; nothing falls back
 * to the CPU.
 *
 * Conventions for every call:
 *   - All pointer arguments are HOST memory, borrowed for the duration of
 *     the call only; the library copies what it needs.
 *   - Arrays of vectors are row-major n x 3 doubles: x[3*i + k].
 *   - Positions and velocities passed in or out are HELIOCENTRIC (star at
 *     the origin, at rest); the library converts to democratic heliocentric
 *     coordinates inside (Sec. 2.1.1, footnote 1).
 *   - Any consistent units; G and M0 are parameters (the workloads use
 *     G = 1, au, M_sun and yr / 2 pi).
 *   - Every function returns an opal_status; on an error other than OPAL_OK
 *     opal_last_error() gives a one-line reason.  After a failed opal_step
 *     the state is the one at the start of the step that failed.
 *   - A simulation object must not be used from two host threads at once.
 */
#ifndef OPAL_H
#define OPAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opal_sim opal_sim; /* opaque; owns all its device memory */

typedef enum {
    OPAL_OK = 0,
    OPAL_EINVAL = 1,      /* invalid argument (n <= 0, non-finite value, m < 0, dt == 0 ...) */
    OPAL_ENOMEM = 2,      /* device or host allocation failed */
    OPAL_ECUDA = 3,       /* a CUDA runtime call failed */
    OPAL_EKEPLER = 4,     /* a Kepler drift did not converge within its iteration cap */
    OPAL_EBS = 5,         /* a Bulirsch-Stoer group used up its substep cap */
    OPAL_EOVERFLOW = 6,   /* the encounter pair list or a group exceeded its capacity */
    OPAL_ENONFINITE = 7   /* a non-finite value appeared in the state */
} opal_status;

typedef struct {
    double G;            /* gravitational constant (> 0) */
    double M0;           /* mass of the central star (> 0) */
    double dt;           /* step; negative integrates backwards (Mercury's direction flag) */
    double rcrit_hill;   /* critical radius in Hill radii (>= 0; the workloads use 3) */
    double bs_tol;       /* Bulirsch-Stoer relative tolerance per substep (> 0; default 1e-12) */
    int32_t precision;   /* 0: FP64 kick; 1: mixed (FP32 pair arithmetic, compensated FP64 totals) */
    int32_t changeover;  /* 0: rational y^2/(2y^2-2y+1); 1: quintic 10y^3-15y^4+6y^5 */
    int32_t kepler_max_iter;   /* cap on drift iterations; 0 = default (50) */
    int32_t bs_max_substeps;   /* cap on BS substeps per group per step; 0 = default (1<<20) */
    int64_t encounter_capacity;/* max flagged pairs per step; 0 = default (max(4096, 4 n)) */
    double r_star;       /* the star's radius (>= 0; 0 = off): a body whose Kepler drift passes
                            within it is accreted at the end of the step (Sec. 2.1.2, mce_cent) */
    double r_eject;      /* ejection distance (>= 0; 0 = off): bodies farther from the star are
                            removed at the end of every eject_every-th step (Sec. 2.1.2: 400 au) */
    int64_t eject_every; /* steps between ejection checks (>= 1 when r_eject > 0; Sec. 2.1.2:
                            every 200 yr, i.e. 200 yr / dt) */
} opal_params;

/* Fill *p with the defaults: G = M0 = 1, dt = 0.01 yr (2 pi / 100),
 * rcrit_hill = 3, bs_tol = 1e-12, precision = 1, changeover = 0, caps 0,
 * no star collisions and no ejections (r_star = r_eject = eject_every = 0).
 *
 * Removals (r_star or r_eject > 0).  At the end of a step, in ascending id
 * order, every live body whose drift passed within r_star of the star (its
 * Kepler orbit's pericentre inside the drift, or an end nearer) is accreted:
 * the star's mass grows by the body's, and the heliocentric frame moves to
 * the merged star (every other position shifts by -m x / M0'; barycentric
 * velocities are unchanged).  Then, on every eject_every-th step, every live
 * body farther than r_eject is removed.  The energy each removal takes from
 * the Hamiltonian is added to E_merged_lost, and the next step evaluates the
 * accelerations afresh. */
void opal_default_params(opal_params* p);

/* Create a simulation of one system of n bodies.
 *   m[n] masses (>= 0), x[3n] heliocentric positions (nonzero), v[3n]
 *   heliocentric velocities, radius[n] physical radii (>= 0).
 * Bodies of zero mass are small bodies (Sec. 2.1: massless particles that
 * feel the star and the big bodies): they are the source of no force, and
 * two small bodies never interact (no encounter, no collision); a small body
 * that touches a big one merges into it.  Every small body must come after
 * every big body (mass > 0), as in Mercury's separate big and small lists;
 * the kick and the encounter scan then cost (N_big + N_small) x N_big.
 * Computes the accelerations of the first kick and captures the per-step
 * CUDA graph.  Body i gets id i.  On success *out owns the simulation.
 * Errors: OPAL_EINVAL (bad argument, or a big body after a small one),
 * OPAL_ENOMEM, OPAL_ECUDA. */
opal_status opal_create(const opal_params* p, int64_t n, const double* m, const double* x,
                        const double* v, const double* radius, opal_sim** out);

/* Create an ensemble of nsys independent systems sharing the parameters.
 * n_per_sys[nsys] body counts; m, x, v, radius hold the systems one after
 * another (system s starts at body sum_{t<s} n_per_sys[t]).  All systems
 * advance together: one opal_step call steps every system.  Within each
 * system the small bodies (zero mass) follow the big ones, as for
 * opal_create. */
opal_status opal_ensemble_create(const opal_params* p, int32_t nsys, const int64_t* n_per_sys,
                                 const double* m, const double* x, const double* v,
                                 const double* radius, opal_sim** out);

/* Advance every system by nsteps steps (synchronous).  Stops at the first
 * step that fails; that step is undone and its status returned
 * (OPAL_EKEPLER, OPAL_EBS, OPAL_EOVERFLOW, OPAL_ENONFINITE or OPAL_ECUDA).
 * In the mixed form the kick runs beside the encounter integrator, on the
 * state after the drift, and is corrected for the encounter members
 * afterwards, while under 3% of the big bodies were in encounters in the
 * previous call (in order, after the encounters, above 8%); the environment
 * variable OPAL_STEP_ORDER=overlap or inorder forces one. */
opal_status opal_step(opal_sim* sim, int64_t nsteps);

/* Enqueue nsteps steps on the simulation's stream and return at once;
 * opal_wait() then blocks until they finish and returns what opal_step
 * would have (a failed step stops the rest and is undone, as there). */
opal_status opal_step_async(opal_sim* sim, int64_t nsteps);
opal_status opal_wait(opal_sim* sim);

/* The star's mass of system sys (M0 at create, plus what it has accreted). */
opal_status opal_central_mass(const opal_sim* sim, int32_t sys, double* M0);

/* Number of systems and total body capacity (sum of the n given at create). */
int32_t opal_num_systems(const opal_sim* sim);
int64_t opal_num_bodies(const opal_sim* sim);
/* Steps completed so far. */
int64_t opal_steps_done(const opal_sim* sim);

/* Copy out the live bodies of system sys (0 for a single system), in id
 * order.  Buffers are caller-owned with room for that system's n at create;
 * any of ids, m, x, v, radius may be NULL.  *n_alive receives the count.
 * Velocities are heliocentric. */
opal_status opal_get_state(const opal_sim* sim, int32_t sys, int64_t* n_alive, int64_t* ids,
                           double* m, double* x, double* v, double* radius);

/* Total energy E, angular momentum L and momentum P (in democratic
 * heliocentric variables: P = sum m V, barycentric) of system sys, in FP64;
 * *E_merged_lost is the running sum of the energy removed by mergers, so
 * E + E_merged_lost is the conserved quantity.  Any output may be NULL. */
opal_status opal_energy_momentum(const opal_sim* sim, int32_t sys, double* E, double L[3],
                                 double P[3], double* E_merged_lost);

/* Energy E, angular momentum L and momentum P of one system given in
 * caller-owned DEVICE arrays, computed the way opal_energy_momentum does it
 * (democratic heliocentric variables, FP64, fixed-order sums), without
 * allocating anything.  The paper has no counterpart: this is a diagnostic
 * for callers that cannot allocate device memory at the point of the check.
 * Those are callers whose device memory is all held by another allocator
 * (a caching allocator that has reserved the GPU's HBM), and callers that
 * must not synchronize the device while steps are in flight (cudaMalloc
 * and cudaFree may synchronize; this call only enqueues two kernels).
 *   n          bodies, 0 <= n <= 131072; a larger n returns OPAL_EINVAL and
 *              launches nothing (the scratch is a fixed 1024 x 13 doubles
 *              in device memory, one row per 128-body block).
 *   G, M0      as in opal_params (finite, > 0).
 *   m[n], x[3n], v[3n]   masses, heliocentric positions and heliocentric
 *              velocities (row-major n x 3), device memory of the current
 *              device (or managed), 8-byte aligned; borrowed, not kept.
 *              Bodies with m = 0 contribute nothing.
 *   out[7]     device memory: E, L[3], P[3], written by the second kernel.
 *   stream     cudaStream_t the kernels go on (NULL: the legacy stream).
 * The call returns once the kernels are enqueued: synchronize the stream
 * before reading out.  Nothing has to be zeroed first: out and every
 * scratch row the call reads are written by the same call.
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture begins.  The address is kept per device and
 * context: after a device reset (a new primary context) the next call looks
 * it up again, so make that call outside any capture as well.  All calls on a device share the one
 * scratch array, so two calls in flight at once (other streams or other
 * host threads) race and may return wrong values: serialize them.
 * Errors: OPAL_EINVAL (n out of range, G or M0 invalid, a NULL, misaligned
 * or host pointer), OPAL_ECUDA (symbol lookup or launch failed); the
 * reason is in opal_last_error(NULL). */
opal_status opal_energy_momentum_noalloc(int64_t n, double G, double M0, const double* m, const double* x,
                                         const double* v, double* out, void* stream);

/* Counters of the last completed step, summed over systems:
 * out[0] flagged pairs, out[1] groups, out[2] mergers, out[3] BS substeps,
 * out[4] pairs that reached the exact minimum-separation test,
 * out[5] largest drift iteration count, out[6] bodies accreted by the star,
 * out[7] bodies ejected. */
opal_status opal_last_step_stats(const opal_sim* sim, int64_t out[8]);

/* The CUDA stream every kernel of this simulation runs on (a cudaStream_t). */
void* opal_stream(const opal_sim* sim);

/* Run nsteps steps launching each kernel separately (no graph) and return
 * the average device time per launch of each kernel, measured with CUDA
 * events on the simulation's stream: ms[k] for kernel k, names[k] its name;
 * *nk receives the kernel count (at most cap).  Same results as opal_step. */
opal_status opal_profile_steps(opal_sim* sim, int64_t nsteps, int32_t cap, int32_t* nk,
                               double* ms, const char** names);

/* One line naming the kick kernel variant and launch shape in use (chosen
 * at create by timing the variants on the simulation's own bodies when the
 * pair count makes it worthwhile; OPAL_KICK_VARIANT=<index> forces one). */
const char* opal_kick_config(const opal_sim* sim);

/* Timing of the kick inside the step graph: with enable != 0 the graph is
 * re-captured with CUDA event records on the simulation's stream around the
 * kick kernel, and opal_last_kick_ms() returns the device time of the kick in
 * the most recent step (waiting for it), or -1 when timing is off. */
opal_status opal_time_kick(opal_sim* sim, int32_t enable);
double opal_last_kick_ms(const opal_sim* sim);

/* The kick kernel alone: reps launches (reps >= 1, after one untimed
 * launch) of the step's kick kernel on the simulation's stream, on the
 * sorted copies the last step left (the same item list and launch shape as
 * in the step graph, without the encounter integrator beside it), timed with
 * CUDA events on that stream; *ms gets the mean device time of one launch.
 * It rewrites only the kick's partial rows, which every step computes
 * afresh, so the simulation's state and later steps are unchanged.
 * Errors: OPAL_EINVAL (NULL argument, reps < 1), OPAL_ECUDA. */
opal_status opal_time_kick_alone(opal_sim* sim, int32_t reps, double* ms);

/* Number of kernel launches in one step (kernel nodes of the step graph). */
int32_t opal_graph_kernels(const opal_sim* sim);

/* The step order the last opal_step or opal_step_async call ran: 1 when the
 * kick ran beside the encounter integrator (overlap; see opal_step), 0 when
 * it ran after it, -1 for a NULL sim. */
int32_t opal_step_overlap(const opal_sim* sim);

/* Reason for the last error on sim (or on the calling thread when sim is NULL). */
const char* opal_last_error(const opal_sim* sim);

void opal_destroy(opal_sim* sim);

#ifdef __cplusplus
}
#endif
#endif
