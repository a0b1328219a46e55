/*
 * opal_testing.h -- test hooks of the GB300 hybrid symplectic step.
 *
 * Each hook runs one stage of the step on its own, through the same kernels
 * opal_step launches, so the tests can compare a stage with the oracle on
 * identical inputs.  Pointers are host memory, borrowed for the call; arrays
 * of vectors are row-major n x 3; body order is the order given at create.
 * The hooks overwrite parts of the simulation's state: use a simulation made
 * for the test.  Same status codes as opal.h.
 */
#ifndef OPAL_TESTING_H
#define OPAL_TESTING_H

#include <stdint.h>

#include "opal.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kick accelerations at the simulation's current positions and masses
 * (Sec. 3.1, force block, LOOP 2): a[3n] = G sum_j m_j K(r_ij; max(rc_i, rc_j))
 * (x_j - x_i) / r_ij^3, in the simulation's precision and changeover form.
 * rc[n] (may be NULL to keep the simulation's) replaces the critical radii.
 * The result also becomes the simulation's stored accelerations. */
opal_status opal_debug_accel(opal_sim* sim, const double* rc, double* a);

/* Keplerian drift of n independent bodies about mu over dt (Sec. 3.1, third
 * block), in place on x[3n], v[3n]; iters[n] gets the iteration count, or
 * -1 where the solve did not converge within max_iter (0 = default 50), in
 * which case that body is left unchanged. */
opal_status opal_debug_drift(int64_t n, double mu, double dt, int32_t max_iter, double* x, double* v,
                             int32_t* iters);

/* Close-encounter scan of system 0 (Sec. 3.1, mce_snif block) on given
 * start-of-drift (x0, V0) and after-drift (x1, V1) states and critical radii
 * rc[n], with the simulation's dt.  Writes the flagged pairs, i < j, sorted,
 * into pi[cap], pj[cap]; *count gets their number and *ncand (may be NULL)
 * the pairs that reached the exact FP64 test.  The simulation's positions
 * and velocities are overwritten. */
opal_status opal_debug_scan(opal_sim* sim, const double* x0, const double* V0, const double* x1,
                            const double* V1, const double* rc, int64_t cap, int32_t* pi, int32_t* pj,
                            int64_t* count, int64_t* ncand);

/* Bulirsch-Stoer integration over the simulation's dt of all bodies of a
 * one-system simulation (at most 64) as a single encounter group, from
 * (x0, V0), with critical radii rc, masses m, radii radius, flags alive
 * (Sec. 2.1.1 footnote 2; mce_coll for mergers).  Outputs x, V and updates
 * m, radius, alive in place; *E_lost gets the energy removed by mergers and
 * *substeps the substeps used. */
opal_status opal_debug_bs_group(opal_sim* sim, const double* x0, const double* V0, const double* rc, double* x,
                                double* V, double* m, double* radius, int32_t* alive, double* E_lost,
                                int64_t* substeps);

/* Grid barriers of the whole-GPU encounter kernel (groups of more than 64
 * members, whose blocks meet at grid-wide barriers between the phases of
 * every derivative).  Each barrier wait is bounded by the global timer:
 * after wait_ns (wait_ns = 0 restores the default, 4 s) the waiting block
 * sets an abort flag that every block leaves through, and the step fails
 * with OPAL_EBS and is undone from its saved start.  hold = 1 makes the
 * last block to arrive wait as well instead of releasing the others, as if
 * a block never arrived, so the first barrier's waits run out; hold = 0
 * restores normal barriers.  The setting holds for the simulation's later
 * steps; the step graph is captured again.  Errors: OPAL_EINVAL for
 * wait_ns < 0 or hold not 0 or 1; OPAL_ECUDA if the capture fails. */
opal_status opal_debug_barrier(opal_sim* sim, int64_t wait_ns, int32_t hold);

/* Measured ALU peaks of the current device, for rooflines: out[0] FP32 FMA
 * TFLOP/s (an FMA counts 2), out[1] FP64 FMA TFLOP/s, out[2] MUFU reciprocal
 * square roots, Tops/s.  Independent FMA (or rsqrt) chains on every SM, a few
 * milliseconds each, timed with CUDA events on the default stream after one
 * warm-up launch.  Needs no simulation; allocates 64 bytes of device memory
 * for the call.  OPAL_EINVAL for a NULL out, OPAL_ECUDA if a launch fails. */
opal_status opal_probe_alu_peaks(double out[3]);

/* Device timeline of a step, for measurement.  In a library built with
 * OPAL_TIMELINE defined (paper_2601_19654_gb300/build.py, timeline=True, into
 * its own directory), thread 0 of every block of the step's kernels reads the
 * device's global nanosecond timer when the block starts and when it leaves,
 * and each kernel keeps the earliest start and the latest end.
 * opal_timeline_kernels() is the number of kernel slots (0 in the normal
 * build, which compiles none of it); opal_timeline_name(id) the kernel of slot
 * id (a static string; NULL out of range).  opal_timeline(sim, 1, NULL)
 * resets the slots (after the simulation's stream is idle); opal_timeline(sim,
 * 0, out) copies them to out[2 * opal_timeline_kernels()], start and end of
 * slot id at out[2 id] and out[2 id + 1] in ns (a start of ~0 means the kernel
 * did not run since the reset).  Errors: OPAL_EINVAL for a NULL sim or out, or
 * in the normal build; OPAL_ECUDA if a copy fails. */
int32_t opal_timeline_kernels(void);
const char* opal_timeline_name(int32_t id);
opal_status opal_timeline(opal_sim* sim, int32_t reset, uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif
