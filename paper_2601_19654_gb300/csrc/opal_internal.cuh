// Internal layout and device helpers of the GB300 hybrid symplectic step.
//
// Body arrays are structure-of-arrays in HBM, systems packed one after
// another, each padded to a multiple of kPad bodies (ghost bodies: m = 0,
// alive = 0, parked far away).  All FP64 state stays resident on the device
// for the lifetime of a simulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/opal.h"

namespace opal {

constexpr int kPad = 256;        // body padding of every system (largest kick i-tile)
constexpr int kSeg = 64;         // bodies per partial-sum segment
constexpr int kBodyThreads = 128;
constexpr int kBsMaxMembers = 64;   // bodies per encounter group of the lockstep kernels
constexpr int64_t kHugeWaitNs = 4000000000;   // the whole-GPU encounter kernel's barrier wait limit (4 s)
constexpr int kHugeAbortDetail = 2999999;      // status detail of its barrier aborts: this, or this + 1 + group
constexpr int kKickJTile = 256;
constexpr int kKickBox = 128;      // positions per tile box of the kick's sorted copies     // j-bodies the kick stages in shared memory at a time
constexpr int kBsManyGroups = 608;  // above this many groups a step integrates them packed, lane per member
constexpr int kBucketDiv = 4;       // body slots per bucket of the spatial sort (cap / 4 buckets a system)
constexpr int kBsOut = 9;           // doubles per member slot of the BS side buffer: x, V, m, R, alive
constexpr int kFixParts = 4;        // the kick's correction after the encounters: member ranges per body
constexpr int kBsRows = 8;          // extrapolation rows: n_k = 2, 4, ..., 16
constexpr float kFar = 1.0e18f;     // parking coordinate of ghost and dead bodies (float copies)


// status codes mirror opal_status
enum : int { kOk = 0, kEinval = 1, kEnomem = 2, kEcuda = 3, kEkepler = 4, kEbs = 5, kEoverflow = 6,
             kEnonfinite = 7 };

// four doubles, 32-byte aligned (one shared-memory slot of a j-body)
struct __align__(32) D4 {
    double x, y, z, w;
};

// Device control block: status word and per-step counters.
struct Ctl {
    int status;          // first error of the current opal_step call (0 = ok)
    int detail;          // body or group index that raised it
    // counters of the current step: zeroed together at its start, from ncand
    // up to steps_done
    int ncand;           // pairs passing both FP32 bounds (this step)
    int nnear;           // pairs passing the FP32 midpoint test (this step)
    int nflag;           // flagged pairs (this step)
    int ngroups;         // encounter groups (this step)
    int ninvolved;       // bodies in groups (this step)
    int ninv_big;        // of them big bodies, the sources of force (this step)
    int naccf;           // bodies whose drift passed within the star's radius (this step)
    int nacc, nej;       // bodies accreted and ejected at the end of the step (this step)
    int nmerge;          // mergers (this step)
    int kepler_max;      // largest drift iteration count (this step)
    int nlarge;          // groups too large for one warp (this step)
    int ncls[4];         // groups of 2, 3-4, 5-8, 9-16 members (this step)
    int qcls[4];         // how far the packed encounter kernel has taken each list (this step)
    int nhard;           // groups left to the lockstep kernels when groups are many (this step)
    int qlock[3];        // queues of the lockstep kernels: up to 4, 32, 64 members (this step)
    int nhuge;           // groups of more than 64 members (this step)
    int ntov;            // tile pairs whose boxes overlap (this step)
    unsigned long long nsub;  // BS substeps (this step)
    long long steps_done;
    int cand_overflow;   // candidates lost to a full candidate list (forces a status)
    int reprime;         // a removal happened: the next step evaluates the accelerations afresh
    // work queue of the kick: next item, blocks done; the last block out puts
    // both back to zero, so every launch starts from an empty queue
    int kick_next;
    int kick_done;
};

// Encounter groups of more than 64 members: working arrays of one group
// (component-major [q][cap] arrays, cap = the largest such group).
constexpr int kHugeMax = 8192;    // members of the largest group these buffers take
constexpr int kHugeCand = 1024;   // member pairs in contact after one substep
constexpr int kHugeWide = 16;     // wide-rc members whose rows run one chunk a task (others: kHugeGroup chunks)
constexpr int kHugeGroup = 8;     // chunks a pair-phase task takes for the other members
struct HugeBuf {
    int64_t cap;
    double* y;                // [6][cap]: substep state
    double *z0, *z1;          // [kBsRows][6][cap]: each midpoint sequence's chain
    double* row;              // [kBsRows][6][cap]: extrapolation tableau (in place)
    double* pos;              // [kBsRows][3][cap]: each sequence's positions of the current evaluation
    float4* posf;             // [kBsRows][cap]: the same in float, with rc (rounded up)
    double* part;             // [kBsRows][cap * chunks][3]: (1 - K) sums of each (member, 64-member chunk)
    double *m, *R, *rc, *pinv;
    int *alive, *gid;
    int* perm;                // [cap]: members in spatial order; chunk ch is perm[64 ch .. 64 ch + 63]
    int* wide;                // [cap]: 1 for a member with a wide critical radius (its row runs a chunk a task)
    unsigned int* key;        // [cap]: their spatial keys
    float4* cbox;             // [2][kBsRows][chunks][2]: box of each chunk's evaluation points (lo xyz +
                              // largest rc, hi xyz), by round parity
};
// barrier and bookkeeping of the whole-GPU encounter kernel (zeroed every step)
struct HugeCtl {
    unsigned int bar_count, bar_gen;
    int abort, skip;
    int bb[4];                          // the group's box in x and y (order-mapped: min x, max x, min y, max y)
    int nwide;                          // members with a wide critical radius, listed in wlist
    int wlist[kHugeWide];
    int rcmm[2];                        // bits of the members' largest and smallest float rc (>= 0)
    int ncand, nmerge;
    double El;
    unsigned long long err[kBsRows];   // grid-wide maximum error of each row (bits of a double >= 0)
    int2 cand[kHugeCand];
};

// Neville coefficients 1 / ((n_k / n_{k-j})^2 - 1) with n_k = 2(k+1): exact
// rationals (k-j+1)^2 / ((k+1)^2 - (k-j+1)^2), rounded once.
static __constant__ double kNeville[kBsRows][kBsRows] = {
    {0, 0, 0, 0, 0, 0, 0, 0},
    {0, 1.0 / 3.0, 0, 0, 0, 0, 0, 0},
    {0, 4.0 / 5.0, 1.0 / 8.0, 0, 0, 0, 0, 0},
    {0, 9.0 / 7.0, 4.0 / 12.0, 1.0 / 15.0, 0, 0, 0, 0},
    {0, 16.0 / 9.0, 9.0 / 16.0, 4.0 / 21.0, 1.0 / 24.0, 0, 0, 0},
    {0, 25.0 / 11.0, 16.0 / 20.0, 9.0 / 27.0, 4.0 / 32.0, 1.0 / 35.0, 0, 0},
    {0, 36.0 / 13.0, 25.0 / 24.0, 16.0 / 33.0, 9.0 / 40.0, 4.0 / 45.0, 1.0 / 48.0, 0},
    {0, 49.0 / 15.0, 36.0 / 28.0, 25.0 / 39.0, 16.0 / 48.0, 9.0 / 55.0, 4.0 / 60.0, 1.0 / 63.0},
};

// Per-system constants.
struct SysInfo {
    int64_t off;      // first body
    int64_t cap;      // padded body count (multiple of kPad)
    int64_t n;        // bodies given at create
    int64_t nb;       // big bodies (m > 0): the first nb; the rest are small (massless)
    int64_t seg0;     // first partial-sum segment (off / kSeg)
    int64_t nseg;     // cap / kSeg
    int64_t slot0;    // first row of the kick's partial-acceleration buffer
    int32_t nchunk;   // j-chunks of the kick for this system
    int32_t pad;
};

// One unit of kick work: an i-tile against a j-range of the same system.
struct KickItem {
    int32_t sys;
    int32_t chunk;    // index of the j-range within the system (the partial row it writes)
    int64_t i0, i1;   // i-tiles at i0, i0 + istep, ... below i1 (global sorted positions)
    int64_t istep;
    int64_t j0, j1;   // j-range (global sorted positions, half-open)
};

// One unit of scan / energy work: an i-tile against a j-tile at or above it.
struct PairTile {
    int32_t sys;
    int32_t pad;
    int64_t i0, j0;   // tile starts (global); tiles are kSeg bodies
};

struct Params {
    double G, M0, dt, rcrit_hill, bs_tol;
    int precision, changeover, kepler_max_iter, bs_max_substeps;
    int64_t encounter_capacity;
    double r_star;       // star's radius: a drift passing within it is accreted (0: off)
    double r_eject;      // ejection distance (0: off)
    int64_t eject_every; // steps between ejection checks
};

// All device pointers of one simulation (passed by value to kernels).
struct Dev {
    int64_t ntot;
    int nsys;
    int overlap;       // 1: the kick runs beside the BS and is fixed afterwards; 0: after it
    int gated;         // the launch belongs to the re-evaluation after a removal: run only if one happened
    int huge_hold;     // test hook: the whole-GPU encounter kernel's barriers never release (waits run out)
    int64_t huge_wait_ns;   // limit of one wait at that kernel's grid barriers (default 4 s)
    Params p;
    double* M0s;       // [nsys] the star's mass of each system (it grows by what it accretes)
    int* accf;         // [ntot] the body's drift passed within the star's radius this step
    SysInfo* sys;
    int32_t* body_sys;
    // FP64 state
    double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
    double *x0, *y0, *z0, *vx0, *vy0, *vz0;      // start of drift
    double *xs, *ys, *zs, *vxs, *vys, *vzs, *rcs; // start of step (undo)
    double *m, *R, *rc;
    double* hcb;                        // cbrt(m / 3 M0): the mass factor of the Hill radius
    int32_t* alive;
    // float copies for the pair kernels
    float4* kh;    // (x_hi, y_hi, z_hi, m) after drift / BS
    float4* kl;    // (x_lo, y_lo, z_lo, max(4 rc^2, tiny))
    float* rcf;    // rc as float (rounded up)
    float* rcmax;  // per system: largest rc of the step (rounded up)
    // the kick's copies in the scan's spatial order (position p holds body
    // csorted[p]), written before each kick: hi parts and mass as separate
    // arrays, lo parts with 4 rc^2, rc; and per 128-position tile its box
    // of live positions and largest near threshold (two float4: lo xyz +
    // threshold, hi xyz)
    float *ks_x, *ks_y, *ks_z, *ks_m;
    float4* ks_lo;
    float* ks_rc;
    int rows_g = 8;  // warps a position takes in k_kick_rows (1, 2, 4 or 8: eight rows a warp)
    unsigned long long* timeline = nullptr;   // [kTlCount][2] (timeline builds only)
    double* ksum;    // [3 ntot]: each body's kick partial rows summed (by k_kick_rows), by body index
    float4* kbox;    // per 128 positions
    float4* kbox2;   // per 256 positions
    float4* cen;   // (c_hi, s): midpoint of the body's path over the step and the radius
                   // s bounding the path's distance from it (plus rc and margins)
    float4* sc0;   // (x0_hi, y0_hi, z0_hi, s)
    float4* sc1;   // (x0_lo, y0_lo, z0_lo, 0)
    float4* sv0;   // (V0, |V0|)
    float4* sv1;   // (V1, |V1|)
    // partial sums
    double *pacc_x, *pacc_y, *pacc_z;   // kick partials [slot rows]
    double *pP_close;                   // [3][nseg_tot] momentum before the closing jump
    double *pP_open;                    // [3][nseg_tot] momentum before the opening jump
    double* Ptot;                       // [2][nsys][3] those momenta summed: 0 opening, 1 closing jump
    double* Pjump;                      // [2][nsys][3] each jump's displacement dt/2 P / M0, with its total
    int* pcnt;                          // [2][nsys] blocks done with their segments (see system_total)
    int64_t nseg_tot;
    // spatial order of the scan: each system's bodies counting-sorted by the
    // cell of their path midpoint, and the box of every 64-body tile
    int* sbox;                          // [2][nsys][3] order-mapped min, then max, of the midpoints
    int* ckey;                          // per body: its bucket
    int* cstart;                        // [ncell] bucket counts
    int* ccursor;                       // [ncell] scatter cursors
    int2* cscratch;                     // (body, bucket or -1 if dead) after the scatter, any order in a bucket
    int* csorted;                       // bodies in sorted order, ascending ids within a cell
    float4* cen_sorted;                 // their midpoint records, in sorted order
    float* tbox;                        // [ntot / 64][6] tile boxes of c +- s
    int ncell;                          // buckets: one per kBucketDiv body slots
    // encounter pipeline
    int* tov;                           // tile pairs whose boxes overlap (indices into the tile list)
    int2* near;  int64_t near_cap;      // pairs passing the midpoint test
    int2* cand;  int64_t cand_cap;      // FP32-bound candidates
    int2* flag;  int64_t flag_cap;      // flagged pairs
    int32_t* label;                     // per body; -1 when not in a group
    int32_t* members;                   // group members, grouped, ascending
    int32_t* goff;                      // [ngroups + 1] member offsets
    int32_t* glarge;                    // groups of more than 4 members
    int32_t* gcls;                      // [4][gcap]: groups by size class (2, 4, 8, 16 members at most)
    int32_t* ghard;                     // [gcap]: groups for the lockstep kernels when groups are many
    int32_t* ghuge;                     // [gcap]: groups of more than 64 members
    HugeBuf hb;                         // working arrays of the whole-GPU encounter kernel
    HugeCtl* hctl;
    int64_t gcap;                       // capacity of each class list
    int* gcount;                        // per body: members of the group it roots (zero between steps)
    int* gofs;                          // per root: its group's first member slot
    int* gidx;                          // per root: its group's index
    double* glost;                      // per group energy lost to mergers
    double* undo;                       // per member slot: m, R, alive (3 doubles)
    double* bsout;                      // per member slot: the BS result (kBsOut doubles)
    D4* okx;                            // per member slot: x, y, z, m before it
    int* mlo;                           // [nsys] first member slot of the system (or a large value)
    int* mhi;                           // [nsys] one past its last member slot (or 0)
    double *cfx, *cfy, *cfz;            // [kFixParts][ntot]: kick correction parts (others), row parts (members)
    double* E_lost;                     // per system running sum
    Ctl* ctl;
};

// ---------------------------------------------------------------------------
// device helpers

__device__ __forceinline__ void set_status(Ctl* c, int code, int detail) {
    if (atomicCAS(&c->status, 0, code) == 0) c->detail = detail;
}

// Float-float arithmetic (a value held as hi + lo, two floats) for the
// mixed kick's row totals: Knuth's TwoSum gives a + b exactly as a rounded
// sum and its error; ff_add adds two such pairs (the hi parts by TwoSum, the
// lo parts and that error in float, then renormalised), within a few units
// of 2^-48 (|a| + |b|), on the FP32 pipe.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 t = two_sum(a.x, b.x);
    const float e = __fadd_rn(t.y, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(t.x, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, t.x)));
}

// Two members of an encounter group can collide unless both are small bodies
// (zero mass), which never interact (Sec. 2.1).
__device__ __forceinline__ bool bs_can_touch(double mu, double mw) { return mu > 0.0 || mw > 0.0; }

__device__ __forceinline__ double dot3(double ax, double ay, double az, double bx, double by, double bz) {
    return ax * bx + ay * by + az * bz;
}

// Fixed-order reduction of 3 values over a block of kBodyThreads threads into
// kBodyThreads / kSeg segments: out[c][seg] for each 64-body half.
__device__ __forceinline__ void segment_sums(const Dev& d, int64_t first_body, double vx, double vy, double vz, double* part) {
    __shared__ double buf[3][kBodyThreads];
    buf[0][threadIdx.x] = vx;
    buf[1][threadIdx.x] = vy;
    buf[2][threadIdx.x] = vz;
    __syncthreads();
    for (int w = kSeg / 2; w >= 1; w >>= 1) {
        int t = threadIdx.x % kSeg;
        if (t < w) {
            buf[0][threadIdx.x] += buf[0][threadIdx.x + w];
            buf[1][threadIdx.x] += buf[1][threadIdx.x + w];
            buf[2][threadIdx.x] += buf[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x % kSeg == 0) {
        int64_t sg = (first_body + threadIdx.x) / kSeg;
        part[sg] = buf[0][threadIdx.x];
        part[d.nseg_tot + sg] = buf[1][threadIdx.x];
        part[2 * d.nseg_tot + sg] = buf[2][threadIdx.x];
    }
}


// After segment_sums into part: the last block of system s to get here sums
// all the system's segments in a fixed order (each thread a strided set, then
// a tree over the block) and stores the total in out[0..2] and, when jump is
// given, the jump's displacement dt/2 P / M0 in jump[0..2], so the kernel
// that needs them reads three numbers.  counter[s] is back at zero afterwards
// (the step's memsets clear it too, in case a failing step left it behind).
__device__ __forceinline__ void system_total(const Dev& d, const double* part, const SysInfo& si, int s,
                                             int* counter, double* out, double* jump) {
    __shared__ int last;
    __shared__ double red[3][kBodyThreads];
    __syncthreads();   // this block's segment partials are written
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&counter[s], 1) == (int)(si.cap / kBodyThreads) - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double px = 0.0, py = 0.0, pz = 0.0;
    for (int64_t k = threadIdx.x; k < si.nseg; k += kBodyThreads) {
        const int64_t sg = si.seg0 + k;
        px += __ldcg(part + sg);
        py += __ldcg(part + d.nseg_tot + sg);
        pz += __ldcg(part + 2 * d.nseg_tot + sg);
    }
    red[0][threadIdx.x] = px;
    red[1][threadIdx.x] = py;
    red[2][threadIdx.x] = pz;
    __syncthreads();
    for (int w = kBodyThreads / 2; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        out[threadIdx.x] = red[threadIdx.x][0];
        // the jump's displacement, once for the system (every body's jump adds it)
        if (jump) jump[threadIdx.x] = 0.5 * d.p.dt * red[threadIdx.x][0] / d.M0s[s];
    }
    if (threadIdx.x == 0) counter[s] = 0;
}

// Comparisons of doubles as their bit patterns: for values >= +0 the IEEE
// patterns order as the values, and a value is <= 0 exactly when its pattern,
// read as a signed integer, is.  The integer units take these tests, which
// leaves the FP64 pipe (one warp instruction per many cycles) to the
// arithmetic on the encounter integrator's critical chain.
__device__ __forceinline__ bool ge_nonneg(double a, double b) {   // a >= b, both >= +0
    return __double_as_longlong(a) >= __double_as_longlong(b);
}
__device__ __forceinline__ bool gt_nonneg(double a, double b) {   // a > b, both >= +0
    return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool le_zero(double a) { return __double_as_longlong(a) <= 0; }

// The mutual term's factor G m_o (1 - K) / r^3 inside rc, given G m_o / r^3
// and y = (r - 0.1 rc) / (0.9 rc) < 1: for the rational form 1 - K is
// (1 - y)^2 / (2y^2 - 2y + 1), formed with its one division last, so that
// the division waits on the fewest operations before it (the encounter
// integrator's chains are FP64 latency); the quintic's 1 - K as written.
__device__ __forceinline__ double mutual_factor(double gm_ri3, double y, int form) {
    if (__double_as_longlong(y) <= 0) return gm_ri3;   // y <= 0: K = 0
    if (form == 0) {
        const double u = 1.0 - y;
        return (gm_ri3 * (u * u)) / fma(2.0 * y, -u, 1.0);   // 2y^2 - 2y + 1 = 1 - 2y(1 - y)
    }
    return gm_ri3 * (1.0 - y * y * y * (10.0 - 15.0 * y + 6.0 * y * y));
}

// Changeover weight K(r; rc): the rational form y^2/(2y^2-2y+1) or the
// quintic 10y^3-15y^4+6y^5, y = (r - 0.1 rc)/(0.9 rc); 1 beyond rc, 0 below 0.1 rc.
__device__ __forceinline__ double changeover(double r, double rc, int form) {
    if (r >= rc) return 1.0;
    double y = (r - 0.1 * rc) / (0.9 * rc);
    if (y <= 0.0) return 0.0;
    if (form == 0) return y * y / (2.0 * y * y - 2.0 * y + 1.0);
    return y * y * y * (10.0 - 15.0 * y + 6.0 * y * y);
}

__device__ __forceinline__ float changeover_f(float r, float rc, int form) {
    if (r >= rc) return 1.0f;
    float y = (r - 0.1f * rc) / (0.9f * rc);
    if (y <= 0.0f) return 0.0f;
    if (form == 0) return y * y / (2.0f * y * y - 2.0f * y + 1.0f);
    return y * y * y * (10.0f - 15.0f * y + 6.0f * y * y);
}

// Stumpff functions c0..c3: at an argument quartered until |z| <= 0.1,
//   c2 = sum_j (-z)^j / (2j+2)!,  c3 = sum_j (-z)^j / (2j+3)!,
// by Horner's rule in -z over j = 0..6 (the next terms are below 1e-23 of the
// sums there), c0 = 1 - z c2 and c1 = 1 - z c3; then the double-angle
// relations undo the quartering.
__device__ __forceinline__ void stumpff(double z, double& c0, double& c1, double& c2, double& c3) {
    constexpr double k2[7] = {1.0 / 2, 1.0 / 24, 1.0 / 720, 1.0 / 40320, 1.0 / 3628800, 1.0 / 479001600,
                              1.0 / 87178291200.0};
    constexpr double k3[7] = {1.0 / 6, 1.0 / 120, 1.0 / 5040, 1.0 / 362880, 1.0 / 39916800, 1.0 / 6227020800.0,
                              1.0 / 1307674368000.0};
    int nq = 0;
    while (fabs(z) > 0.1) {
        z *= 0.25;
        nq++;
    }
    const double w = -z;
    double s2 = k2[6], s3 = k3[6];
#pragma unroll
    for (int j = 5; j >= 0; j--) {
        s2 = fma(s2, w, k2[j]);
        s3 = fma(s3, w, k3[j]);
    }
    c2 = s2;
    c3 = s3;
    c0 = 1.0 - z * c2;
    c1 = 1.0 - z * c3;
    for (; nq > 0; nq--) {
        c3 = (c2 + c0 * c3) * 0.25;
        c2 = c1 * c1 * 0.5;
        c1 = c0 * c1;
        c0 = 2.0 * c0 * c0 - 1.0;
    }
}

// Universal-variable Kepler drift over dt (mu = G M0).  Bracketed Newton on
// F(chi) = r0 G1 + eta G2 + mu G3 - dt (F increasing, root in [0, dt/q] with q
// the pericentre distance), bisecting when a Newton step leaves the bracket;
// bound orbits first drop whole periods from dt and start from dt / r0,
// unbound ones start from the logarithmic value of Vallado's Algorithm 8.
// Returns iterations used, or -1 on non-convergence (state untouched).
// Divisions are few: 1/r0 (from a reciprocal square root), 1/mu, one for the
// bracket, one per Newton step and 1/r at the end; the period is only
// formed when the step may exceed it.
__device__ __forceinline__ int kepler_drift(double mu, double dt, int max_iter, double& x, double& y, double& z,
                                            double& vx, double& vy, double& vz) {
    const double rr = dot3(x, y, z, x, y, z);
    const double ir0 = rsqrt(rr), r0 = rr * ir0;
    double v2 = dot3(vx, vy, vz, vx, vy, vz);
    double eta = dot3(x, y, z, vx, vy, vz);
    double beta = 2.0 * mu * ir0 - v2;
    if (beta > 0.0) {
        // |dt| > period = 2 pi mu / beta^1.5, tested on the squares
        const double tpm = 2.0 * 3.14159265358979323846 * mu;
        if (dt * dt * (beta * beta * beta) > tpm * tpm) dt = fmod(dt, tpm / (beta * sqrt(beta)));
    }
    const double imu = 1.0 / mu;
    double hx = y * vz - z * vy, hy = z * vx - x * vz, hz = x * vy - y * vx;
    double p = dot3(hx, hy, hz, hx, hy, hz) * imu;
    double ecc2 = 1.0 - p * beta * imu;
    // dt / q with q = p / (1 + e), the pericentre distance
    const double dtq = dt * (1.0 + sqrt(ecc2 > 0.0 ? ecc2 : 0.0)) / p;
    double lo, hi;
    if (dt >= 0.0) {
        lo = 0.0;
        hi = p > 0.0 ? dtq : HUGE_VAL;
    } else {
        lo = p > 0.0 ? dtq : -HUGE_VAL;
        hi = 0.0;
    }
    double chi = dt * ir0;
    if (beta < 0.0) {
        // unbound orbit: logarithmic starting value (Vallado, Algorithm 8)
        double a = mu / beta, sg = dt >= 0.0 ? 1.0 : -1.0;
        double den = eta + sg * sqrt(-mu * a) * (1.0 - r0 / a);
        double arg = -2.0 * beta * dt / den;
        if (den != 0.0 && arg > 0.0 && isfinite(arg)) chi = sg * sqrt(-a / mu) * log(arg);
    }
    if (chi < lo) chi = lo;
    if (chi > hi) chi = hi;
    double c0, c1, c2, c3;
    int conv = 0, it;
    double dchi_prev = HUGE_VAL;
    for (it = 1; it <= max_iter; it++) {
        stumpff(beta * chi * chi, c0, c1, c2, c3);
        double G0 = c0, G1 = chi * c1, G2 = chi * chi * c2, G3 = chi * chi * chi * c3;
        double F = r0 * G1 + eta * G2 + mu * G3 - dt;
        double dF = r0 * G0 + eta * G1 + mu * G2;
        if (F < 0.0) lo = chi;
        else hi = chi;
        double chin = chi - F / dF;
        if (!(chin >= lo && chin <= hi)) chin = 0.5 * (lo + hi);
        double dchi = chin - chi;
        chi = chin;
        if (fabs(dchi) <= 1e-15 * fabs(chi) || (fabs(dchi) <= 1e-12 * fabs(chi) && fabs(dchi) >= dchi_prev)) {
            conv = 1;
            break;
        }
        dchi_prev = fabs(dchi);
    }
    if (!conv) return -1;
    stumpff(beta * chi * chi, c0, c1, c2, c3);
    double G0 = c0, G1 = chi * c1, G2 = chi * chi * c2, G3 = chi * chi * chi * c3;
    double r = r0 * G0 + eta * G1 + mu * G2;
    const double ir = 1.0 / r;
    double f = 1.0 - mu * G2 * ir0, g = dt - mu * G3;
    double fd = -mu * G1 * (ir * ir0), gd = 1.0 - mu * G2 * ir;
    double nx = f * x + g * vx, ny = f * y + g * vy, nz = f * z + g * vz;
    double nvx = fd * x + gd * vx, nvy = fd * y + gd * vy, nvz = fd * z + gd * vz;
    x = nx; y = ny; z = nz;
    vx = nvx; vy = nvy; vz = nvz;
    return it;
}

// Closest approach to the star during a drift from (x0, v0) to (x1, v1) over
// dt on the Kepler orbit about mu (the star-collision test, Sec. 2.1.2
// mce_cent): the pericentre distance q = p / (1 + e) when the pericentre is
// passed, else the nearer end.  The passage is read off the mean anomaly,
// which advances uniformly: on an ellipse M = E - e sin E (e cos E = 1 - r/a,
// e sin E = x.v / sqrt(mu a)), pericentres at M = 2 pi k; on a hyperbola
// M = e sinh F - F (e sinh F = x.v / sqrt(-mu a)), the pericentre at M = 0.
__device__ __forceinline__ double drift_min_r(double mu, double dt, double x0, double y0, double z0, double vx0,
                                              double vy0, double vz0, double x1, double y1, double z1, double vx1,
                                              double vy1, double vz1) {
    const double r0 = sqrt(dot3(x0, y0, z0, x0, y0, z0)), r1 = sqrt(dot3(x1, y1, z1, x1, y1, z1));
    double rmin = fmin(r0, r1);
    const double eta0 = dot3(x0, y0, z0, vx0, vy0, vz0);
    const double beta = 2.0 * mu / r0 - dot3(vx0, vy0, vz0, vx0, vy0, vz0);
    const double hx = y0 * vz0 - z0 * vy0, hy = z0 * vx0 - x0 * vz0, hz = x0 * vy0 - y0 * vx0;
    const double p = dot3(hx, hy, hz, hx, hy, hz) / mu;
    const double e2 = 1.0 - p * beta / mu;
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    const double q = p / (1.0 + e);
    bool passed;
    if (beta > 0.0) {
        const double a = mu / beta, n = sqrt(mu / (a * a * a));
        const double ecE = 1.0 - r0 / a, esE = eta0 / sqrt(mu * a);
        const double M0 = atan2(esE, ecE) - esE, M1 = M0 + n * dt;
        const double lo = fmin(M0, M1), hi = fmax(M0, M1);
        const double tp = 2.0 * 3.14159265358979323846;
        passed = tp * ceil(lo / tp) <= hi;
    } else if (beta < 0.0) {
        const double a = mu / beta, n = sqrt(mu / (-a * a * a));
        const double esF = eta0 / sqrt(-mu * a);
        const double F0 = e > 0.0 ? asinh(esF / e) : 0.0;
        const double M0 = esF - F0, M1 = M0 + n * dt;
        passed = (M0 <= 0.0 && M1 >= 0.0) || (M0 >= 0.0 && M1 <= 0.0);
    } else {
        passed = dt * eta0 < 0.0 && dt * dot3(x1, y1, z1, vx1, vy1, vz1) >= 0.0;   // parabolic
    }
    return passed ? fmin(rmin, q) : rmin;
}

// float hi/lo split of a double: hi = rn(x), lo = rn(x - hi)
__device__ __forceinline__ void split_hl(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// float copies of a live body for the pair kernels, and parking of a dead one
__device__ __forceinline__ void park_floats(const Dev& d, int64_t b) {
    float far = kFar * (1.0f + (float)(b & 1023) * (1.0f / 1024.0f));
    d.kh[b] = make_float4(far, far, far, 0.0f);
    d.kl[b] = make_float4(0.0f, 0.0f, 0.0f, 1e-30f);
    d.rcf[b] = 0.0f;
    d.sc0[b] = make_float4(far, far, far, 0.0f);
    d.cen[b] = make_float4(far, far, far, 0.0f);
    d.sc1[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    d.sv0[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    d.sv1[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

__device__ __forceinline__ void kick_floats(const Dev& d, int64_t b, double x, double y, double z, double m,
                                            double rc) {
    float hx, lx, hy, ly, hz, lz;
    split_hl(x, hx, lx);
    split_hl(y, hy, ly);
    split_hl(z, hz, lz);
    d.kh[b] = make_float4(hx, hy, hz, (float)m);
    d.kl[b] = make_float4(lx, ly, lz, 0.0f);
    d.rcf[b] = __double2float_ru(rc);
}

// order-preserving map of a float to an int (for atomic min / max), and back
__device__ __forceinline__ int ford(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float fordinv(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// ---------------------------------------------------------------------------
// Profiling: while opal_profile_steps runs, a recorder is installed and every
// launcher records a CUDA event on the stream after each kernel it launches.
struct ProfRec {
    cudaStream_t stream;
    int n, cap;
    const char* names[64];
    cudaEvent_t ev[64];
};
extern thread_local ProfRec* g_prof;
inline void prof_mark(const char* name) {
    if (g_prof && g_prof->n < g_prof->cap) {
        cudaEventRecord(g_prof->ev[g_prof->n], g_prof->stream);
        g_prof->names[g_prof->n++] = name;
    }
}

// ---------------------------------------------------------------------------
// Device timeline, for measurement: in a build with OPAL_TIMELINE defined,
// thread 0 of every block of the step's kernels reads the global timer when
// the block starts and when it leaves, and each kernel keeps its earliest
// start and latest end (atomic min and max on the pair [2 id], [2 id + 1]),
// so that a step's launches, concurrent branches included, can be read back
// as they ran.  The normal build compiles none of it.
enum TimelineId {
    kTlReset, kTlOpen, kTlSortCount, kTlSortPrefix, kTlSortScatter, kTlSortOrder, kTlTileBox, kTlTileCull,
    kTlScanTiles, kTlChord, kTlConfirm, kTlGroupLink, kTlGroupCount, kTlGroupOffsets, kTlGroupPlace,
    kTlGroupOrder, kTlBsPacked, kTlBsWs, kTlBs256, kTlBs512, kTlBsHuge, kTlKickStage, kTlKick, kTlKickRows,
    kTlApply, kTlFix, kTlClose, kTlFinish, kTlCount
};
#ifdef OPAL_TIMELINE
struct TimelineScope {
    unsigned long long* t;
    int id;
    __device__ static unsigned long long now() {
        unsigned long long v;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
        return v;
    }
    __device__ TimelineScope(unsigned long long* tl, int i) : t(tl), id(i) {
        if (t && threadIdx.x == 0) atomicMin(t + 2 * id, now());
    }
    __device__ ~TimelineScope() {
        if (t && threadIdx.x == 0) atomicMax(t + 2 * id + 1, now());
    }
};
#define OPAL_TIMELINE_SCOPE(id) TimelineScope opal_timeline_scope_(d.timeline, (id))
#else
#define OPAL_TIMELINE_SCOPE(id)
#endif

// ---------------------------------------------------------------------------
// kernel launchers (defined in the kernel translation units)

void launch_to_dh(const Dev& d, cudaStream_t s);
void launch_prime(const Dev& d, cudaStream_t s);
void launch_open(const Dev& d, cudaStream_t s);
// counting sort of each system's bodies by the cell of cen (csorted); the
// caller resets the buckets and notes the boxes first
void launch_sort_bodies(const Dev& d, cudaStream_t s);
void launch_order_prep(const Dev& d, cudaStream_t s);
void launch_step_reset(const Dev& d, int nsm, cudaStream_t s);
void launch_remove(const Dev& d, cudaStream_t s);
void launch_scan(const Dev& d, const PairTile* tiles, int64_t ntiles, int grid, cudaStream_t s);
void launch_confirm(const Dev& d, int grid, cudaStream_t s);
void launch_group(const Dev& d, int nsm, cudaStream_t s);
cudaError_t bs_setup();   // dynamic shared memory of the BS kernels
void launch_bs_packed(const Dev& d, int nsm, cudaStream_t s);
cudaError_t launch_bs_lockstep(const Dev& d, int nsm, cudaStream_t s, cudaStream_t s2, cudaEvent_t fork, cudaEvent_t join,
                        bool small_first);
void launch_kick(const Dev& d, const KickItem* items, int64_t nitems, int grid, int precision, int variant,
                 cudaStream_t s);
// after the BS: apply its results; fix the kick's rows when it ran beside the BS
cudaError_t launch_bs_huge(const Dev& d, int nsm, cudaStream_t s);
void launch_bs_apply(const Dev& d, int nsm, cudaStream_t s);
void launch_kick_fix(const Dev& d, int nsm, cudaStream_t s);
int kick_num_variants(int precision);
const char* kick_variant_name(int precision, int variant);
int kick_occupancy(int precision, int variant);
int kick_threads(int precision, int variant);      // threads a block of variant v
int kick_itile(int precision, int variant);   // i-bodies per i-tile (a divisor of kPad)
bool kick_jmajor(int precision, int variant); // items: one j-tile against a run of i-tiles (else an i-tile against j-tiles)
void launch_kick_stage(const Dev& d, int precision, cudaStream_t s);   // the sorted copies the mixed kick reads
void launch_kick_rows(const Dev& d, cudaStream_t s);   // after every kick: its partial rows summed a body
void launch_close(const Dev& d, cudaStream_t s);
void launch_first_accel_finish(const Dev& d, cudaStream_t s);
void launch_finish(const Dev& d, cudaStream_t s);
// Record a one-line reason as the calling thread's last error (opal_last_error(NULL)).
void set_thread_error(const char* fmt, ...);

void launch_energy(const Dev& d, const PairTile* tiles, int64_t ntiles, const int64_t* tile_off,
                   double* pair_part, double* body_part, double* out, int grid, cudaStream_t s);
// get_state of system sys (cap bodies): records (x, y, z, heliocentric v, m, R)
// and live flags, one a body, into rec and alive; P: 3 doubles of scratch
// (counter: nsys ints, zero on entry)
void launch_export(const Dev& d, int sys, int64_t cap, double* P, int* counter, double* rec, int* alive,
                   cudaStream_t s);
void launch_debug_drift(int n, double mu, double dt, int max_iter, double* x, double* v, int* iters, cudaStream_t s);
void launch_debug_scan_prep(const Dev& d, cudaStream_t s);

}  // namespace opal
