// Body-parallel kernels of the step: the opening half (kick, jump, save,
// Keplerian drift, critical radii, float copies for the pair kernels), the
// closing half (jump, kick, momentum partials for the next step), the undo
// of a failed step, and the coordinate conversions at the boundary.
//
// Paper: Sec. 3.1, Hamiltonian block (LOOP 1 velocities, LOOP 2 momentum
// reduction, LOOP 3 positions, LOOP 4 copy of x and v) and third block
// (arxes_drift on every body, failure flag); Hill / critical radii from the
// instantaneous heliocentric distance, Sec. 2.1.1 item (4) and footnotes.
#include "opal_internal.cuh"

namespace opal {

// box of the path midpoints of the system's live bodies (block-reduced,
// then one atomic per block and bound)
__device__ void note_box(const Dev& d, int s, int64_t b) {
    __shared__ int red[6][kBodyThreads / 32];
    float v[6];
    if (d.alive[b]) {
        float4 c = d.cen[b];
        v[0] = v[3] = c.x;
        v[1] = v[4] = c.y;
        v[2] = v[5] = c.z;
    } else {
        v[0] = v[1] = v[2] = 3.0e38f;
        v[3] = v[4] = v[5] = -3.0e38f;
    }
    for (int k = 0; k < 6; k++) {
        float x = v[k];
        for (int o = 16; o >= 1; o >>= 1) {
            float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = k < 3 ? fminf(x, y) : fmaxf(x, y);
        }
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = ford(x);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        int x = red[k][0];
        for (int w = 1; w < kBodyThreads / 32; w++) x = k < 3 ? min(x, red[k][w]) : max(x, red[k][w]);
        if (k < 3) atomicMin(&d.sbox[3 * s + k], x);
        else atomicMax(&d.sbox[3 * d.nsys + 3 * s + k - 3], x);
    }
}

__device__ __forceinline__ void note_rcmax(const Dev& d, int s, double rc) {
    // rc >= 0: the order of non-negative floats matches the order of their
    // bits.  One atomic a warp (the lanes of a warp lie in one system): the
    // largest over the lanes here, then the lowest of them stores it
    const unsigned act = __activemask();
    const unsigned v = __reduce_max_sync(act, (unsigned)__float_as_int(__double2float_ru(rc)));
    if ((int)(threadIdx.x & 31) == __ffs(act) - 1) atomicMax(reinterpret_cast<int*>(d.rcmax) + s, (int)v);
}

__device__ __forceinline__ float norm3f(float x, float y, float z) { return sqrtf(fmaf(z, z, fmaf(y, y, x * x))); }

// scan inputs of a live body: start-of-drift hi/lo, velocities, and the
// midpoint c = (x0 + x1)/2 + dt (V0 - V1)/8 of its Hermite path over the
// step with the radius s around c that holds the whole path:
// |x1 - x0|/2 + (sqrt 3/18)|x0 - x1 + dt V1| + (4/27 + 1/8)|dt||V0 - V1|,
// plus rc, and margins far above FP32 rounding.
__device__ __forceinline__ void scan_floats(const Dev& d, int64_t b, double ox, double oy, double oz, double ovx,
                                            double ovy, double ovz, double x, double y, double z, double vx,
                                            double vy, double vz, double rc) {
    const double T = d.p.dt;
    double wx = x - ox, wy = y - oy, wz = z - oz;
    double ex = -wx + T * vx, ey = -wy + T * vy, ez = -wz + T * vz;
    double dvx = ovx - vx, dvy = ovy - vy, dvz = ovz - vz;
    double cx = 0.5 * (ox + x) + 0.125 * T * dvx, cy = 0.5 * (oy + y) + 0.125 * T * dvy,
           cz = 0.5 * (oz + z) + 0.125 * T * dvz;
    // the norms in FP32 (the FP64 pipe is this kernel's bound): their relative
    // error, a few 1e-7, is far inside the 1e-5 margin, and the differences
    // they are taken of are formed in FP64
    const float fcx = (float)cx, fcy = (float)cy, fcz = (float)cz;
    const float nw = norm3f((float)wx, (float)wy, (float)wz), ne = norm3f((float)ex, (float)ey, (float)ez),
                ndv = norm3f((float)dvx, (float)dvy, (float)dvz);
    const float rho = 0.5f * nw + 0.0962251f * ne + 0.2731482f * fabsf((float)T) * ndv;   // sqrt 3/18, 4/27 + 1/8 rounded up
    const float srf = (rho + __double2float_ru(rc)) * 1.00001f + 1e-6f * norm3f(fcx, fcy, fcz);
    d.cen[b] = make_float4(fcx, fcy, fcz, srf);
    const float v0n = norm3f((float)ovx, (float)ovy, (float)ovz), v1n = norm3f((float)vx, (float)vy, (float)vz);
    float hx, lx, hy, ly, hz, lz;
    split_hl(ox, hx, lx);
    split_hl(oy, hy, ly);
    split_hl(oz, hz, lz);
    d.sc0[b] = make_float4(hx, hy, hz, srf);
    d.sc1[b] = make_float4(lx, ly, lz, 0.0f);
    d.sv0[b] = make_float4((float)ovx, (float)ovy, (float)ovz, v0n);
    d.sv1[b] = make_float4((float)vx, (float)vy, (float)vz, v1n);
}

// ---------------------------------------------------------------------------
// create time: heliocentric -> democratic heliocentric velocities, one block
// per system: V_i = v_i - sum_j m_j v_j / (M0 + sum_j m_j).
__global__ void k_to_dh(Dev d) {
    const SysInfo si = d.sys[blockIdx.x];
    __shared__ double red[4][256];
    double sx = 0, sy = 0, sz = 0, sm = 0;
    for (int64_t k = threadIdx.x; k < si.cap; k += blockDim.x) {
        int64_t b = si.off + k;
        if (!d.alive[b]) continue;
        sx += d.m[b] * d.vx[b];
        sy += d.m[b] * d.vy[b];
        sz += d.m[b] * d.vz[b];
        sm += d.m[b];
    }
    red[0][threadIdx.x] = sx;
    red[1][threadIdx.x] = sy;
    red[2][threadIdx.x] = sz;
    red[3][threadIdx.x] = sm;
    __syncthreads();
    for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    double Mt = d.M0s[blockIdx.x] + red[3][0];
    double cx = red[0][0] / Mt, cy = red[1][0] / Mt, cz = red[2][0] / Mt;
    for (int64_t k = threadIdx.x; k < si.cap; k += blockDim.x) {
        int64_t b = si.off + k;
        if (!d.alive[b]) continue;
        d.vx[b] -= cx;
        d.vy[b] -= cy;
        d.vz[b] -= cz;
    }
}

// create time: critical radii and float copies at the initial positions
__global__ void k_prime(Dev d) {
    if (d.gated && (d.ctl->status || !d.ctl->reprime)) return;
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= d.ntot) return;
    int s = d.body_sys[b];
    d.hcb[b] = cbrt(d.m[b] / (3.0 * d.M0s[s]));
    if (!d.alive[b]) {
        d.rc[b] = 0.0;
        park_floats(d, b);
        return;
    }
    double r = sqrt(dot3(d.x[b], d.y[b], d.z[b], d.x[b], d.y[b], d.z[b]));
    double rc = d.p.rcrit_hill * r * d.hcb[b];
    d.rc[b] = rc;
    kick_floats(d, b, d.x[b], d.y[b], d.z[b], d.m[b], rc);
    note_rcmax(d, s, rc);
}

// ---------------------------------------------------------------------------
// Opening half of a step, one thread per body.
__global__ void __launch_bounds__(kBodyThreads) k_open(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlOpen);
    if (d.ctl->status) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int s = d.body_sys[(int64_t)blockIdx.x * kBodyThreads];
    const SysInfo si = d.sys[s];
    const double* J = d.Pjump + 3 * s;   // the opening jump dt/2 P / M0 (summed by the last close)
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctl->reprime = 0;   // any re-evaluation has run
    const double half = 0.5 * d.p.dt, M0 = d.M0s[s];
    // undo copy of the start of the step
    double x = d.x[b], y = d.y[b], z = d.z[b], vx = d.vx[b], vy = d.vy[b], vz = d.vz[b];
    d.xs[b] = x; d.ys[b] = y; d.zs[b] = z;
    d.vxs[b] = vx; d.vys[b] = vy; d.vzs[b] = vz;
    d.rcs[b] = d.rc[b];
    int iters = 0;
    if (d.alive[b]) {
        // kick (LOOP 1), jump with the momentum sum (LOOPs 2-3), copy (LOOP 4)
        vx += half * d.ax[b];
        vy += half * d.ay[b];
        vz += half * d.az[b];
        x += J[0];
        y += J[1];
        z += J[2];
        d.x0[b] = x; d.y0[b] = y; d.z0[b] = z;
        d.vx0[b] = vx; d.vy0[b] = vy; d.vz0[b] = vz;
        const double ox = x, oy = y, oz = z, ovx = vx, ovy = vy, ovz = vz;
        iters = kepler_drift(d.p.G * M0, d.p.dt, d.p.kepler_max_iter, x, y, z, vx, vy, vz);
        if (iters < 0) {
            set_status(d.ctl, kEkepler, (int)b);
            iters = d.p.kepler_max_iter;
        }
        // a drift passing within the star's radius: accreted at the end of the step
        if (d.p.r_star > 0.0 && drift_min_r(d.p.G * M0, d.p.dt, ox, oy, oz, ovx, ovy, ovz, x, y, z, vx, vy, vz) <=
                                    d.p.r_star) {
            d.accf[b] = 1;
            atomicAdd(&d.ctl->naccf, 1);
        }
        d.x[b] = x; d.y[b] = y; d.z[b] = z;
        d.vx[b] = vx; d.vy[b] = vy; d.vz[b] = vz;
        double r1 = sqrt(dot3(x, y, z, x, y, z));
        double rc = d.p.rcrit_hill * r1 * d.hcb[b];   // R_H = |x| cbrt(m / 3 M0), times f_hill
        d.rc[b] = rc;
        kick_floats(d, b, x, y, z, d.m[b], rc);
        note_rcmax(d, s, rc);
        scan_floats(d, b, ox, oy, oz, ovx, ovy, ovz, x, y, z, vx, vy, vz, rc);
    } else {
        park_floats(d, b);
    }
    // largest iteration count of the block, and the box of the midpoints
    __shared__ int itmax;
    if (threadIdx.x == 0) itmax = 0;
    __syncthreads();
    atomicMax(&itmax, iters);
    __syncthreads();
    if (threadIdx.x == 0 && itmax > 0) atomicMax(&d.ctl->kepler_max, itmax);
    note_box(d, s, b);
}

// ---------------------------------------------------------------------------
// The kick's partial rows of every body, summed (after each kick, on its
// stream).  A group of G warps (G = rows_g: enough for eight rows a warp of
// the largest system's rows, at most eight) takes 32 sorted positions, its
// lanes one position each; warp w of the group adds rows 8w .. 8w + 7 (then
// 8w + 8G .., and so on) in order, one coalesced 256-byte load a row and the
// warp's 24 loads in flight together, and the group's warps are combined by
// a fixed tree in shared memory, so the sum does not depend on the schedule.
// A block of eight warps so takes 32 (8 / G) positions.  The control word is
// read beside the rows, not before them.  Mixed form: the rows are exact
// float pairs and the sums float-float (FP32 pipe; FP64 additions would take
// this chip's FP64 pipe half the kernel), converted to FP64 at the end; FP64
// form: FP64 rows and sums.  The mixed kick writes a body's row at its
// sorted position, the FP64 kick at its index; the sum goes to ksum at the
// body's index.  Systems start at multiples of 256 positions, so a block
// lies in one system.
constexpr int kRowWarps = 8, kRowsPerWarp = 8;
template <bool MIXED>
struct RowAcc;
template <>
struct RowAcc<true> {   // float-float
    using T = float2;
    static __device__ T zero() { return make_float2(0.0f, 0.0f); }
    static __device__ T load(const double* a, int64_t i) { return reinterpret_cast<const float2*>(a)[i]; }
    static __device__ T add(T x, T y) { return ff_add(x, y); }
    static __device__ double value(T x) { return (double)x.x + (double)x.y; }
};
template <>
struct RowAcc<false> {   // FP64
    using T = double;
    static __device__ T zero() { return 0.0; }
    static __device__ T load(const double* a, int64_t i) { return a[i]; }
    static __device__ T add(T x, T y) { return x + y; }
    static __device__ double value(T x) { return x; }
};

template <bool MIXED>
__global__ void __launch_bounds__(32 * kRowWarps, 4) k_kick_rows(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlKickRows);
    using A = RowAcc<MIXED>;
    using T = typename A::T;
    __shared__ T red[kRowWarps][3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int G = d.rows_g, gw = w % G;   // the warp's place in its group of G
    const int64_t p0 = (int64_t)blockIdx.x * 32 * (kRowWarps / G);   // grid: ntot / (32 (8 / G)) blocks
    const int64_t p = p0 + (w / G) * 32 + lane;
    const int status = d.ctl->status, reprime = d.ctl->reprime;
    const int b = MIXED ? d.csorted[p] : (int)p;
    const SysInfo si = d.sys[d.body_sys[p0]];
    const int64_t local = p - si.off;
    T ax = A::zero(), ay = A::zero(), az = A::zero();
#pragma unroll 1
    for (int c0 = kRowsPerWarp * gw; c0 < si.nchunk; c0 += kRowsPerWarp * G) {
        T bx[kRowsPerWarp], by[kRowsPerWarp], bz[kRowsPerWarp];
#pragma unroll
        for (int u = 0; u < kRowsPerWarp; u++) {
            const int c = c0 + u;
            const int64_t slot = si.slot0 + (int64_t)c * si.cap + local;
            const bool in = c < si.nchunk;
            bx[u] = in ? A::load(d.pacc_x, slot) : A::zero();
            by[u] = in ? A::load(d.pacc_y, slot) : A::zero();
            bz[u] = in ? A::load(d.pacc_z, slot) : A::zero();
        }
#pragma unroll
        for (int u = 0; u < kRowsPerWarp; u++) {
            ax = A::add(ax, bx[u]);
            ay = A::add(ay, by[u]);
            az = A::add(az, bz[u]);
        }
    }
    if (status || (d.gated && !reprime)) return;   // the same for every thread of the block
    red[w][0][lane] = ax;
    red[w][1][lane] = ay;
    red[w][2][lane] = az;
    __syncthreads();
    for (int h = G / 2; h >= 1; h >>= 1) {
        if (gw < h)
            for (int q = 0; q < 3; q++) red[w][q][lane] = A::add(red[w][q][lane], red[w + h][q][lane]);
        __syncthreads();
    }
    if (gw == 0) {
        d.ksum[3 * (int64_t)b] = A::value(red[w][0][lane]);
        d.ksum[3 * (int64_t)b + 1] = A::value(red[w][1][lane]);
        d.ksum[3 * (int64_t)b + 2] = A::value(red[w][2][lane]);
    }
}

// The first group g in [a, ng) whose lowest member is at least body, for a
// whole warp: groups ascend by their lowest member, and each round the 32
// lanes test 32 evenly spaced groups of the remaining range and keep the
// stretch between the last one below and the first one not below (a range
// of ng groups takes about log32(ng) rounds, each one pair of dependent
// loads, where a one-thread bisection takes log2(ng)).
__device__ int warp_first_group_from(const Dev& d, int ng, int a, int64_t body) {
    const int lane = threadIdx.x & 31;
    int b = ng;   // the answer lies in [a, b]
    while (a < b) {
        const int step = (b - a + 31) / 32;
        const int g = a + lane * step;
        const bool below = g < b && d.members[d.goff[g]] < body;
        const int nb = __popc(__ballot_sync(0xffffffffu, below));   // the lanes below are 0 .. nb - 1
        if (nb == 0) return a;
        const int last = a + (nb - 1) * step;
        const int next = a + nb * step;
        a = last + 1;
        if (next < b) b = next;
    }
    return a;
}

// Closing half: the summed kick partials into a, jump with the momentum of
// the post-encounter state, kick, and the momentum partials the next
// step's jump needs (of V + dt/2 a, the velocities after its opening kick).
// first != 0 (create time): only a and the partials, no jump or kick.
__global__ void __launch_bounds__(kBodyThreads) k_close(Dev d, int first) {
    OPAL_TIMELINE_SCOPE(kTlClose);
    if (d.ctl->status || (d.gated && !d.ctl->reprime)) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int s = d.body_sys[(int64_t)blockIdx.x * kBodyThreads];
    const SysInfo si = d.sys[s];
    const double* J = d.Pjump + 3 * (d.nsys + s);   // the closing jump dt/2 P / M0
    const double half = 0.5 * d.p.dt, G = d.p.G;
    // the kick's partial rows, already summed by k_kick_rows
    double ax = d.ksum[3 * b], ay = d.ksum[3 * b + 1], az = d.ksum[3 * b + 2];
    // after encounters, when the kick ran beside the BS: a member's row was
    // recomputed at its new place (in parts, added here in order); every
    // other body's row gets the members' terms at their new places added (the mixed kick left the members out
    // as sources: mass 0 in its float copy), or in the FP64 form, which never
    // runs beside the BS, their old terms swapped for new ones
    if (!first && d.ctl->ninvolved > 0) {
        const bool member = d.label[b] >= 0;
        if (member) d.label[b] = -1;   // in both orders: next step's groups start from no labels
        if (d.overlap && d.alive[b]) {
            if (member) {
                ax = d.cfx[b];
                ay = d.cfy[b];
                az = d.cfz[b];
#pragma unroll
                for (int q = 1; q < kFixParts; q++) {
                    ax += d.cfx[q * d.ntot + b];
                    ay += d.cfy[q * d.ntot + b];
                    az += d.cfz[q * d.ntot + b];
                }
            } else {
                double cx = d.cfx[b], cy = d.cfy[b], cz = d.cfz[b];
#pragma unroll
                for (int q = 1; q < kFixParts; q++) {
                    cx += d.cfx[q * d.ntot + b];
                    cy += d.cfy[q * d.ntot + b];
                    cz += d.cfz[q * d.ntot + b];
                }
                ax += cx;
                ay += cy;
                az += cz;
            }
        }
    }
    ax *= G;
    ay *= G;
    az *= G;
    double px = 0, py = 0, pz = 0;
    if (d.alive[b]) {
        double x = d.x[b], y = d.y[b], z = d.z[b], vx = d.vx[b], vy = d.vy[b], vz = d.vz[b];
        if (!first) {
            x += J[0];
            y += J[1];
            z += J[2];
            vx += half * ax;
            vy += half * ay;
            vz += half * az;
            d.x[b] = x; d.y[b] = y; d.z[b] = z;
            d.vx[b] = vx; d.vy[b] = vy; d.vz[b] = vz;
        }
        d.ax[b] = ax; d.ay[b] = ay; d.az[b] = az;
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) && isfinite(vz) &&
              isfinite(ax) && isfinite(ay) && isfinite(az)))
            set_status(d.ctl, kEnonfinite, (int)b);
        double m = d.m[b];
        px = m * (vx + half * ax);
        py = m * (vy + half * ay);
        pz = m * (vz + half * az);
    } else {
        d.ax[b] = 0.0; d.ay[b] = 0.0; d.az[b] = 0.0;
    }
    segment_sums(d, (int64_t)blockIdx.x * kBodyThreads, px, py, pz, d.pP_open);
    system_total(d, d.pP_open, si, s, d.pcnt, d.Ptot + 3 * s, d.Pjump + 3 * s);
    if (!first && (int64_t)blockIdx.x * kBodyThreads == si.off && threadIdx.x < 32) {
        // energy removed by this step's mergers in this system: groups come in
        // ascending order of their lowest member, so the system's groups are the
        // run whose lowest member lies in [off, off + cap), found by two 32-way
        // searches; one warp sums them in a fixed order
        const int ng = d.ctl->ngroups;
        const int lo = warp_first_group_from(d, ng, 0, si.off);
        const int hi = warp_first_group_from(d, ng, lo, si.off + si.cap);
        double e = 0.0;
        for (int g = lo + (int)threadIdx.x; g < hi; g += 32) e += d.glost[g];
        for (int o = 16; o >= 1; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (threadIdx.x == 0 && e != 0.0) d.E_lost[s] += e;
    }
}

// Undo of a failed step (runs every step; returns at once when all is well).
__global__ void k_finish(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlFinish);
    const Ctl* c = d.ctl;
    if (!c->status) {
        if (blockIdx.x == 0 && threadIdx.x == 0) d.ctl->steps_done++;
        return;
    }
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < d.ntot;
         b += (int64_t)gridDim.x * blockDim.x) {
        d.x[b] = d.xs[b]; d.y[b] = d.ys[b]; d.z[b] = d.zs[b];
        d.vx[b] = d.vxs[b]; d.vy[b] = d.vys[b]; d.vz[b] = d.vzs[b];
        d.rc[b] = d.rcs[b];
        d.label[b] = -1;   // the step may have stopped with pairs marked but not grouped
    }
    // masses, radii and flags of group members as they were before the BS
    int nmem = c->ninvolved;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nmem; k += (int64_t)gridDim.x * blockDim.x) {
        int b = d.members[k];
        if (d.undo[3 * k + 2] >= 0.0) {   // slot written when the BS results were applied
            d.m[b] = d.undo[3 * k];
            d.hcb[b] = cbrt(d.m[b] / (3.0 * d.M0s[d.body_sys[b]]));
            d.R[b] = d.undo[3 * k + 1];
            d.alive[b] = (int)d.undo[3 * k + 2];
        }
    }
}

// get_state of system s, first pass: its momentum sum m V over the live
// bodies, by fixed-order segments (the step's closing-jump partials are free
// between steps), the total written by the system's last block.
__global__ void __launch_bounds__(kBodyThreads) k_export_sum(Dev d, int s, double* P, int* counter) {
    const SysInfo si = d.sys[s];
    const int64_t first = si.off + (int64_t)blockIdx.x * kBodyThreads;
    const int64_t b = first + threadIdx.x;
    double px = 0.0, py = 0.0, pz = 0.0;
    if (d.alive[b]) {
        const double m = d.m[b];
        px = m * d.vx[b];
        py = m * d.vy[b];
        pz = m * d.vz[b];
    }
    segment_sums(d, first, px, py, pz, d.pP_close);
    system_total(d, d.pP_close, si, s, counter, P, nullptr);
}

// second pass: one record a body for the host, (x, y, z, heliocentric v =
// V + P / M0, m, R), and its live flag
__global__ void __launch_bounds__(kBodyThreads) k_export_write(Dev d, int s, const double* P, double* rec,
                                                               int* alive) {
    const SysInfo si = d.sys[s];
    const int64_t k = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int64_t b = si.off + k;
    const double M0 = d.M0s[s];
    double* r = rec + 8 * k;
    r[0] = d.x[b];
    r[1] = d.y[b];
    r[2] = d.z[b];
    r[3] = d.vx[b] + P[0] / M0;
    r[4] = d.vy[b] + P[1] / M0;
    r[5] = d.vz[b] + P[2] / M0;
    r[6] = d.m[b];
    r[7] = d.R[b];
    alive[k] = d.alive[b];
}

// ---------------------------------------------------------------------------
// test hooks: the drift alone, and the scan inputs from a given x0, V0, x1, V1, rc
__global__ void k_debug_drift(int n, double mu, double dt, int max_iter, double* x, double* v, int* iters) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    double px = x[3 * b], py = x[3 * b + 1], pz = x[3 * b + 2], vx = v[3 * b], vy = v[3 * b + 1], vz = v[3 * b + 2];
    int it = kepler_drift(mu, dt, max_iter, px, py, pz, vx, vy, vz);
    x[3 * b] = px; x[3 * b + 1] = py; x[3 * b + 2] = pz;
    v[3 * b] = vx; v[3 * b + 1] = vy; v[3 * b + 2] = vz;
    iters[b] = it;
}

__global__ void __launch_bounds__(kBodyThreads) k_debug_scan_prep(Dev d) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = d.body_sys[(int64_t)blockIdx.x * kBodyThreads];
    if (d.alive[b]) {
        kick_floats(d, b, d.x[b], d.y[b], d.z[b], d.m[b], d.rc[b]);
        note_rcmax(d, s, d.rc[b]);
        scan_floats(d, b, d.x0[b], d.y0[b], d.z0[b], d.vx0[b], d.vy0[b], d.vz0[b], d.x[b], d.y[b], d.z[b],
                    d.vx[b], d.vy[b], d.vz[b], d.rc[b]);
    } else {
        park_floats(d, b);
    }
    note_box(d, s, b);   // every thread of the block, from this one call site
}

// create time: sort keys from the current positions, so that the first kicks
// already run on a spatially sorted body order
__global__ void __launch_bounds__(kBodyThreads) k_order_prep(Dev d) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = d.body_sys[(int64_t)blockIdx.x * kBodyThreads];
    if (d.alive[b]) d.cen[b] = make_float4((float)d.x[b], (float)d.y[b], (float)d.z[b], 0.0f);
    note_box(d, s, b);   // every thread of the block, from this one call site
}

// ---------------------------------------------------------------------------
// End of a step with star collisions or ejections on (Sec. 2.1.2): one block
// per system removes, in ascending index, every live body whose drift passed
// within the star's radius (accreted: the star's mass grows by the body's and
// the heliocentric frame moves to the merged star, every other position by
// -m_i x_i / M0'; barycentric velocities stay), then, on every eject_every-th
// step, every live body beyond r_eject.  Each removal adds the drop of the
// Hamiltonian (kinetic, stellar, mutual and |P|^2 / 2 M0 terms: O(N) sums) to
// the system's E_lost, and any removal makes the next step evaluate the
// accelerations afresh.
constexpr int kRemThreads = 256;

__device__ void remove_body(const Dev& d, const SysInfo& si, int s, int64_t i, bool accrete,
                            double (*red)[kRemThreads]) {
    const double G = d.p.G, M0 = d.M0s[s];
    const double mi = d.m[i], xi = d.x[i], yi = d.y[i], zi = d.z[i];
    const double vxi = d.vx[i], vyi = d.vy[i], vzi = d.vz[i];
    const double M0n = accrete ? M0 + mi : M0;
    const double cx = accrete ? mi * xi / M0n : 0.0, cy = accrete ? mi * yi / M0n : 0.0,
                 cz = accrete ? mi * zi / M0n : 0.0;
    // s1 = sum m/|x|, s2 = the same after (i gone, frame moved), s3 = sum m/|x - x_i|, P
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = threadIdx.x; k < si.n; k += kRemThreads) {
        const int64_t j = si.off + k;
        if (!d.alive[j] || d.m[j] == 0.0) continue;   // (a small body adds no such term)
        const double mj = d.m[j], xj = d.x[j], yj = d.y[j], zj = d.z[j];
        v[0] += mj / sqrt(xj * xj + yj * yj + zj * zj);
        v[3] += mj * d.vx[j];
        v[4] += mj * d.vy[j];
        v[5] += mj * d.vz[j];
        if (j != i) {
            const double ax = xj - cx, ay = yj - cy, az = zj - cz;
            const double bx = xj - xi, by = yj - yi, bz = zj - zi;
            v[1] += mj / sqrt(ax * ax + ay * ay + az * az);
            v[2] += mj / sqrt(bx * bx + by * by + bz * bz);
        }
    }
    __syncthreads();
    for (int c = 0; c < 6; c++) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = kRemThreads / 2; w >= 1; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 6; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double px = red[3][0], py = red[4][0], pz = red[5][0];
        const double qx = px - mi * vxi, qy = py - mi * vyi, qz = pz - mi * vzi;
        const double dE = 0.5 * mi * (vxi * vxi + vyi * vyi + vzi * vzi) - G * M0 * red[0][0] +
                          G * M0n * red[1][0] + (px * px + py * py + pz * pz) / (2.0 * M0) -
                          (qx * qx + qy * qy + qz * qz) / (2.0 * M0n) - G * mi * red[2][0];
        d.E_lost[s] += dE;
    }
    if (accrete)
        for (int64_t k = threadIdx.x; k < si.n; k += kRemThreads) {
            const int64_t j = si.off + k;
            if (!d.alive[j] || j == i) continue;
            d.x[j] -= cx;
            d.y[j] -= cy;
            d.z[j] -= cz;
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.alive[i] = 0;
        d.m[i] = 0.0;
        park_floats(d, i);
        if (accrete) d.M0s[s] = M0n;
        atomicAdd(accrete ? &d.ctl->nacc : &d.ctl->nej, 1);
        d.ctl->reprime = 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kRemThreads) k_remove(Dev d) {
    __shared__ double red[6][kRemThreads];
    __shared__ int lst[kRemThreads];
    __shared__ int wsum[kRemThreads / 32];
    if (d.ctl->status) return;
    const int s = blockIdx.x;
    const SysInfo si = d.sys[s];
    const bool eject = d.p.r_eject > 0.0 && d.p.eject_every > 0 && d.ctl->steps_done % d.p.eject_every == 0;
    const bool accrete_any = d.ctl->naccf > 0;
    if (!accrete_any && !eject) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int pass = 0; pass < 2; pass++) {
        if ((pass == 0 && !accrete_any) || (pass == 1 && !eject)) continue;
        for (int64_t c0 = 0; c0 < si.n; c0 += kRemThreads) {
            const int64_t b = si.off + c0 + threadIdx.x;
            bool want = false;
            if (c0 + (int64_t)threadIdx.x < si.n && d.alive[b]) {
                if (pass == 0) {
                    want = d.accf[b] != 0;
                } else {
                    const double x = d.x[b], y = d.y[b], z = d.z[b];
                    want = sqrt(x * x + y * y + z * z) > d.p.r_eject;
                }
            }
            // this chunk's bodies to remove, in ascending index
            const unsigned bm = __ballot_sync(0xffffffffu, want);
            if (lane == 0) wsum[warp] = __popc(bm);
            __syncthreads();
            int off = __popc(bm & ((1u << lane) - 1u)), total = 0;
            for (int w = 0; w < kRemThreads / 32; w++) {
                if (w < warp) off += wsum[w];
                total += wsum[w];
            }
            if (want) lst[off] = (int)b;
            __syncthreads();
            for (int q = 0; q < total; q++) remove_body(d, si, s, lst[q], pass == 0, red);
            __syncthreads();
        }
    }
}

// Start of a step: the counters, bounds and scratch the step's kernels
// accumulate into, zeroed or preset in one launch (rather than ten memsets).
__global__ void __launch_bounds__(256) k_step_reset(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlReset);
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    int* c = reinterpret_cast<int*>(reinterpret_cast<char*>(d.ctl) + offsetof(Ctl, ncand));
    constexpr int nc = (int)((offsetof(Ctl, steps_done) - offsetof(Ctl, ncand)) / sizeof(int));
    int* h = reinterpret_cast<int*>(d.hctl);
    constexpr int nh = (int)(sizeof(HugeCtl) / sizeof(int));
    for (int64_t i = i0; i < d.ntot; i += st) {
        d.gcount[i] = 0;
        d.accf[i] = 0;
    }
    for (int64_t i = i0; i < d.ncell; i += st) d.cstart[i] = 0;
    for (int64_t i = i0; i < nc; i += st) c[i] = 0;
    for (int64_t i = i0; i < nh; i += st) h[i] = 0;
    for (int64_t i = i0; i < d.nsys; i += st) {
        d.rcmax[i] = 0.0f;
        d.mlo[i] = 0x7f7f7f7f;                     // above any member slot
        d.mhi[i] = 0;
        d.pcnt[i] = 0;
        d.pcnt[d.nsys + i] = 0;
    }
    for (int64_t i = i0; i < 3 * d.nsys; i += st) {
        d.sbox[i] = 0x7f7f7f7f;                    // order-mapped +huge: the min starts above everything
        d.sbox[3 * d.nsys + i] = (int)0x80808080;  // and the max below
    }
}

// ---------------------------------------------------------------------------
void launch_step_reset(const Dev& d, int nsm, cudaStream_t s) {
    k_step_reset<<<2 * nsm, 256, 0, s>>>(d);
    prof_mark("memsets");
}
void launch_remove(const Dev& d, cudaStream_t s) {
    k_remove<<<d.nsys, kRemThreads, 0, s>>>(d);
    prof_mark("removals: star collisions and ejections");
}
void launch_order_prep(const Dev& d, cudaStream_t s) {
    k_order_prep<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d);
}
void launch_debug_drift(int n, double mu, double dt, int max_iter, double* x, double* v, int* iters, cudaStream_t s) {
    k_debug_drift<<<(n + 127) / 128, 128, 0, s>>>(n, mu, dt, max_iter, x, v, iters);
}
void launch_debug_scan_prep(const Dev& d, cudaStream_t s) {
    k_debug_scan_prep<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d);
}
void launch_to_dh(const Dev& d, cudaStream_t s) { k_to_dh<<<d.nsys, 256, 0, s>>>(d); }
void launch_prime(const Dev& d, cudaStream_t s) {
    k_prime<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d);
}
void launch_open(const Dev& d, cudaStream_t s) {
    k_open<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d);
    prof_mark("open: kick+jump+drift");
}
void launch_kick_rows(const Dev& d, cudaStream_t s) {
    const unsigned grid = (unsigned)(d.ntot / (32 * (kRowWarps / d.rows_g)));
    if (d.p.precision == 1) k_kick_rows<true><<<grid, 32 * kRowWarps, 0, s>>>(d);
    else k_kick_rows<false><<<grid, 32 * kRowWarps, 0, s>>>(d);
    prof_mark("kick: partial rows summed");
}
void launch_close(const Dev& d, cudaStream_t s) {
    k_close<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d, 0);
    prof_mark("close: jump+kick");
}
void launch_first_accel_finish(const Dev& d, cudaStream_t s) {
    k_close<<<(unsigned)(d.ntot / kBodyThreads), kBodyThreads, 0, s>>>(d, 1);
}
void launch_finish(const Dev& d, cudaStream_t s) {
    k_finish<<<152, 256, 0, s>>>(d);
    prof_mark("finish");
}
void launch_export(const Dev& d, int sys, int64_t cap, double* P, int* counter, double* rec, int* alive,
                   cudaStream_t s) {
    const unsigned nb = (unsigned)(cap / kBodyThreads);
    k_export_sum<<<nb, kBodyThreads, 0, s>>>(d, sys, P, counter);
    k_export_write<<<nb, kBodyThreads, 0, s>>>(d, sys, P, rec, alive);
}

}  // namespace opal
