// The kick's pair kernel: a_i = sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
// (Sec. 3.1, force block, LOOP 2, with the changeover weight K of the hybrid
// integrator).  G is applied when the partials are reduced.
//
// Work is a list of items (i-tile of 128 bodies x a j-range of the same
// system) that the blocks of a persistent grid take from a queue; each item
// writes its partial sums to its own row of a buffer that the closing kernel
// reduces in a fixed order, so results do not depend on the schedule.
// j-bodies are staged through shared memory and read by every thread of the
// block (broadcast).  Pairs closer than 2 (rc_i + rc_max) take a slow path
// that handles the changeover, the self pair and exact coincidence; all
// other pairs take the plain Newtonian fast path.
//
// Mixed form: FP32 separations of the hi parts of a hi/lo float split of the
// FP64 positions (the lo parts are added on the slow path), MUFU rsqrt, FP32
// sums over each 128-body j-tile folded into a float hi/lo pair with Knuth's
// TwoSum, converted to FP64 at the end.  FP64 form: the same in doubles.
#include "opal_internal.cuh"

namespace opal {

constexpr int kJTile = kKickJTile;

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Knuth's TwoSum: hi + lo accumulates t without losing its low-order bits.
__device__ __forceinline__ void fold(float& hi, float& lo, float t) {
    float s = hi + t;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (t - bp);
    hi = s;
    lo += err;
}

// Slow path of the mixed kick: the lo parts refine the separation, then the
// changeover weight; returns (s, dx, dy, dz) with the weighted 1/r^3 in s.
// li, lj: lo parts of i and j; rcj: rc of j (all already on chip).
__device__ __forceinline__ float4 slow_pair_f(float4 li, float4 lj, float dx, float dy, float dz, float mj,
                                              float rci, float rcj, int form) {
    dx += lj.x - li.x;
    dy += lj.y - li.y;
    dz += lj.z - li.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float s = 0.0f;
    if (r2 > 0.0f) {
        float r = sqrtf(r2);
        float rcij = fmaxf(rci, rcj);
        float K = changeover_f(r, rcij, form);
        s = mj * K / (r2 * r);
    }
    return make_float4(s, dx, dy, dz);
}

__device__ __forceinline__ double slow_pair_d(double r2, double mj, double rci, double rcj, int form) {
    if (!(r2 > 0.0)) return 0.0;
    double r = sqrt(r2);
    double rcij = fmax(rci, rcj);
    double K = changeover(r, rcij, form);
    return mj * K / (r2 * r);
}

// A block leaves the kick's item queue; the last one out empties it for the
// next launch.
__device__ __forceinline__ void queue_done(const Dev& d) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&d.ctl->kick_done, 1) == (int)gridDim.x - 1) {
            d.ctl->kick_next = 0;
            d.ctl->kick_done = 0;
            __threadfence();
        }
    }
}

// One staged j-tile against the thread's NI i-bodies.  NEAR: some pair may be
// closer than the i-body's threshold, so every pair is tested and the close
// ones take the slow path; otherwise every pair is a plain Newtonian term.
template <int NI, bool NEAR, int NJ>
__device__ __forceinline__ void kick_tile(const float4* sj, const float4* sl, const float* src, int nj,
                                          const float (&xi)[NI], const float (&yi)[NI], const float (&zi)[NI],
                                          const float (&thr)[NI], const float (&rci)[NI], const float4 (&li)[NI],
                                          int form, float (&tx)[NI], float (&ty)[NI], float (&tz)[NI]) {
    // NJ > 0: a full tile, the trip count known at compile time.  Near tiles
    // are few: a rolled loop keeps their registers down.
    const int n = NJ > 0 ? NJ : nj;
#pragma unroll(NEAR ? 2 : 8)
    for (int jj = 0; jj < n; jj++) {
        const float4 pj = sj[jj];
#pragma unroll
        for (int q = 0; q < NI; q++) {
            float dx = pj.x - xi[q], dy = pj.y - yi[q], dz = pj.z - zi[q];
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float s;
            if (NEAR && r2 < thr[q]) {
                float4 r = slow_pair_f(li[q], sl[jj], dx, dy, dz, pj.w, rci[q], src[jj], form);
                s = r.x;
                dx = r.y;
                dy = r.z;
                dz = r.w;
            } else {
                float ri = rsqrt_approx(r2);
                s = (pj.w * ri) * (ri * ri);
            }
            tx[q] = fmaf(s, dx, tx[q]);
            ty[q] = fmaf(s, dy, ty[q]);
            tz[q] = fmaf(s, dz, tz[q]);
        }
    }
}

// Box of the points the block's threads hold (each thread: its own box bl, bh,
// empty when have is false), reduced over the block through red; every
// thread gets the result.  An empty box comes out with lo > hi.  The caller
// makes sure no thread still reads red from an earlier use.
template <int T>
__device__ __forceinline__ void block_box(bool have, const float (&bl)[3], const float (&bh)[3],
                                          int (*red)[T / 32], float (&lo)[3], float (&hi)[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int a = __reduce_min_sync(0xffffffffu, have ? ford(bl[k]) : 0x7fffffff);
        const int b = __reduce_max_sync(0xffffffffu, have ? ford(bh[k]) : (int)0x80000000);
        if ((threadIdx.x & 31) == 0) {
            red[k][threadIdx.x >> 5] = a;
            red[k + 3][threadIdx.x >> 5] = b;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int a = red[k][0], b = red[k + 3][0];
#pragma unroll
        for (int wq = 1; wq < T / 32; wq++) {
            a = min(a, red[k][wq]);
            b = max(b, red[k + 3][wq]);
        }
        lo[k] = fordinv(a);
        hi[k] = fordinv(b);
    }
}

__device__ __forceinline__ void box_add(const float4& p, bool& have, float (&bl)[3], float (&bh)[3]) {
    if (p.x < 0.5f * kFar) {   // parked (dead or padding) bodies stay out
        bl[0] = fminf(bl[0], p.x); bl[1] = fminf(bl[1], p.y); bl[2] = fminf(bl[2], p.z);
        bh[0] = fmaxf(bh[0], p.x); bh[1] = fmaxf(bh[1], p.y); bh[2] = fmaxf(bh[2], p.z);
        have = true;
    }
}

// Items index the system's bodies in the order the encounter scan sorted
// them (cells of the path midpoints, so a 128-body tile is compact).  Each
// staged j-tile gets its box; when that box is farther from the i-tile's box
// than the largest i threshold allows, no pair of the tile can need the slow
// path and the tile runs without the per-pair test.
template <int T, int NI, int MINB>
__global__ void __launch_bounds__(T, MINB) k_kick_mixed(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    if (d.gated && !d.ctl->reprime) return;   // the re-evaluation after a removal, with none
    constexpr int JPT = kJTile / T;   // j records each thread stages
    __shared__ float4 sj[kJTile];
    __shared__ int sid[kJTile];
    __shared__ float4 sl[kJTile];     // lo parts and rc of the j-tile, staged only when it is near
    __shared__ float src[kJTile];
    __shared__ int red[6][T / 32];
    __shared__ int red_t[T / 32];
    __shared__ int s_item;
    if (d.ctl->status) return;
    const int form = d.p.changeover;
    for (;;) {
        // items are taken in list order (largest first) by whichever block is free
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&d.ctl->kick_next, 1);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= nitems) break;
        const KickItem w = items[it];
        const SysInfo si = d.sys[w.sys];
        const float rcm = d.rcmax[w.sys];
        float xi[NI], yi[NI], zi[NI], thr[NI], rci[NI];
        float4 li[NI];
        int ii[NI];
        float hx[NI], hy[NI], hz[NI], lx[NI], ly[NI], lz[NI];
        float tmax = 0.0f;
        bool ihave = false;
        float ibl[3] = {3.0e38f, 3.0e38f, 3.0e38f}, ibh[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
        for (int q = 0; q < NI; q++) {
            ii[q] = d.csorted[w.i0 + q * T + threadIdx.x];
            const float4 h = d.kh[ii[q]];
            xi[q] = h.x; yi[q] = h.y; zi[q] = h.z;
            rci[q] = d.rcf[ii[q]];
            li[q] = d.kl[ii[q]];
            float t = 2.0f * (rci[q] + rcm);
            thr[q] = fmaxf(t * t, 1e-30f);
            if (h.x < 0.5f * kFar) tmax = fmaxf(tmax, thr[q]);
            box_add(h, ihave, ibl, ibh);
            hx[q] = hy[q] = hz[q] = lx[q] = ly[q] = lz[q] = 0.0f;
        }
        // box of the i-tile and its largest threshold (>= 0: its bits order as its values)
        float ilo[3], ihi[3];
        __syncthreads();
        {
            const int tm = __reduce_max_sync(0xffffffffu, __float_as_int(tmax));
            if ((threadIdx.x & 31) == 0) red_t[threadIdx.x >> 5] = tm;
        }
        block_box<T>(ihave, ibl, ibh, red, ilo, ihi);
        {
            int t_all = red_t[0];
#pragma unroll
            for (int wq = 1; wq < T / 32; wq++) t_all = max(t_all, red_t[wq]);
            tmax = __int_as_float(t_all) * 1.001f;
        }
        // j records: with few per thread, each tile's are fetched while the
        // previous tile runs (PF); otherwise at the start of the tile
        constexpr bool PF = JPT <= 2;
        int pid[JPT];
        float4 ph[JPT];
        if (PF) {
#pragma unroll
            for (int u = 0; u < JPT; u++) {
                const int64_t k = (int64_t)u * T + threadIdx.x;
                pid[u] = w.j0 + k < w.j1 ? d.csorted[w.j0 + k] : -1;
            }
#pragma unroll
            for (int u = 0; u < JPT; u++) ph[u] = pid[u] >= 0 ? d.kh[pid[u]] : make_float4(kFar, kFar, kFar, 0.0f);
        }
        for (int64_t jb = w.j0; jb < w.j1; jb += kJTile) {
            const int nj = (int)min((int64_t)kJTile, w.j1 - jb);
            __syncthreads();
            if (!PF) {
#pragma unroll
                for (int u = 0; u < JPT; u++) {
                    const int64_t k = jb + (int64_t)u * T + threadIdx.x;
                    pid[u] = k < w.j1 ? d.csorted[k] : -1;
                }
#pragma unroll
                for (int u = 0; u < JPT; u++)
                    ph[u] = pid[u] >= 0 ? d.kh[pid[u]] : make_float4(kFar, kFar, kFar, 0.0f);
            }
            bool have = false;
            float bl[3] = {3.0e38f, 3.0e38f, 3.0e38f}, bh[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
            int cid[JPT];
#pragma unroll
            for (int u = 0; u < JPT; u++) {
                const int k = u * T + threadIdx.x;
                cid[u] = pid[u];
                if (k < nj) {
                    sj[k] = ph[u];
                    sid[k] = pid[u];
                    box_add(ph[u], have, bl, bh);
                }
            }
            if (PF) {   // the next tile's records; their latency hides behind this tile
                const int64_t jn = jb + kJTile;
#pragma unroll
                for (int u = 0; u < JPT; u++) {
                    const int64_t k = jn + (int64_t)u * T + threadIdx.x;
                    pid[u] = k < w.j1 ? d.csorted[k] : -1;
                }
#pragma unroll
                for (int u = 0; u < JPT; u++)
                    ph[u] = pid[u] >= 0 ? d.kh[pid[u]] : make_float4(kFar, kFar, kFar, 0.0f);
            }
            float jlo[3], jhi[3];
            block_box<T>(have, bl, bh, red, jlo, jhi);
            // squared gap between the boxes (huge when either is empty)
            float g2 = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float g = fmaxf(0.0f, fmaxf(jlo[k] - ihi[k], ilo[k] - jhi[k]));
                g2 = fmaf(g, g, g2);
            }
            float tx[NI], ty[NI], tz[NI];
#pragma unroll
            for (int q = 0; q < NI; q++) tx[q] = ty[q] = tz[q] = 0.0f;
            if (g2 < tmax) {   // block-uniform: stage what the slow path needs
#pragma unroll
                for (int u = 0; u < JPT; u++) {
                    const int k = u * T + threadIdx.x;
                    if (k < nj) {
                        sl[k] = d.kl[cid[u]];
                        src[k] = d.rcf[cid[u]];
                    }
                }
                __syncthreads();
                if (nj == kJTile)
                    kick_tile<NI, true, kJTile>(sj, sl, src, nj, xi, yi, zi, thr, rci, li, form, tx, ty, tz);
                else
                    kick_tile<NI, true, 0>(sj, sl, src, nj, xi, yi, zi, thr, rci, li, form, tx, ty, tz);
            } else if (nj == kJTile) {
                kick_tile<NI, false, kJTile>(sj, sl, src, nj, xi, yi, zi, thr, rci, li, form, tx, ty, tz);
            } else {
                kick_tile<NI, false, 0>(sj, sl, src, nj, xi, yi, zi, thr, rci, li, form, tx, ty, tz);
            }
#pragma unroll
            for (int q = 0; q < NI; q++) {
                fold(hx[q], lx[q], tx[q]);
                fold(hy[q], ly[q], ty[q]);
                fold(hz[q], lz[q], tz[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NI; q++) {
            int64_t slot = si.slot0 + (int64_t)w.chunk * si.cap + (ii[q] - si.off);
            d.pacc_x[slot] = (double)hx[q] + (double)lx[q];
            d.pacc_y[slot] = (double)hy[q] + (double)ly[q];
            d.pacc_z[slot] = (double)hz[q] + (double)lz[q];
        }
    }
    queue_done(d);
}

template <int T>
__global__ void __launch_bounds__(T) k_kick_fp64(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    if (d.gated && !d.ctl->reprime) return;   // the re-evaluation after a removal, with none
    __shared__ D4 sj[kJTile];
    __shared__ int s_item;
    if (d.ctl->status) return;
    const int form = d.p.changeover;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&d.ctl->kick_next, 1);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= nitems) break;
        const KickItem w = items[it];
        const SysInfo si = d.sys[w.sys];
        const double rcm = (double)d.rcmax[w.sys];
        const int64_t i = w.i0 + threadIdx.x;
        const double xi = d.x[i], yi = d.y[i], zi = d.z[i], rci = d.rc[i];
        double t = 2.0 * (rci + rcm);
        const double thr = fmax(t * t, 1e-300);
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (int64_t jb = w.j0; jb < w.j1; jb += kJTile) {
            const int nj = (int)min((int64_t)kJTile, w.j1 - jb);
            __syncthreads();
            for (int k = threadIdx.x; k < nj; k += T) {
                int64_t j = jb + k;
                sj[k] = D4{d.x[j], d.y[j], d.z[j], d.m[j]};
            }
            __syncthreads();
#pragma unroll 2
            for (int jj = 0; jj < nj; jj++) {
                const D4 pj = sj[jj];
                double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
                double r2 = dx * dx + dy * dy + dz * dz;
                double s;
                if (r2 < thr) {
                    s = slow_pair_d(r2, pj.w, rci, d.rc[jb + jj], form);
                } else {
                    double ri = rsqrt(r2);
                    s = (pj.w * ri) * (ri * ri);
                }
                ax += s * dx;
                ay += s * dy;
                az += s * dz;
            }
        }
        int64_t slot = si.slot0 + (int64_t)w.chunk * si.cap + (i - si.off);
        d.pacc_x[slot] = ax;
        d.pacc_y[slot] = ay;
        d.pacc_z[slot] = az;
    }
    queue_done(d);
}

// ---------------------------------------------------------------------------
// After the encounter integrator.  k_kick_apply puts each member's BS result
// into the state, keeping the old float copies and position.  When the kick
// ran beside the BS (overlap), on the state after the drift, its partial rows
// hold every group member at its old place, and k_kick_fix then
//   - recomputes the full row of each member at its new place,
//   - for every other body swaps the members' old terms for their new ones,
//   - sums m V per 64-body segment for the closing jump (after the mergers;
//     this part runs in both orders).
// A pair's term is computed exactly as the kick computes it: the slow path
// when r^2 < (2 (rc_i + rc_max))^2, where the kick's tile test sends it too.

// one pair term of the mixed kick: i (hi, lo, rc, threshold) and j (hi, lo, rc)
__device__ __forceinline__ float3 term_f(float4 hi, float4 li, float rci, float thr, float4 hj, float4 lj, float rcj,
                                         int form) {
    float dx = hj.x - hi.x, dy = hj.y - hi.y, dz = hj.z - hi.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float s;
    if (r2 < thr) {
        float4 r = slow_pair_f(li, lj, dx, dy, dz, hj.w, rci, rcj, form);
        s = r.x;
        dx = r.y;
        dy = r.z;
        dz = r.w;
    } else {
        float ri = rsqrt_approx(r2);
        s = (hj.w * ri) * (ri * ri);
    }
    return make_float3(s * dx, s * dy, s * dz);
}

// one pair term of the FP64 kick
__device__ __forceinline__ void term_d(double xi, double yi, double zi, double rci, double thr, const D4& pj,
                                       double rcj, int form, double& ax, double& ay, double& az) {
    double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
    double r2 = dx * dx + dy * dy + dz * dz;
    double s;
    if (r2 < thr) {
        s = slow_pair_d(r2, pj.w, rci, rcj, form);
    } else {
        double ri = rsqrt(r2);
        s = (pj.w * ri) * (ri * ri);
    }
    ax = s * dx;
    ay = s * dy;
    az = s * dz;
}

__global__ void __launch_bounds__(256) k_kick_apply(Dev d) {
    if (d.ctl->status) return;
    const int nm = d.ctl->ninvolved;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nm; k += gridDim.x * blockDim.x) {
        const int g = d.members[k];
        const int s = d.body_sys[g];
        atomicMin(&d.mlo[s], k);
        atomicMax(&d.mhi[s], k + 1);
        d.undo[3 * k] = d.m[g];
        d.undo[3 * k + 1] = d.R[g];
        d.undo[3 * k + 2] = (double)d.alive[g];
        d.okx[k] = D4{d.x[g], d.y[g], d.z[g], d.m[g]};
        const double* o = d.bsout + (int64_t)kBsOut * k;
        if (o[8] < 0.0) {   // no encounter kernel wrote this member's result
            set_status(d.ctl, kEoverflow, -6);
            continue;
        }
        d.x[g] = o[0]; d.y[g] = o[1]; d.z[g] = o[2];
        d.vx[g] = o[3]; d.vy[g] = o[4]; d.vz[g] = o[5];
        d.m[g] = o[6];
        d.hcb[g] = cbrt(o[6] / (3.0 * d.M0s[s]));
        d.R[g] = o[7];
        const int al = (int)o[8];
        d.alive[g] = al;
        if (al) kick_floats(d, g, o[0], o[1], o[2], o[6], d.rc[g]);
        else park_floats(d, g);
    }
}

constexpr int kFixThreads = kBodyThreads;

__global__ void __launch_bounds__(kFixThreads) k_kick_fix(Dev d, int nbody_blocks) {
    __shared__ float4 snh[kFixThreads], snl[kFixThreads];
    __shared__ float snr[kFixThreads];
    __shared__ D4 snx[kFixThreads], sox[kFixThreads];
    __shared__ double snrd[kFixThreads];
    __shared__ double red[3][kFixThreads];
    __shared__ int wcnt[kFixThreads / 32];
    if (d.ctl->status) return;
    const int nm = d.ctl->ninvolved;
    const int form = d.p.changeover;
    const bool mixed = d.p.precision == 1;
    if ((int)blockIdx.x < nbody_blocks * kFixParts) {
        // body block bb, part q of the system's members (q = 0 also sums momenta)
        const int bb = (int)blockIdx.x % nbody_blocks, q = (int)blockIdx.x / nbody_blocks;
        const int64_t b = (int64_t)bb * kFixThreads + threadIdx.x;
        const int s = d.body_sys[(int64_t)bb * kFixThreads];
        const bool al = d.alive[b] != 0;
        if (q == 0) {
            const double m = al ? d.m[b] : 0.0;
            segment_sums(d, (int64_t)bb * kFixThreads, m * d.vx[b], m * d.vy[b], m * d.vz[b], d.pP_close);
            system_total(d, d.pP_close, d.sys[s], s, d.pcnt + d.nsys, d.Ptot + 3 * (d.nsys + s));
        }
        if (nm == 0 || !d.overlap) return;
        const int ka = d.mlo[s], kz = d.mhi[s];
        const int k0 = ka + (int)((int64_t)(kz - ka) * q / kFixParts);
        const int k1 = ka + (int)((int64_t)(kz - ka) * (q + 1) / kFixParts);
        const int64_t big_end = d.sys[s].off + d.sys[s].nb;
        const bool want = al && d.label[b] < 0;   // members get their full rows below
        const float rcm = d.rcmax[s];
        // i-side values of both forms
        const float4 hi = d.kh[b], li = d.kl[b];
        const float rci = d.rcf[b];
        const float tf = 2.0f * (rci + rcm);
        const float thrf = fmaxf(tf * tf, 1e-30f);
        const double xi = d.x[b], yi = d.y[b], zi = d.z[b], rcid = d.rc[b];
        const double td = 2.0 * (rcid + (double)rcm);
        const double thrd = fmax(td * td, 1e-300);
        // mixed: the members' new terms (the kick left them out as sources)
        // summed in float and folded into hi/lo pairs (FP64 arithmetic costs
        // far more on this chip); FP64: new minus old terms, in doubles
        double cx = 0.0, cy = 0.0, cz = 0.0;
        float hx = 0.0f, hy = 0.0f, hz = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
        for (int kb = k0; kb < k1; kb += kFixThreads) {
            const int nk = min(kFixThreads, k1 - kb);
            __syncthreads();
            // only members that were big at the start of the step are sources
            // (a small one adds nothing, old or new), so only they are staged
            const int k = kb + threadIdx.x;
            const int g = (int)threadIdx.x < nk ? d.members[k] : -1;
            const bool src = g >= 0 && g < big_end;
            const unsigned bm = __ballot_sync(0xffffffffu, src);
            if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = __popc(bm);
            __syncthreads();
            int slot = __popc(bm & ((1u << (threadIdx.x & 31)) - 1u)), n = 0;
#pragma unroll
            for (int w = 0; w < kFixThreads / 32; w++) {
                if (w < (int)(threadIdx.x >> 5)) slot += wcnt[w];
                n += wcnt[w];
            }
            if (src) {
                if (mixed) {
                    snh[slot] = d.kh[g];
                    snl[slot] = d.kl[g];
                    snr[slot] = d.rcf[g];
                } else {
                    snx[slot] = D4{d.x[g], d.y[g], d.z[g], d.m[g]};
                    sox[slot] = d.okx[k];
                    snrd[slot] = d.rc[g];
                }
            }
            __syncthreads();
            if (!want || n == 0) continue;
            if (mixed) {
                // the kick left the members out as sources: their new terms only
                float tx = 0.0f, ty = 0.0f, tz = 0.0f;
                for (int q = 0; q < n; q++) {
                    const float3 tn = term_f(hi, li, rci, thrf, snh[q], snl[q], snr[q], form);
                    tx += tn.x;
                    ty += tn.y;
                    tz += tn.z;
                }
                fold(hx, lx, tx);
                fold(hy, ly, ty);
                fold(hz, lz, tz);
                continue;
            }
            for (int q = 0; q < n; q++) {
                {
                    double nx, ny, nz, ox, oy, oz;
                    term_d(xi, yi, zi, rcid, thrd, snx[q], snrd[q], form, nx, ny, nz);
                    term_d(xi, yi, zi, rcid, thrd, sox[q], snrd[q], form, ox, oy, oz);
                    cx += nx - ox;
                    cy += ny - oy;
                    cz += nz - oz;
                }
            }
        }
        if (want) {
            if (mixed) {
                cx = (double)hx + (double)lx;
                cy = (double)hy + (double)ly;
                cz = (double)hz + (double)lz;
            }
            const int64_t o = (int64_t)q * d.ntot + b;   // this part's share of the correction
            d.cfx[o] = cx;
            d.cfy[o] = cy;
            d.cfz[o] = cz;
        }
        return;
    }
    // member rows, one block per member at a time
    if (!d.overlap) return;
    const int first = nbody_blocks * kFixParts;
    for (int k = (int)blockIdx.x - first; k < nm; k += (int)gridDim.x - first) {
        const int g = d.members[k];
        const int s = d.body_sys[g];
        const SysInfo si = d.sys[s];
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (d.alive[g]) {
            const float rcm = d.rcmax[s];
            const float4 hi = d.kh[g], li = d.kl[g];
            const float rci = d.rcf[g];
            const float tf = 2.0f * (rci + rcm);
            const float thrf = fmaxf(tf * tf, 1e-30f);
            const double xi = d.x[g], yi = d.y[g], zi = d.z[g], rcid = d.rc[g];
            const double td = 2.0 * (rcid + (double)rcm);
            const double thrd = fmax(td * td, 1e-300);
            if (mixed) {
                // float sums of 16 terms at a time, folded into hi/lo pairs
                float hx = 0.0f, hy = 0.0f, hz = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
                const int64_t jend = si.off + si.nb;   // sources: the big bodies
                for (int64_t j0 = si.off + threadIdx.x; j0 < jend; j0 += 8 * kFixThreads) {
                    // eight records loaded together (their latencies overlap); lo parts
                    // and rc only for the rare pair that takes the slow path
                    float4 hj[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int64_t j = j0 + (int64_t)u * kFixThreads;
                        hj[u] = (j < jend && j != g) ? d.kh[j] : make_float4(kFar, kFar, kFar, 0.0f);
                    }
                    float tx = 0.0f, ty = 0.0f, tz = 0.0f;
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int64_t j = j0 + (int64_t)u * kFixThreads;
                        float dx = hj[u].x - hi.x, dy = hj[u].y - hi.y, dz = hj[u].z - hi.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        float sv;
                        if (r2 < thrf) {
                            const float4 r = slow_pair_f(li, d.kl[j], dx, dy, dz, hj[u].w, rci, d.rcf[j], form);
                            sv = r.x;
                            dx = r.y;
                            dy = r.z;
                            dz = r.w;
                        } else {
                            const float ri = rsqrt_approx(r2);
                            sv = (hj[u].w * ri) * (ri * ri);
                        }
                        tx += sv * dx;
                        ty += sv * dy;
                        tz += sv * dz;
                    }
                    fold(hx, lx, tx);
                    fold(hy, ly, ty);
                    fold(hz, lz, tz);
                }
                ax = (double)hx + (double)lx;
                ay = (double)hy + (double)ly;
                az = (double)hz + (double)lz;
            } else for (int64_t j = si.off + threadIdx.x; j < si.off + si.nb; j += kFixThreads) {
                if (j == g) continue;
                {
                    double tx, ty, tz;
                    term_d(xi, yi, zi, rcid, thrd, D4{d.x[j], d.y[j], d.z[j], d.m[j]}, d.rc[j], form, tx, ty, tz);
                    ax += tx;
                    ay += ty;
                    az += tz;
                }
            }
        }
        __syncthreads();
        red[0][threadIdx.x] = ax;
        red[1][threadIdx.x] = ay;
        red[2][threadIdx.x] = az;
        __syncthreads();
        for (int w = kFixThreads / 2; w >= 1; w >>= 1) {
            if ((int)threadIdx.x < w) {
                red[0][threadIdx.x] += red[0][threadIdx.x + w];
                red[1][threadIdx.x] += red[1][threadIdx.x + w];
                red[2][threadIdx.x] += red[2][threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            d.cfx[g] = red[0][0];
            d.cfy[g] = red[1][0];
            d.cfz[g] = red[2][0];
        }
    }
}

void launch_bs_apply(const Dev& d, int nsm, cudaStream_t s) {
    k_kick_apply<<<nsm, 256, 0, s>>>(d);
    prof_mark("apply BS results");
}

void launch_kick_fix(const Dev& d, int nsm, cudaStream_t s) {
    const int nb = (int)(d.ntot / kFixThreads);
    k_kick_fix<<<nb * kFixParts + 2 * nsm, kFixThreads, 0, s>>>(d, nb);
    prof_mark("kick fix: member rows and corrections");
}

// Kick variants the autotuner picks from: (threads, i-bodies per thread,
// minimum resident blocks); every variant covers a 128-body i-tile.
struct KickVariant {
    const char* name;
    int threads;
    int ni;           // i-bodies per thread: an item's i-tile is threads x ni bodies
    void (*launch)(const Dev&, const KickItem*, int64_t, int, cudaStream_t);
    int (*occupancy)();
    int (*regs)();
};

template <int T, int NI, int MINB>
void launch_mixed(const Dev& d, const KickItem* items, int64_t nitems, int grid, cudaStream_t s) {
    k_kick_mixed<T, NI, MINB><<<grid, T, 0, s>>>(d, items, nitems);
}
template <int T, int NI, int MINB>
int occ_mixed() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kick_mixed<T, NI, MINB>, T, 0);
    return nb;
}
template <int T, int NI, int MINB>
int regs_mixed() {
    cudaFuncAttributes a{};
    cudaFuncGetAttributes(&a, k_kick_mixed<T, NI, MINB>);
    return a.numRegs;
}
template <int T>
int regs_fp64() {
    cudaFuncAttributes a{};
    cudaFuncGetAttributes(&a, k_kick_fp64<T>);
    return a.numRegs;
}
template <int T>
void launch_fp64(const Dev& d, const KickItem* items, int64_t nitems, int grid, cudaStream_t s) {
    k_kick_fp64<T><<<grid, T, 0, s>>>(d, items, nitems);
}
template <int T>
int occ_fp64() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_kick_fp64<T>, T, 0);
    return nb;
}

static const KickVariant kMixed[] = {
    {"mixed t128 i1", 128, 1, launch_mixed<128, 1, 6>, occ_mixed<128, 1, 6>, regs_mixed<128, 1, 6>},
    {"mixed t64 i2", 64, 2, launch_mixed<64, 2, 12>, occ_mixed<64, 2, 12>, regs_mixed<64, 2, 12>},
    {"mixed t128 i2", 128, 2, launch_mixed<128, 2, 4>, occ_mixed<128, 2, 4>, regs_mixed<128, 2, 4>},
    {"mixed t128 i1 r", 128, 1, launch_mixed<128, 1, 4>, occ_mixed<128, 1, 4>, regs_mixed<128, 1, 4>},
    {"mixed t128 i1 5", 128, 1, launch_mixed<128, 1, 5>, occ_mixed<128, 1, 5>, regs_mixed<128, 1, 5>},
};
static const KickVariant kFp64[] = {
    {"fp64 t128", 128, 1, launch_fp64<128>, occ_fp64<128>, regs_fp64<128>},
};

int kick_num_variants(int precision) {
    return precision == 1 ? (int)(sizeof(kMixed) / sizeof(kMixed[0])) : (int)(sizeof(kFp64) / sizeof(kFp64[0]));
}
const char* kick_variant_name(int precision, int v) { return precision == 1 ? kMixed[v].name : kFp64[v].name; }
int kick_itile(int precision, int v) {
    const KickVariant& k = precision == 1 ? kMixed[v] : kFp64[v];
    return k.threads * k.ni;
}
// registers one block holds as the SM allocates them (per warp, in units of
// 8 per thread)
int kick_block_regs(int precision, int v) {
    const KickVariant& k = precision == 1 ? kMixed[v] : kFp64[v];
    return k.threads * ((k.regs() + 7) / 8 * 8);
}
int kick_occupancy(int precision, int v) { return precision == 1 ? kMixed[v].occupancy() : kFp64[v].occupancy(); }
int kick_threads(int precision, int v) { return precision == 1 ? kMixed[v].threads : kFp64[v].threads; }
void launch_kick(const Dev& d, const KickItem* items, int64_t nitems, int grid, int precision, int v,
                 cudaStream_t s) {
    if (precision == 1) kMixed[v].launch(d, items, nitems, grid, s);
    else kFp64[v].launch(d, items, nitems, grid, s);
    prof_mark("kick");
}

}  // namespace opal
