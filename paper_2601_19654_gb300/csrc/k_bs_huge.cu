// Bulirsch-Stoer of an encounter group of more than 64 members (a giant
// planet's critical sphere holding hundreds of small bodies), on the whole
// GPU: one group at a time, the blocks in step through grid-wide barriers.
//
// The method is the sequential one of the small-group kernels (Sec. 2.1.1
// footnote 2; modified midpoint n_k = 2, 4, ..., 16, Neville extrapolation in
// h^2, the same acceptance test and step control, perfect mergers in the
// sequential order after each accepted substep).  Each derivative evaluation
// is split in two phases:
//   pairs:   one warp per (member b, chunk of 64 members): an FP32 test with a
//            margin far above FP32 rounding sends the pairs that may be inside
//            the critical distance to the FP64 (1 - K) term; the warp's sum
//            goes to its (b, chunk) slot;
//   members: one thread per member: Kepler term plus the chunk slots in chunk
//            order, then the midpoint step (or, at a sequence's end, its row of
//            the tableau and the error, folded into a grid-wide maximum).
// Every thread takes the same decisions from the same values in global
// memory, so the control flow is identical in all blocks.  A barrier that
// waits longer than its limit (four seconds; a test hook sets it shorter)
// sets an abort flag: every block leaves and the step reports OPAL_EBS.
#include "opal_internal.cuh"

namespace opal {

constexpr int kHugeThreads = 256;
constexpr int kHugeChunk = 64;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier (all blocks of the launch are resident); false once aborted.
// Each wait is bounded by wait_ns of the global timer.  hold (a test hook):
// the last block to arrive does not release the others but waits too, so
// every wait runs out, as if a block never arrived.
__device__ bool huge_sync(HugeCtl* hc, unsigned long long wait_ns, int hold) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = &hc->bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&hc->bar_count, 1u) == gridDim.x - 1 && !hold) {
            hc->bar_count = 0;   // nobody adds again before the generation moves
            __threadfence();
            atomicAdd(&hc->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (*(volatile int*)&hc->abort) break;
                if (global_ns() - t0 > wait_ns) {
                    atomicExch(&hc->abort, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&hc->abort == 0;
}

// (1 - K) term of member b against o (as the small-group kernels compute it),
// at the positions pos ([3][cap]) of one sequence's evaluation point
__device__ __forceinline__ void huge_pair(const Dev& d, const Params& p, const double* pos, int b, int o, double xb,
                                          double yb, double zb, double& ax, double& ay, double& az) {
    const HugeBuf& H = d.hb;
    if (le_zero(H.m[o])) return;   // a small body (m = 0): no source
    const int w = gt_nonneg(H.rc[b], H.rc[o]) ? b : o;
    const double rc = H.rc[w];
    const int64_t c = H.cap;
    const double dx = pos[o] - xb, dy = pos[c + o] - yb, dz = pos[2 * c + o] - zb;
    const double dr2 = dx * dx + dy * dy + dz * dz;
    if (ge_nonneg(dr2, rc * rc)) return;   // 1 - K = 0 at or beyond rc
    const double dri = rsqrt(dr2), dr = dr2 * dri;
    if (ge_nonneg(dr, rc)) return;
    const double t = mutual_factor(p.G * H.m[o] * (dri * dri * dri), (dr - 0.1 * rc) * H.pinv[w], p.changeover);
    ax += t * dx;
    ay += t * dy;
    az += t * dz;
}

// Chunk culling.  The pair phase tests a pair in FP32 against
// lim = max(rc_b, rc_o) + slack_b; a chunk whose box of float positions
// (with its largest rc) lies farther from member b than max(rc_b, rc_max) +
// slack_b holds no pair that passes, since FP32 subtraction, squares and sums
// round monotonically (the factor 1.001 covers a contraction into an FMA).
// The pair phase skips such a (member, chunk) task and the member phase,
// taking the same decision from the same values, skips its slot: culled
// chunks would only add zeros.
__device__ __forceinline__ bool chunk_culled(float4 pb, float4 blo, float4 bhi) {
    const float slack = 1e-5f * (1.0f + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z));
    const float lim = fmaxf(pb.w, blo.w) + slack;
    const float gx = fmaxf(0.0f, fmaxf(blo.x - pb.x, pb.x - bhi.x));
    const float gy = fmaxf(0.0f, fmaxf(blo.y - pb.y, pb.y - bhi.y));
    const float gz = fmaxf(0.0f, fmaxf(blo.z - pb.z, pb.z - bhi.z));
    return gx * gx + gy * gy + gz * gz > lim * lim * 1.001f;
}

// chunk boxes of sequence k for round parity par: two float4 per chunk
__device__ __forceinline__ float4* huge_cbox(const HugeBuf& H, int par, int k) {
    const int64_t nch = (H.cap + kHugeChunk - 1) / kHugeChunk;
    return H.cbox + 2 * (((int64_t)par * kBsRows + k) * nch);
}

// Box of the float positions held by each 64 consecutive threads of the
// block (one chunk: two warps), members with have = false left out; the
// group's first thread writes it to dst (two float4: lo xyz and the largest
// rc, hi xyz; an empty chunk gets lo = +3e38, hi = -3e38).  Every thread of
// the block calls it: it synchronises the block.
__device__ void chunk_box_store(bool have, float4 p, float4* dst, int (*red)[kHugeThreads / 32]) {
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const float c[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int lo = __reduce_min_sync(0xffffffffu, have ? ford(c[k]) : 0x7fffffff);
        const int hi = __reduce_max_sync(0xffffffffu, have ? ford(c[k]) : (int)0x80000000);
        if (lane == 0) {
            red[k][wq] = lo;
            red[3 + k][wq] = hi;
        }
    }
    const int wm = __reduce_max_sync(0xffffffffu, have ? __float_as_int(p.w) : 0);   // rc >= 0
    if (lane == 0) red[6][wq] = wm;
    __syncthreads();
    if ((threadIdx.x & 63) == 0 && dst) {
        int v[7];
        for (int k = 0; k < 7; k++)
            v[k] = (k < 3) ? min(red[k][wq], red[k][wq + 1]) : max(red[k][wq], red[k][wq + 1]);
        if (v[0] == 0x7fffffff) {
            dst[0] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.0f);
            dst[1] = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.0f);
        } else {
            dst[0] = make_float4(fordinv(v[0]), fordinv(v[1]), fordinv(v[2]), __int_as_float(v[6]));
            dst[1] = make_float4(fordinv(v[3]), fordinv(v[4]), fordinv(v[5]), 0.0f);
        }
    }
    __syncthreads();
}

// 2D Morton key of a point quantised to 16 bits an axis
__device__ __forceinline__ unsigned int spread16(unsigned int v) {
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Slots of sequence k: positions, float positions and the pair sums.
__device__ __forceinline__ const double* huge_pos(const HugeBuf& H, int k) { return H.pos + (int64_t)k * 3 * H.cap; }
__device__ __forceinline__ double* huge_part(const HugeBuf& H, int k) {
    return H.part + (int64_t)k * 3 * H.cap * ((H.cap + kHugeChunk - 1) / kHugeChunk);
}

// pair phase of one round: every (sequence, member, chunk) slot of the nact
// sequences k0 .. k0 + nact - 1, from their evaluation points and the chunk
// boxes of round parity par; chunks are runs of 64 members in spatial order.
// A task takes one member and kHugeGroup chunks (its lanes test the chunks'
// boxes together, then the chunks that can hold a pair run one after
// another), except for the nwide members of wide critical radius (a giant
// planet: every pair of its row passes, in FP64), whose rows take one chunk
// a task so that their terms spread over the GPU.  Culled chunks leave their
// slots unwritten; the member phase skips them by the same test.
__device__ void huge_pairs(const Dev& d, const Params& p, int M, int nch, int k0, int nact, int par, int nwide) {
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int ngrp = (nch + kHugeGroup - 1) / kHugeGroup;
    const int64_t perA = (int64_t)nwide * nch, perB = (int64_t)M * ngrp, per = perA + perB;
    for (int64_t w = gw; w < nact * per; w += nw) {
        const int k = k0 + (int)(w / per);
        const int64_t r = w % per;
        int b, ch0, ch1;
        if (r < perA) {
            b = d.hctl->wlist[r / nch];
            ch0 = (int)(r % nch);
            ch1 = ch0 + 1;
        } else {
            b = (int)((r - perA) / ngrp);
            if (H.wide[b]) continue;   // its row runs a chunk a task
            ch0 = (int)((r - perA) % ngrp) * kHugeGroup;
            ch1 = min(nch, ch0 + kHugeGroup);
        }
        if (!H.alive[b]) continue;   // its slots are never read
        const double* pos = huge_pos(H, k);
        const float4* posf = H.posf + (int64_t)k * c;
        const float4 pb = posf[b];
        const float4* bx = huge_cbox(H, par, k);
        // the task's chunks that can hold a pair (lane j tests chunk ch0 + j)
        unsigned live = __ballot_sync(0xffffffffu, lane < ch1 - ch0 && !chunk_culled(pb, bx[2 * (ch0 + lane)],
                                                                                     bx[2 * (ch0 + lane) + 1]));
        if (!live) continue;
        const double xb = pos[b], yb = pos[c + b], zb = pos[2 * c + b];
        const float slack = 1e-5f * (1.0f + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z));
        while (live) {
            const int ch = ch0 + __ffs(live) - 1;
            live &= live - 1;
            double ax = 0.0, ay = 0.0, az = 0.0;
            for (int u = 0; u < 2; u++) {
                const int io = ch * kHugeChunk + u * 32 + lane;
                if (io >= M) continue;
                const int o = H.perm[io];
                if (o == b || !H.alive[o]) continue;
                const float4 po = posf[o];
                const float dx = po.x - pb.x, dy = po.y - pb.y, dz = po.z - pb.z;
                const float lim = fmaxf(pb.w, po.w) + slack;
                if (dx * dx + dy * dy + dz * dz < lim * lim) huge_pair(d, p, pos, b, o, xb, yb, zb, ax, ay, az);
            }
#pragma unroll
            for (int s = 16; s >= 1; s >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, s);
                ay += __shfl_xor_sync(0xffffffffu, ay, s);
                az += __shfl_xor_sync(0xffffffffu, az, s);
            }
            if (lane == 0) {
                double* q = huge_part(H, k) + 3 * ((int64_t)b * nch + ch);
                q[0] = ax;
                q[1] = ay;
                q[2] = az;
            }
        }
    }
}

// sequence k's evaluation point of member b, in double and in float
__device__ __forceinline__ float4 huge_set_pos(const Dev& d, int k, int b, double x, double y, double z) {
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    double* pos = H.pos + (int64_t)k * 3 * c;
    pos[b] = x;
    pos[c + b] = y;
    pos[2 * c + b] = z;
    const float4 f = make_float4((float)x, (float)y, (float)z, __double2float_ru(H.rc[b]));
    H.posf[(int64_t)k * c + b] = f;
    return f;
}

// exact contact test of two members (the small-group kernels' comparison);
// two small bodies never touch
__device__ __forceinline__ bool huge_touch(const HugeBuf& H, int u, int w) {
    if (!bs_can_touch(H.m[u], H.m[w])) return false;
    const int64_t c = H.cap;
    const double dx = H.y[w] - H.y[u], dy = H.y[c + w] - H.y[c + u], dz = H.y[2 * c + w] - H.y[2 * c + u];
    return sqrt(dx * dx + dy * dy + dz * dz) <= H.R[u] + H.R[w];
}

// perfect merger of members u and w (as the small-group kernels merge)
__device__ void huge_merge(const Dev& d, const Params& p, double M0, int b, int q, double& El, int& survivor) {
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    const double G = p.G;
    const double mb = H.m[b], mq = H.m[q], M = mb + mq;
    double X[2][6];
    for (int k = 0; k < 6; k++) {
        X[0][k] = H.y[k * c + b];
        X[1][k] = H.y[k * c + q];
    }
    double dd[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
    double xn[3], vn[3];
    for (int k = 0; k < 3; k++) {
        xn[k] = (mb * X[0][k] + mq * X[1][k]) / M;
        vn[k] = (mb * X[0][3 + k] + mq * X[1][3 + k]) / M;
    }
    const double vb2 = X[0][3] * X[0][3] + X[0][4] * X[0][4] + X[0][5] * X[0][5];
    const double vq2 = X[1][3] * X[1][3] + X[1][4] * X[1][4] + X[1][5] * X[1][5];
    const double rb = sqrt(X[0][0] * X[0][0] + X[0][1] * X[0][1] + X[0][2] * X[0][2]);
    const double rq = sqrt(X[1][0] * X[1][0] + X[1][1] * X[1][1] + X[1][2] * X[1][2]);
    const double rbq = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
    const double e_before = 0.5 * mb * vb2 + 0.5 * mq * vq2 - G * M0 * mb / rb - G * M0 * mq / rq - G * mb * mq / rbq;
    const double vn2 = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
    const double rn = sqrt(xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2]);
    const double e_after = 0.5 * M * vn2 - G * M0 * M / rn;
    El += e_before - e_after;
    int keep, gone;
    if (mb > mq) keep = b, gone = q;
    else if (mq > mb) keep = q, gone = b;
    else keep = (H.gid[b] < H.gid[q]) ? b : q, gone = (keep == b) ? q : b;
    const double Rn = cbrt(H.R[b] * H.R[b] * H.R[b] + H.R[q] * H.R[q] * H.R[q]);
    for (int k = 0; k < 3; k++) {
        H.y[k * c + keep] = xn[k];
        H.y[(3 + k) * c + keep] = vn[k];
    }
    H.m[keep] = M;
    H.R[keep] = Rn;
    H.m[gone] = 0.0;
    H.alive[gone] = 0;
    survivor = keep;
}

// lexicographic order of member pairs (the sequential sweep's order)
__device__ __forceinline__ bool pair_before(int2 a, int2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }

__global__ void __launch_bounds__(kHugeThreads, 2) k_bs_huge(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlBsHuge);
    __shared__ double red[kHugeThreads / 32];
    __shared__ int bred[7][kHugeThreads / 32];
    HugeCtl* hc = d.hctl;
    const int nh = d.ctl->nhuge;
    if (nh == 0) return;   // fixed before the launch: the same in every block
    const unsigned long long wait_ns = (unsigned long long)d.huge_wait_ns;
    const int hold = d.huge_hold;
    auto huge_sync = [&](HugeCtl* h) { return opal::huge_sync(h, wait_ns, hold); };
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // status set before this kernel: block 0 looks, everyone follows
    if (lead) hc->skip = d.ctl->status;
    if (!huge_sync(hc)) {
        if (lead) set_status(d.ctl, kEbs, kHugeAbortDetail);   // no group started: a barrier wait ran out
        return;
    }
    if (*(volatile int*)&hc->skip) return;
    const Params p = d.p;
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    const double dt = p.dt, tol2 = p.bs_tol * p.bs_tol;
    const int cap = p.bs_max_substeps;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int hi = 0; hi < nh; hi++) {
        const int g = d.ghuge[hi];
        const int m0 = d.goff[g], M = d.goff[g + 1] - m0;
        const int nch = (M + kHugeChunk - 1) / kHugeChunk;
        const double M0g = d.M0s[d.body_sys[d.members[m0]]], GM0 = p.G * M0g;   // the group's star
        for (int64_t b = gt; b < M; b += nt) {
            const int gb = d.members[m0 + b];
            H.gid[b] = gb;
            H.y[b] = d.x0[gb];
            H.y[c + b] = d.y0[gb];
            H.y[2 * c + b] = d.z0[gb];
            H.y[3 * c + b] = d.vx0[gb];
            H.y[4 * c + b] = d.vy0[gb];
            H.y[5 * c + b] = d.vz0[gb];
            H.m[b] = d.m[gb];
            H.R[b] = d.R[gb];
            H.rc[b] = d.rc[gb];
            H.pinv[b] = 1.0 / (0.9 * d.rc[gb]);
            H.alive[b] = d.alive[gb];
        }
        const int Mp = nch * kHugeChunk;   // member slots rounded up to whole chunks
        if (lead) {
            hc->El = 0.0;
            hc->nmerge = 0;
            hc->bb[0] = hc->bb[2] = 0x7fffffff;
            hc->bb[1] = hc->bb[3] = (int)0x80000000;
            hc->rcmm[0] = 0;
            hc->rcmm[1] = 0x7fffffff;
            hc->nwide = 0;
        }
        // The members in spatial order, once a step: a 2D Morton key of each
        // start position over the group's box, ranked (ties by slot), so that
        // a chunk of 64 consecutive members of the order is compact and its
        // box culls the pairs it cannot hold.
        bool ok = huge_sync(hc);
        if (ok) {
            int lx = 0x7fffffff, hx = (int)0x80000000, ly = 0x7fffffff, hy = (int)0x80000000;
            int rmax = 0, rmin = 0x7fffffff;
            for (int64_t b = gt; b < M; b += nt) {
                const int fx = ford((float)H.y[b]), fy = ford((float)H.y[c + b]);
                lx = min(lx, fx);
                hx = max(hx, fx);
                ly = min(ly, fy);
                hy = max(hy, fy);
                if (H.alive[b]) {
                    const int rb = __float_as_int(__double2float_ru(H.rc[b]));   // rc >= 0: bits order as values
                    rmax = max(rmax, rb);
                    rmin = min(rmin, rb);
                }
            }
            lx = __reduce_min_sync(0xffffffffu, lx);
            hx = __reduce_max_sync(0xffffffffu, hx);
            ly = __reduce_min_sync(0xffffffffu, ly);
            hy = __reduce_max_sync(0xffffffffu, hy);
            rmax = __reduce_max_sync(0xffffffffu, rmax);
            rmin = __reduce_min_sync(0xffffffffu, rmin);
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&hc->bb[0], lx);
                atomicMax(&hc->bb[1], hx);
                atomicMin(&hc->bb[2], ly);
                atomicMax(&hc->bb[3], hy);
                atomicMax(&hc->rcmm[0], rmax);
                atomicMin(&hc->rcmm[1], rmin);
            }
            ok = huge_sync(hc);
        }
        if (ok) {
            const float x0 = fordinv(*(volatile int*)&hc->bb[0]), x1 = fordinv(*(volatile int*)&hc->bb[1]);
            const float y0 = fordinv(*(volatile int*)&hc->bb[2]), y1 = fordinv(*(volatile int*)&hc->bb[3]);
            const float sx = 65535.0f / fmaxf(x1 - x0, 1e-30f), sy = 65535.0f / fmaxf(y1 - y0, 1e-30f);
            // wide members: rc above a quarter of the largest, when that is over 8 times the smallest
            const float rmx = __int_as_float(*(volatile int*)&hc->rcmm[0]);
            const float rmn = __int_as_float(*(volatile int*)&hc->rcmm[1]);
            const bool any_wide = rmx > 8.0f * rmn;
            for (int64_t b = gt; b < M; b += nt) {
                const unsigned qx = (unsigned)fminf(65535.0f, fmaxf(0.0f, ((float)H.y[b] - x0) * sx));
                const unsigned qy = (unsigned)fminf(65535.0f, fmaxf(0.0f, ((float)H.y[c + b] - y0) * sy));
                H.key[b] = spread16(qx) | (spread16(qy) << 1);
                int wb = 0;
                if (any_wide && H.alive[b] && __double2float_ru(H.rc[b]) > 0.25f * rmx) {
                    const int q = atomicAdd(&hc->nwide, 1);
                    if (q < kHugeWide) {
                        hc->wlist[q] = (int)b;
                        wb = 1;
                    }
                }
                H.wide[b] = wb;
            }
            ok = huge_sync(hc);
        }
        if (ok) {
            for (int64_t b = gt; b < M; b += nt) {
                const unsigned kb = H.key[b];
                int rank = 0;
                for (int o = 0; o < M; o++) {
                    const unsigned ko = H.key[o];
                    rank += (ko < kb || (ko == kb && o < (int)b)) ? 1 : 0;
                }
                H.perm[rank] = (int)b;
            }
            ok = huge_sync(hc);   // the order is complete before anyone reads it
        }
        if (!ok) {
            if (lead) set_status(d.ctl, kEbs, kHugeAbortDetail + 1 + g);
            return;
        }
        const int nwide = min(*(volatile int*)&hc->nwide, kHugeWide);
        double t = 0.0, Hs = dt;
        int nsub = 0;
        bool failed = false;
        for (;;) {
            const double rem = dt - t;
            int last = 0;
            if (fabs(Hs) >= fabs(rem)) {
                Hs = rem;
                last = 1;
            }
            int kacc = -1;
            // The sequences advance in lockstep: round r evaluates the derivative
            // at the r-th point of every sequence k with n_k = 2 (k + 1) >= r
            // (round 0 at the substep's start, shared by all of them).  Sequence
            // k ends at round n_k with its tableau row, and row k >= 1 is tested
            // then: rows are tested in the sequential order, and the first that
            // passes is the one the sequential method takes, from the same
            // arithmetic.  Two grid barriers a round.  Members are visited in
            // spatial order in whole chunks (block-aligned), so that each chunk's
            // box of the next evaluation points is reduced where they are set.
            for (int64_t base = (int64_t)blockIdx.x * kHugeThreads; base < Mp; base += nt) {
                const int i = (int)(base + threadIdx.x);
                const bool mem = i < M;
                const int b = mem ? H.perm[i] : 0;
                float4 pf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (mem) pf = huge_set_pos(d, 0, b, H.y[b], H.y[c + b], H.y[2 * c + b]);
                chunk_box_store(mem && H.alive[b], pf,
                                ((i & 63) == 0 && i < Mp) ? huge_cbox(H, 0, 0) + 2 * (i >> 6) : nullptr, bred);
            }
            if (!(ok = huge_sync(hc))) break;
            for (int r = 0; r <= 2 * kBsRows && ok; r++) {
                const int k0 = r == 0 ? 0 : max(0, (r + 1) / 2 - 1);
                const int nact = r == 0 ? 1 : kBsRows - k0;
                const int kf = (r >= 2 && r % 2 == 0) ? r / 2 - 1 : -1;   // the sequence that ends this round
                huge_pairs(d, p, M, nch, k0, nact, r & 1, nwide);
                if (!(ok = huge_sync(hc))) break;
                double emax = 0.0;
                for (int64_t base = (int64_t)blockIdx.x * kHugeThreads; base < (int64_t)nact * Mp; base += nt) {
                    const int64_t idx = base + threadIdx.x;
                    const bool act = idx < (int64_t)nact * Mp;
                    const int k = k0 + (act ? (int)(idx / Mp) : 0);
                    const int i = act ? (int)(idx % Mp) : 0;
                    const bool mem = act && i < M;
                    const int b = mem ? H.perm[i] : 0;
                    const int n = 2 * (k + 1);
                    const double h = Hs / n;
                    double* z0 = H.z0 + (int64_t)k * 6 * c;
                    double* z1 = H.z1 + (int64_t)k * 6 * c;
                    // the next evaluation point of this member (sequence k), for the chunk box
                    bool moved = false;
                    float4 pf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    double f[6] = {0, 0, 0, 0, 0, 0};
                    if (mem) {
                        // evaluation point of this round: the substep's start or z1
                        const double* base_pt = r == 0 ? H.y : z1;
                        const double P0 = base_pt[b], P1 = base_pt[c + b], P2 = base_pt[2 * c + b];
                        if (H.alive[b]) {
                            f[0] = base_pt[3 * c + b];
                            f[1] = base_pt[4 * c + b];
                            f[2] = base_pt[5 * c + b];
                            const double r2 = P0 * P0 + P1 * P1 + P2 * P2, ri = rsqrt(r2);
                            const double sk = -GM0 * (ri * ri * ri);
                            double ax = sk * P0, ay = sk * P1, az = sk * P2;
                            // the chunk slots the pair phase wrote: the same culling decision
                            const double* q = huge_part(H, k) + 3 * (int64_t)b * nch;
                            const float4 pb = H.posf[(int64_t)k * c + b];
                            const float4* bx = huge_cbox(H, r & 1, k);
                            for (int ch = 0; ch < nch; ch++) {
                                if (chunk_culled(pb, bx[2 * ch], bx[2 * ch + 1])) continue;
                                ax += q[3 * ch];
                                ay += q[3 * ch + 1];
                                az += q[3 * ch + 2];
                            }
                            f[3] = ax;
                            f[4] = ay;
                            f[5] = az;
                        }
                        if (r == 0) {
                            // the first step of every sequence from the shared derivative
                            for (int kk = 0; kk < kBsRows; kk++) {
                                const double hk = Hs / (2 * (kk + 1));
                                double* a0 = H.z0 + (int64_t)kk * 6 * c;
                                double* a1 = H.z1 + (int64_t)kk * 6 * c;
                                for (int q = 0; q < 6; q++) {
                                    a0[q * c + b] = H.y[q * c + b];
                                    a1[q * c + b] = H.y[q * c + b] + hk * f[q];
                                }
                            }
                        } else if (r < n) {
                            for (int q = 0; q < 6; q++) {
                                const double znew = z0[q * c + b] + 2.0 * h * f[q];
                                z0[q * c + b] = z1[q * c + b];
                                z1[q * c + b] = znew;
                            }
                            pf = huge_set_pos(d, k, b, z1[b], z1[c + b], z1[2 * c + b]);
                            moved = true;
                        } else {
                            // row k of the tableau (in place; sequences end in order) and this member's error
                            double dsq_x = 0.0, dsq_v = 0.0, nx = 0.0, nv = 0.0;
                            for (int q = 0; q < 6; q++) {
                                double cv = 0.5 * (z1[q * c + b] + z0[q * c + b] + h * f[q]), pv = 0.0;
                                for (int j = 1; j <= k; j++) {
                                    double* slot = H.row + ((int64_t)(j - 1) * 6 + q) * c + b;
                                    const double up = *slot;
                                    *slot = cv;
                                    pv = cv;
                                    cv = cv + (cv - up) * kNeville[k][j];
                                }
                                H.row[((int64_t)k * 6 + q) * c + b] = cv;
                                const double df = cv - pv;
                                if (q < 3) {
                                    dsq_x += df * df;
                                    nx += cv * cv;
                                } else {
                                    dsq_v += df * df;
                                    nv += cv * cv;
                                }
                            }
                            if (k >= 1 && H.alive[b]) {
                                // |dX|^2 <= tol^2 |X|^2 and the same for V; a NaN fails it
                                const double e2 =
                                    (dsq_x <= tol2 * fmax(nx, 2.3e-308) && dsq_v <= tol2 * fmax(nv, 2.3e-308))
                                        ? 0.0
                                        : HUGE_VAL;
                                emax = fmax(emax, e2);
                            }
                        }
                    }
                    // the next round's chunk boxes (parity of round r + 1)
                    if (r == 0) {
                        for (int kk = 0; kk < kBsRows; kk++) {
                            float4 pk = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            if (mem) {
                                const double* a1 = H.z1 + (int64_t)kk * 6 * c;
                                pk = huge_set_pos(d, kk, b, a1[b], a1[c + b], a1[2 * c + b]);
                            }
                            chunk_box_store(mem && H.alive[b], pk,
                                            (act && (i & 63) == 0) ? huge_cbox(H, 1, kk) + 2 * (i >> 6) : nullptr,
                                            bred);
                        }
                    } else {
                        const bool cont = act && r < n;   // the same for the 64 threads of a chunk
                        chunk_box_store(moved && H.alive[b], pf,
                                        (cont && (i & 63) == 0) ? huge_cbox(H, (r + 1) & 1, k) + 2 * (i >> 6) : nullptr,
                                        bred);
                    }
                }
                if (kf >= 0) {
                    // grid-wide maximum of the ending sequence's errors (non-negative:
                    // their bits order as they do)
                    for (int o = 16; o >= 1; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
                    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        double m = 0.0;
                        for (int w = 0; w < kHugeThreads / 32; w++) m = fmax(m, red[w]);
                        atomicMax(&hc->err[kf], (unsigned long long)__double_as_longlong(m));
                    }
                }
                if (!(ok = huge_sync(hc))) break;
                if (kf >= 1) {
                    const double e = __longlong_as_double((long long)*(volatile unsigned long long*)&hc->err[kf]);
                    if (e <= tol2) {
                        kacc = kf;
                        break;
                    }
                }
            }
            if (ok && kacc < 0) {
                // rejected: everyone has read the last row's maximum before the rows are cleared
                ok = huge_sync(hc);
                if (lead)
                    for (int k = 0; k < kBsRows; k++) hc->err[k] = 0ull;
            }
            if (!ok) break;
            nsub++;
            if (kacc >= 0) {
                for (int64_t b = gt; b < M; b += nt)
                    for (int q = 0; q < 6; q++) H.y[q * c + b] = H.row[((int64_t)kacc * 6 + q) * c + b];
                t = last ? dt : t + Hs;
                // contacts: candidates in parallel, then the sequential sweep by one thread
                if (lead) hc->ncand = 0;
                if (!(ok = huge_sync(hc))) break;
                // every block has read the accepted row's maximum: clear the rows' maxima
                if (lead)
                    for (int k = 0; k < kBsRows; k++) hc->err[k] = 0ull;
                for (int64_t w = gt; w < (int64_t)M * nch; w += nt) {
                    const int u = (int)(w / nch), ch = (int)(w % nch);
                    if (!H.alive[u]) continue;
                    for (int o = ch * kHugeChunk; o < min(M, (ch + 1) * kHugeChunk); o++) {
                        if (o <= u || !H.alive[o] || !bs_can_touch(H.m[u], H.m[o])) continue;
                        const double dx = H.y[o] - H.y[u], dy = H.y[c + o] - H.y[c + u], dz = H.y[2 * c + o] - H.y[2 * c + u];
                        const double rs = H.R[u] + H.R[o];
                        if (dx * dx + dy * dy + dz * dz <= rs * rs * (1.0 + 1e-9)) {
                            const int i = atomicAdd(&hc->ncand, 1);
                            if (i < kHugeCand) hc->cand[i] = make_int2(u, o);
                        }
                    }
                }
                if (!(ok = huge_sync(hc))) break;
                if (lead && hc->ncand > 0) {
                    int nc = min(hc->ncand, kHugeCand);
                    if (hc->ncand > kHugeCand) set_status(d.ctl, kEoverflow, -8);
                    // sort, then sweep in order; a merger moves its survivor, whose new
                    // contacts later in the order join the list
                    for (int i = 1; i < nc; i++) {
                        const int2 x = hc->cand[i];
                        int j = i - 1;
                        while (j >= 0 && pair_before(x, hc->cand[j])) {
                            hc->cand[j + 1] = hc->cand[j];
                            j--;
                        }
                        hc->cand[j + 1] = x;
                    }
                    for (int i = 0; i < nc; i++) {
                        const int2 pr = hc->cand[i];
                        if (!H.alive[pr.x] || !H.alive[pr.y] || !huge_touch(H, pr.x, pr.y)) continue;
                        double El = hc->El;
                        int sv = -1;
                        huge_merge(d, p, M0g, pr.x, pr.y, El, sv);
                        hc->El = El;
                        hc->nmerge++;
                        for (int x = 0; x < M; x++) {
                            if (x == sv || !H.alive[x] || !huge_touch(H, sv, x)) continue;
                            const int2 np = make_int2(min(sv, x), max(sv, x));
                            if (!pair_before(pr, np)) continue;   // the sweep is past that pair
                            bool have = false;
                            for (int j = i + 1; j < nc; j++)
                                if (hc->cand[j].x == np.x && hc->cand[j].y == np.y) have = true;
                            if (have) continue;
                            if (nc >= kHugeCand) {
                                set_status(d.ctl, kEoverflow, -8);
                                break;
                            }
                            int j = nc++;
                            while (j > i + 1 && pair_before(np, hc->cand[j - 1])) {
                                hc->cand[j] = hc->cand[j - 1];
                                j--;
                            }
                            hc->cand[j] = np;
                        }
                    }
                }
                if (!(ok = huge_sync(hc))) break;
                if (last) break;
                if (kacc <= 2) Hs *= 2.0;
                else if (kacc >= 6) Hs *= 0.5;
            } else {
                Hs *= 0.5;
            }
            if (nsub >= cap) {
                failed = true;
                break;
            }
        }
        if (!ok) {
            if (lead) set_status(d.ctl, kEbs, kHugeAbortDetail + 1 + g);
            return;
        }
        for (int64_t b = gt; b < M; b += nt) {
            double* o = d.bsout + (int64_t)kBsOut * (m0 + b);
            for (int q = 0; q < 6; q++) o[q] = H.y[q * c + b];
            o[6] = H.m[b];
            o[7] = H.R[b];
            o[8] = (double)H.alive[b];
        }
        if (lead) {
            d.glost[g] = hc->El;
            if (hc->nmerge) atomicAdd(&d.ctl->nmerge, hc->nmerge);
            atomicAdd(&d.ctl->nsub, (unsigned long long)nsub);
            if (failed) set_status(d.ctl, kEbs, g);
        }
        if (!huge_sync(hc)) return;   // the buffers are free for the next group
    }
}

cudaError_t launch_bs_huge(const Dev& d, int nsm, cudaStream_t s) {
    // all blocks must be resident at once for the barriers: a cooperative launch
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nsm);
    cfg.blockDim = dim3(kHugeThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_bs_huge, d);
    prof_mark("bs: groups of more than 64");
    return e;
}

}  // namespace opal
