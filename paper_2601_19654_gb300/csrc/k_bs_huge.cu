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
                __nanosleep(200);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int*)&hc->abort == 0;
}

// (1 - K) term of member b against o (as the small-group kernels compute it)
__device__ __forceinline__ void huge_pair(const Dev& d, const Params& p, int b, int o, double xb, double yb,
                                          double zb, double& ax, double& ay, double& az) {
    const HugeBuf& H = d.hb;
    if (le_zero(H.m[o])) return;   // a small body (m = 0): no source
    const int w = gt_nonneg(H.rc[b], H.rc[o]) ? b : o;
    const double rc = H.rc[w];
    const int64_t c = H.cap;
    const double dx = H.pos[o] - xb, dy = H.pos[c + o] - yb, dz = H.pos[2 * c + o] - zb;
    const double dr2 = dx * dx + dy * dy + dz * dz;
    if (ge_nonneg(dr2, rc * rc)) return;   // 1 - K = 0 at or beyond rc
    const double dri = rsqrt(dr2), dr = dr2 * dri;
    if (ge_nonneg(dr, rc)) return;
    double K;
    const double y = (dr - 0.1 * rc) * H.pinv[w];
    if (le_zero(y)) K = 0.0;
    else if (p.changeover == 0) K = y * y / (2.0 * y * y - 2.0 * y + 1.0);
    else K = y * y * y * (10.0 - 15.0 * y + 6.0 * y * y);
    const double wgt = 1.0 - K;
    const double t = p.G * H.m[o] * wgt * (dri * dri * dri);
    ax += t * dx;
    ay += t * dy;
    az += t * dz;
}

// pair phase: every (member, chunk) slot from the positions in H.pos / H.posf
__device__ void huge_pairs(const Dev& d, const Params& p, int M, int nch) {
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = gw; w < (int64_t)M * nch; w += nw) {
        const int b = (int)(w / nch), ch = (int)(w % nch);
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (H.alive[b]) {
            const double xb = H.pos[b], yb = H.pos[c + b], zb = H.pos[2 * c + b];
            const float4 pb = H.posf[b];
            const float slack = 1e-5f * (1.0f + fabsf(pb.x) + fabsf(pb.y) + fabsf(pb.z));
            for (int u = 0; u < 2; u++) {
                const int o = ch * kHugeChunk + u * 32 + lane;
                if (o >= M || o == b || !H.alive[o]) continue;
                const float4 po = H.posf[o];
                const float dx = po.x - pb.x, dy = po.y - pb.y, dz = po.z - pb.z;
                const float lim = fmaxf(pb.w, po.w) + slack;
                if (dx * dx + dy * dy + dz * dz < lim * lim) huge_pair(d, p, b, o, xb, yb, zb, ax, ay, az);
            }
        }
#pragma unroll
        for (int s = 16; s >= 1; s >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, s);
            ay += __shfl_xor_sync(0xffffffffu, ay, s);
            az += __shfl_xor_sync(0xffffffffu, az, s);
        }
        if (lane == 0) {
            double* q = H.part + 3 * (int64_t)w;
            q[0] = ax;
            q[1] = ay;
            q[2] = az;
        }
    }
}

__device__ __forceinline__ void huge_set_pos(const Dev& d, int b, double x, double y, double z) {
    const HugeBuf& H = d.hb;
    const int64_t c = H.cap;
    H.pos[b] = x;
    H.pos[c + b] = y;
    H.pos[2 * c + b] = z;
    H.posf[b] = make_float4((float)x, (float)y, (float)z, __double2float_ru(H.rc[b]));
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

__global__ void __launch_bounds__(kHugeThreads) k_bs_huge(Dev d) {
    __shared__ double red[kHugeThreads / 32];
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
        if (lead) {
            hc->El = 0.0;
            hc->nmerge = 0;
        }
        double t = 0.0, Hs = dt;
        int nsub = 0;
        bool ok = true, failed = false;
        for (;;) {
            const double rem = dt - t;
            int last = 0;
            if (fabs(Hs) >= fabs(rem)) {
                Hs = rem;
                last = 1;
            }
            int kacc = -1;
            for (int k = 0; k < kBsRows && ok; k++) {
                const int n = 2 * (k + 1);
                const double h = Hs / n;
                for (int64_t b = gt; b < M; b += nt) huge_set_pos(d, (int)b, H.y[b], H.y[c + b], H.y[2 * c + b]);
                if (!(ok = huge_sync(hc))) break;
                for (int s = 0; s <= n && ok; s++) {
                    huge_pairs(d, p, M, nch);
                    if (!(ok = huge_sync(hc))) break;
                    double emax = 0.0;
                    for (int64_t b = gt; b < M; b += nt) {
                        // evaluation point of this pass: the substep's start or z1
                        const double* base = s == 0 ? H.y : H.z1;
                        const double P0 = base[b], P1 = base[c + b], P2 = base[2 * c + b];
                        double f[6] = {0, 0, 0, 0, 0, 0};
                        if (H.alive[b]) {
                            f[0] = base[3 * c + b];
                            f[1] = base[4 * c + b];
                            f[2] = base[5 * c + b];
                            const double r2 = P0 * P0 + P1 * P1 + P2 * P2, ri = rsqrt(r2);
                            const double sk = -GM0 * (ri * ri * ri);
                            double ax = sk * P0, ay = sk * P1, az = sk * P2;
                            const double* q = H.part + 3 * (int64_t)b * nch;
                            for (int ch = 0; ch < nch; ch++) {
                                ax += q[3 * ch];
                                ay += q[3 * ch + 1];
                                az += q[3 * ch + 2];
                            }
                            f[3] = ax;
                            f[4] = ay;
                            f[5] = az;
                        }
                        if (s == 0) {
                            for (int q = 0; q < 6; q++) {
                                H.z0[q * c + b] = H.y[q * c + b];
                                H.z1[q * c + b] = H.y[q * c + b] + h * f[q];
                            }
                        } else if (s < n) {
                            for (int q = 0; q < 6; q++) {
                                const double znew = H.z0[q * c + b] + 2.0 * h * f[q];
                                H.z0[q * c + b] = H.z1[q * c + b];
                                H.z1[q * c + b] = znew;
                            }
                        } else {
                            // row k of the tableau (in place) and this member's error
                            double dsq_x = 0.0, dsq_v = 0.0, nx = 0.0, nv = 0.0;
                            for (int q = 0; q < 6; q++) {
                                double cv = 0.5 * (H.z1[q * c + b] + H.z0[q * c + b] + h * f[q]), pv = 0.0;
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
                                    (dsq_x <= tol2 * fmax(nx, 2.3e-308) && dsq_v <= tol2 * fmax(nv, 2.3e-308)) ? 0.0
                                                                                                             : HUGE_VAL;
                                emax = fmax(emax, e2);
                            }
                        }
                        if (s < n) huge_set_pos(d, (int)b, H.z1[b], H.z1[c + b], H.z1[2 * c + b]);
                    }
                    if (s == n) {
                        // grid-wide maximum of the errors (non-negative: their bits order as they do)
                        for (int o = 16; o >= 1; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
                        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
                        __syncthreads();
                        if (threadIdx.x == 0) {
                            double m = 0.0;
                            for (int w = 0; w < kHugeThreads / 32; w++) m = fmax(m, red[w]);
                            atomicMax(&hc->err[k], (unsigned long long)__double_as_longlong(m));
                        }
                    }
                    if (!(ok = huge_sync(hc))) break;
                }
                if (!ok) break;
                const double e = __longlong_as_double((long long)*(volatile unsigned long long*)&hc->err[k]);
                if (!(ok = huge_sync(hc))) break;   // everyone has read the maximum
                if (lead) hc->err[k] = 0ull;
                if (k >= 1 && e <= tol2) {
                    kacc = k;
                    break;
                }
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
