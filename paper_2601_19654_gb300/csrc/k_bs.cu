// Bulirsch-Stoer integration of each encounter group over the step, with
// perfect-merger collisions (Sec. 2.1.1 footnote 2: the bodies in a close
// encounter have their interaction and Keplerian Hamiltonians advanced by BS;
// Sec. 3.2 listing: they restart from the saved x0, v0; mce_coll, Sec. 2.1.2).
//
// Equations of a group, democratic heliocentric variables:
//   dx_b/dt = V_b,
//   dV_b/dt = -G M0 x_b/|x_b|^3 + sum_{c in group} G m_c (1 - K(r_bc; rc_bc)) (x_c - x_b)/r_bc^3.
// A substep of length H: modified midpoint with n_k = 2, 4, ..., 16 steps and
// Neville extrapolation in h^2; row k (k >= 1) is accepted when
//   max_b max(|dX_b|/|X_b|, |dV_b|/|V_b|) <= bs_tol,  d = T[k][k] - T[k][k-1].
// Step control as the oracle's: first substep = the whole step; accepted at
// k <= 2 -> double, at k >= 6 -> halve; not accepted by k = 7 -> retry at
// half length; the substep count is capped.
//
// Layout: one thread per (sequence k, member b); all eight midpoint
// sequences advance in lockstep, one derivative evaluation per round.
// Sequence k finishes at round n_k = 2k + 2, its thread extrapolates row k
// for its member at once (row k - 1 is two rounds old), and the group stops
// at the first row that passes the test, as the sequential method does.  On
// this chip a warp instruction costs the FP64 pipe the same whatever the
// number of active lanes, so the rounds of a group cost what one sequence
// would, and groups of up to 4 members fit one warp.  Four such warps (on
// the four schedulers of an SM) try the step sizes H, H/2, H/4, H/8 at once:
// the first one accepted in that order is the one the sequential method
// would reach after its rejections, so only the cost of rejections changes.
#include <cooperative_groups.h>

#include "opal_internal.cuh"

namespace opal {

namespace cg = cooperative_groups;

// Few groups (kBsManyGroups or fewer in a step): the lockstep kernels (one
// block per group, all sequences and four step sizes at once) give each group
// the shortest chain of dependent operations.  Many groups: the packed kernel
// (one lane per member, many groups per warp) makes each group's first
// attempt, the whole step, which settles most of them; the groups it rejects
// go on to the lockstep kernels, which start them again from the beginning.

// NT threads hold A attempts (step sizes H, H/2, ..., H/2^(A-1)) of one group
// of up to M members, one thread per (attempt, sequence, member).
template <int NT, int A>
struct BsSh {
    static constexpr int M = NT / (A * kBsRows);
    double y[6][M];                     // current state, component-major: X, Y, Z, VX, VY, VZ
    double pos[A][kBsRows][3][M];       // positions of each sequence's evaluation in progress
    double row[A][kBsRows][6][M];       // the last extrapolated row of each member
    double diag[A][kBsRows][6][M];      // T[k][k] of every finished row (the accepted one is kept)
    double raw[A][6][M];                // midpoint result of the sequence finishing this round
    double df2[A][6][M], cur2[A][6][M]; // per component: squared change and squared value
    int ok[A][kBsRows][M];              // each member passes the acceptance test, per finished row
    double m[M], R[M], rc[M];
    // per member: rc^2, 1 / (0.9 rc) and 0.1 rc (a pair uses the member with the larger rc)
    double prc2[M], pinv[M], pc01[M];
    int alive[M], gid[M];
    int big[M];                         // a big body (a source of force), not a small one
    int kacc[A];                        // accepted row of each attempt, -1 while none
    int gi, kq[4];                      // cluster form: the group taken, every attempt's accepted row
    int decision, collide, nmerge;      // (cluster form: decision holds the substep attempt 0 accepted)
    int dec;                            // cluster form: the attempt taken after a substep
    double El;
};

// Perfect merger of members b and q of a group held in S (y[6][.], m, R, gid,
// alive), M0 the star's mass: mass, momentum and centre of mass kept, R = cbrt(R_b^3 + R_q^3),
// the heavier body (lower id on a tie) survives; El gets the energy removed.
template <class SH>
__device__ void bs_merge(SH& S, const Params& p, double M0, int b, int q, double& El, int& nmerge) {
    const double G = p.G;
    double mb = S.m[b], mq = S.m[q], M = mb + mq;
    double d[3] = {S.y[0][q] - S.y[0][b], S.y[1][q] - S.y[1][b], S.y[2][q] - S.y[2][b]};
    double xn[3], vn[3];
    for (int k = 0; k < 3; k++) {
        xn[k] = (mb * S.y[k][b] + mq * S.y[k][q]) / M;
        vn[k] = (mb * S.y[3 + k][b] + mq * S.y[3 + k][q]) / M;
    }
    double vb2 = S.y[3][b] * S.y[3][b] + S.y[4][b] * S.y[4][b] + S.y[5][b] * S.y[5][b];
    double vq2 = S.y[3][q] * S.y[3][q] + S.y[4][q] * S.y[4][q] + S.y[5][q] * S.y[5][q];
    double rb = sqrt(S.y[0][b] * S.y[0][b] + S.y[1][b] * S.y[1][b] + S.y[2][b] * S.y[2][b]);
    double rq = sqrt(S.y[0][q] * S.y[0][q] + S.y[1][q] * S.y[1][q] + S.y[2][q] * S.y[2][q]);
    double rbq = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double e_before = 0.5 * mb * vb2 + 0.5 * mq * vq2 - G * M0 * mb / rb - G * M0 * mq / rq - G * mb * mq / rbq;
    double vn2 = vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2];
    double rn = sqrt(xn[0] * xn[0] + xn[1] * xn[1] + xn[2] * xn[2]);
    double e_after = 0.5 * M * vn2 - G * M0 * M / rn;
    El += e_before - e_after;
    int keep, gone;
    if (mb > mq) keep = b, gone = q;
    else if (mq > mb) keep = q, gone = b;
    else keep = (S.gid[b] < S.gid[q]) ? b : q, gone = (keep == b) ? q : b;
    double Rn = cbrt(S.R[b] * S.R[b] * S.R[b] + S.R[q] * S.R[q] * S.R[q]);
    for (int k = 0; k < 3; k++) {
        S.y[k][keep] = xn[k];
        S.y[3 + k][keep] = vn[k];
    }
    S.m[keep] = M;
    S.R[keep] = Rn;
    S.m[gone] = 0.0;
    S.alive[gone] = 0;
    nmerge++;
}

// (1 - K) weighted attraction of a member at (xb, yb, zb) towards one at
// (xo, yo, zo) of mass mo, added to (ax, ay, az).  rc, rc2, c01, inv belong to
// the member with the larger rc (rc_bo = max(rc_b, rc_o)): rc, rc^2, 0.1 rc and
// 1 / (0.9 rc), so K needs no division by rc.  Callers pass big members only:
// a small body pulls nothing (Sec. 2.1: only big bodies are gravity sources).

__device__ __forceinline__ void bs_pair(const Params& p, double xb, double yb, double zb, double xo, double yo,
                                        double zo, double mo, double rc, double rc2, double c01, double inv,
                                        double& ax, double& ay, double& az) {
    const double dx = xo - xb, dy = yo - yb, dz = zo - zb;
    const double dr2 = dx * dx + dy * dy + dz * dz;
    if (ge_nonneg(dr2, rc2)) return;   // 1 - K = 0 at or beyond rc
    const double dri = rsqrt(dr2), dr = dr2 * dri;
    if (ge_nonneg(dr, rc)) return;
    const double t = mutual_factor(p.G * mo * (dri * dri * dri), (dr - c01) * inv, p.changeover);
    ax += t * dx;
    ay += t * dy;
    az += t * dz;
}

// acceleration of member b of sequence k at its position (x, y, z): the part
// of lane si of the sp lanes that share (k, b) -- the stellar term (si = 0)
// and the mutual terms of every sp-th other member from the si-th; the
// caller sums the sp parts
template <int NT, int A>
__device__ __forceinline__ void bs_accel(const BsSh<NT, A>& S, const Params& p, double GM0, int nm, int a, int k,
                                         int b, int si, int sp, double xb, double yb, double zb, double& ax,
                                         double& ay, double& az) {
    double r2 = xb * xb + yb * yb + zb * zb, ri = rsqrt(r2);
    double s = si == 0 ? -GM0 * (ri * ri * ri) : 0.0;
    ax = s * xb;
    ay = s * yb;
    az = s * zb;
    // the j-th other member in ascending order (the oracle's order when sp = 1):
    // every lane has the same number of them, so the lanes run each pass
    // together (a loop over all o that skips o == b would run the FP64 pair
    // code once per member, each time with a different lane idle)
    for (int j = si; j < nm - 1; j += sp) {
        const int o = j + (j >= b ? 1 : 0);
        if (!S.alive[o] || !S.big[o]) continue;   // (integer tests: no FP64 work)
        const int w = gt_nonneg(S.rc[b], S.rc[o]) ? b : o;   // rc_bo = max(rc_b, rc_o)
        bs_pair(p, xb, yb, zb, S.pos[a][k][0][o], S.pos[a][k][1][o], S.pos[a][k][2][o], S.m[o], S.rc[w],
                S.prc2[w], S.pc01[w], S.pinv[w], ax, ay, az);
    }
}

// CA > 1 (the cluster form): the CA attempts of a group are the CA blocks of
// a thread-block cluster, one attempt each on its own SM, so one group's
// rounds do not share an SM's FP64 pipe; the blocks exchange the decisions
// and the accepted state through distributed shared memory.  Every block of
// a cluster takes the same path (the same values decide it), so the cluster
// barriers are always met.
template <int NT, int A, int CA>
__global__ void __launch_bounds__(NT, NT == 32 ? 4 : 512 / NT) k_bs(Dev d, int kind) {
    OPAL_TIMELINE_SCOPE((NT == 256 ? kTlBs256 : kTlBs512));
    using Sh = BsSh<NT, A>;
    constexpr int M = Sh::M;
    constexpr int TA = NT / A;            // threads per attempt
    extern __shared__ __align__(16) unsigned char bs_smem[];   // one Sh (dynamic: above the static limit)
    Sh& S = *reinterpret_cast<Sh*>(bs_smem);
    const int arank = CA > 1 ? (int)cg::this_cluster().block_rank() : 0;   // this block's attempt
    if (CA == 1 && d.ctl->status) return;   // (the cluster form reads nothing another kernel may change)
    const Params p = d.p;
    // kind 0: groups of up to 4 members, 1: 5-32, 2: 33-64.  The groups it looks
    // at: few groups: all (kind 0) or the list of those above 4 members; many
    // groups: the list the packed kernel left.  (Four attempts pay for groups of
    // up to 4 members; for larger ones they only add FP64 work to the SM.)
    const bool small = kind == 0;
    const int lo = kind == 0 ? 1 : (kind == 1 ? 5 : 33);
    const bool many = d.ctl->ngroups > kBsManyGroups;
    const int* list = many ? d.ghard : (small ? nullptr : d.glarge);
    const int ng = many ? d.ctl->nhard : (small ? d.ctl->ngroups : d.ctl->nlarge);
    const int tid = threadIdx.x;
    const int a = tid / TA, lt = tid % TA;
    const int cap = p.bs_max_substeps;
    const double tol2 = p.bs_tol * p.bs_tol;
    static_assert(CA == 1 || NT == 32, "the cluster form has one warp per attempt");
    __shared__ int s_gi;
    // cluster form: substeps are numbered (the same in every block); attempt 0
    // announces an acceptance by writing its substep number into every block's
    // decision, so no stale announcement can be taken for a later substep
    int epoch = 0;
    if (tid == 0) S.decision = -1;
    for (;;) {
        // blocks take groups from a queue, so a long group holds up only its own block
        __syncthreads();
        if (CA > 1) {
            // the cluster's first block takes the group; the others read it there
            if (arank == 0 && tid == 0) S.gi = atomicAdd(&d.ctl->qlock[kind], 1);
            cg::this_cluster().sync();
            if (tid == 0) s_gi = cg::this_cluster().map_shared_rank(&S, 0)->gi;
            cg::this_cluster().sync();
        } else if (tid == 0) {
            s_gi = atomicAdd(&d.ctl->qlock[kind], 1);
        }
        __syncthreads();
        const int gi = s_gi;
        if (gi >= ng) break;
        const int g = list ? list[gi] : gi;
        const int mb = d.goff[g], nm = d.goff[g + 1] - mb;
        if (nm < lo || (nm > M && kind < 2)) continue;   // another lockstep kernel's group
        if (nm > M) {
            if (tid == 0 && arank == 0) set_status(d.ctl, kEoverflow, 1000000 + g);
            return;
        }
        // sp lanes a (sequence, member), adjacent, split its mutual terms (a
        // power of two, so that a warp's shuffles sum them; no more parts than
        // the group has big members, the only sources)
        int nbg = 0;
        for (int q = 0; q < nm; q++) {
            const int gb = d.members[mb + q];
            const SysInfo& gs = d.sys[d.body_sys[gb]];
            nbg += gb - gs.off < gs.nb ? 1 : 0;
        }
        int sp = 1;
        while (2 * sp * kBsRows * nm <= TA && sp < 32 && 2 * sp <= nbg) sp *= 2;
        const int si = lt % sp, k = (lt / sp) / nm, b = (lt / sp) % nm;   // part, sequence, member
        const bool act = k < kBsRows;
        const double M0g = d.M0s[d.body_sys[d.members[mb]]];   // the star of the group's system
        if (tid < nm) {
            int gb = d.members[mb + tid];
            S.gid[tid] = gb;
            S.y[0][tid] = d.x0[gb];
            S.y[1][tid] = d.y0[gb];
            S.y[2][tid] = d.z0[gb];
            S.y[3][tid] = d.vx0[gb];
            S.y[4][tid] = d.vy0[gb];
            S.y[5][tid] = d.vz0[gb];
            S.m[tid] = d.m[gb];
            S.R[tid] = d.R[gb];
            S.rc[tid] = d.rc[gb];
            S.alive[tid] = d.alive[gb];
            const SysInfo& gs = d.sys[d.body_sys[gb]];
            S.big[tid] = gb - gs.off < gs.nb;
        }
        if (tid == 0) {
            S.El = 0.0;
            S.nmerge = 0;
        }
        __syncthreads();
        if (tid < nm) {
            const double rcp = S.rc[tid];
            S.prc2[tid] = rcp * rcp;
            S.pc01[tid] = 0.1 * rcp;
            S.pinv[tid] = 1.0 / (0.9 * rcp);
        }
        __syncthreads();
        const double dt = p.dt;
        const int n = 2 * (k + 1);
        double t = 0.0, H = dt;
        int nsub = 0, failed = 0, finished = 0;
        while (!finished && !failed) {
            // attempt 0 takes min(H, what remains); attempt j takes half of attempt j-1,
            // exactly the step sizes the sequential method would try after rejections
            double rem = dt - t;
            int last0 = 0;
            if (fabs(H) >= fabs(rem)) {
                H = rem;
                last0 = 1;
            }
            const double Ha = ldexp(H, -(a + arank));
            const double h = Ha / n;
            double za[6], zb[6];
            if (act)
                for (int c = 0; c < 6; c++) za[c] = zb[c] = S.y[c][b];
            if (lt == 0) S.kacc[a] = -1;
            if (CA == 1 && tid == 0) S.decision = -1;
            epoch++;
            __syncthreads();
            for (int r = 0; r <= 2 * kBsRows; r++) {
                const bool live = act && r <= n;
                if (live) {
                    const double* zp = (r == 0) ? za : zb;
                    S.pos[a][k][0][b] = zp[0];
                    S.pos[a][k][1][b] = zp[1];
                    S.pos[a][k][2][b] = zp[2];
                }
                __syncthreads();
                double f[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                if (live && S.alive[b]) {
                    const double* zp = (r == 0) ? za : zb;
                    f[0] = zp[3];
                    f[1] = zp[4];
                    f[2] = zp[5];
                    bs_accel<NT, A>(S, p, p.G * M0g, nm, a, k, b, si, sp, zp[0], zp[1], zp[2], f[3], f[4], f[5]);
                }
                // sum the sp parts (every lane of the block takes part)
                for (int o = sp >> 1; o >= 1; o >>= 1) {
                    f[3] += __shfl_xor_sync(0xffffffffu, f[3], o);
                    f[4] += __shfl_xor_sync(0xffffffffu, f[4], o);
                    f[5] += __shfl_xor_sync(0xffffffffu, f[5], o);
                }
                if (live) {
                    if (r == 0) {
                        for (int c = 0; c < 6; c++) zb[c] = za[c] + h * f[c];
                    } else if (r < n) {
                        for (int c = 0; c < 6; c++) {
                            double znew = za[c] + 2.0 * h * f[c];
                            za[c] = zb[c];
                            zb[c] = znew;
                        }
                    } else {
                        // sequence k done: its midpoint result, extrapolated below
                        for (int c = 0; c < 6; c++) S.raw[a][c][b] = 0.5 * (zb[c] + za[c] + h * f[c]);
                    }
                }
                if (r >= 2 && (r & 1) == 0) {
                    // row kr of the tableau, one lane per (component, member) of each
                    // attempt: the six Neville chains of a member run side by side
                    const int kr = r / 2 - 1;
                    __syncthreads();
                    if (lt < 6 * nm) {
                        const int c = lt / nm, bb = lt % nm;
                        double cur = S.raw[a][c][bb];
                        double prev_col = 0.0;
                        for (int j = 1; j <= kr; j++) {
                            const double up = S.row[a][j - 1][c][bb];
                            S.row[a][j - 1][c][bb] = cur;
                            prev_col = cur;
                            cur = cur + (cur - up) * kNeville[kr][j];
                        }
                        S.row[a][kr][c][bb] = cur;
                        S.diag[a][kr][c][bb] = cur;
                        const double df = cur - prev_col;
                        S.df2[a][c][bb] = df * df;
                        S.cur2[a][c][bb] = cur * cur;
                    }
                    __syncthreads();
                    if (lt < nm) {
                        // this member passes the acceptance test: |dX|^2 <= tol^2 |X|^2
                        // and the same for V (the test without its divisions); a NaN fails
                        int pass = 1;
                        if (kr >= 1 && S.alive[lt]) {
                            const double dsq_x = S.df2[a][0][lt] + S.df2[a][1][lt] + S.df2[a][2][lt];
                            const double nx = S.cur2[a][0][lt] + S.cur2[a][1][lt] + S.cur2[a][2][lt];
                            const double dsq_v = S.df2[a][3][lt] + S.df2[a][4][lt] + S.df2[a][5][lt];
                            const double nv = S.cur2[a][3][lt] + S.cur2[a][4][lt] + S.cur2[a][5][lt];
                            pass = dsq_x <= tol2 * fmax(nx, 2.3e-308) && dsq_v <= tol2 * fmax(nv, 2.3e-308);
                        }
                        S.ok[a][kr][lt] = pass;
                    }
                }
                __syncthreads();
                if (r >= 4 && (r & 1) == 0) {
                    const int kr = r / 2 - 1;           // row finished this round
                    if (lt == 0 && S.kacc[a] < 0 && kr >= 1) {
                        int all = 1;
                        for (int q = 0; q < nm; q++) all &= S.ok[a][kr][q];
                        if (all) S.kacc[a] = kr;
                    }
                    if (CA > 1) {
                        // attempt 0 accepted: every block of the cluster learns it
                        __syncthreads();
                        if (arank == 0 && tid == 0 && S.kacc[0] >= 0)
                            for (int q = 0; q < CA; q++) cg::this_cluster().map_shared_rank(&S, q)->decision = epoch;
                    } else {
                        __syncthreads();
                        if (tid == 0)
                            for (int q = 0; q < A; q++) S.kq[q] = S.kacc[q];
                    }
                    if (CA == 1 && tid == 0) {
                        // attempt 0 accepted: done; at the last round every attempt has
                        // decided and the first accepted one (in halving order) is taken
                        constexpr int NA = CA > 1 ? CA : A;
                        if (S.kq[0] >= 0) S.decision = 0;
                        else if (r == 2 * kBsRows) {
                            int dcs = NA;
                            for (int q = NA - 1; q >= 0; q--)
                                if (S.kq[q] >= 0) dcs = q;
                            S.decision = dcs;
                        }
                    }
                    if (CA == 1) {
                        __syncthreads();
                        if (S.decision >= 0) break;
                    }
                }
                if (CA > 1) {
                    // every round: has attempt 0 announced this substep?  (one warp)
                    int seen = 0;
                    if (tid == 0) seen = *reinterpret_cast<volatile int*>(&S.decision) == epoch;
                    if (__shfl_sync(0xffffffffu, seen, 0)) break;
                }
            }
            if (CA > 1) {
                // every block is out of its rounds; each reads every attempt's row
                // and takes the first accepted one in halving order (all alike)
                cg::this_cluster().sync();
                if (tid == 0) {
                    int dcs = CA;
                    for (int q = CA - 1; q >= 0; q--) {
                        S.kq[q] = cg::this_cluster().map_shared_rank(&S, q)->kacc[0];
                        if (S.kq[q] >= 0) dcs = q;
                    }
                    S.dec = dcs;
                }
                __syncthreads();
            }
            const int dec = CA > 1 ? S.dec : S.decision;
            // replay the sequential control flow over the attempts just made
            constexpr int NA = CA > 1 ? CA : A;
            for (int q = 0; q < NA; q++) {
                nsub++;
                const double Hq = ldexp(H, -q);
                if (q == dec) {
                    const int kacc = S.kq[q];
                    if (CA > 1) {
                        // the accepted state from attempt q's block (the cluster barrier
                        // after the replay keeps it there until every block has it)
                        if (lt < 6 * nm)
                            S.y[lt / nm][lt % nm] =
                                cg::this_cluster().map_shared_rank(&S, q)->diag[0][kacc][lt / nm][lt % nm];
                    } else if (a == q && lt < 6 * nm) {
                        S.y[lt / nm][lt % nm] = S.diag[q][kacc][lt / nm][lt % nm];
                    }
                    const int lastq = (q == 0) ? last0 : 0;
                    t = lastq ? dt : t + Hq;
                    if (tid == 0) S.collide = 0;
                    __syncthreads();
                    // any pair in contact?  (exact sequential resolution only if so)
                    for (int e = tid; e < nm * nm; e += NT) {
                        int u = e / nm, w = e % nm;
                        if (w > u && S.alive[u] && S.alive[w] && bs_can_touch(S.m[u], S.m[w])) {
                            double dx = S.y[0][w] - S.y[0][u], dy = S.y[1][w] - S.y[1][u],
                                   dz = S.y[2][w] - S.y[2][u];
                            if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[u] + S.R[w]) S.collide = 1;
                        }
                    }
                    __syncthreads();
                    if (S.collide && tid == 0) {
                        for (int u = 0; u < nm; u++)
                            for (int w = u + 1; w < nm && S.alive[u]; w++) {
                                if (!S.alive[w] || !bs_can_touch(S.m[u], S.m[w])) continue;
                                double dx = S.y[0][w] - S.y[0][u], dy = S.y[1][w] - S.y[1][u],
                                       dz = S.y[2][w] - S.y[2][u];
                                if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[u] + S.R[w])
                                    bs_merge(S, p, M0g, u, w, S.El, S.nmerge);
                            }
                    }
                    __syncthreads();
                    if (lastq) {
                        finished = 1;
                        break;
                    }
                    H = Hq;
                    if (kacc <= 2) H *= 2.0;
                    else if (kacc >= 6) H *= 0.5;
                    if (nsub >= cap) failed = 1;
                    break;
                }
                if (nsub >= cap) {   // attempt q rejected
                    failed = 1;
                    break;
                }
            }
            if (dec == NA && !failed) H = ldexp(H, -NA);   // every attempt rejected
            // cluster form: no block resets its accepted row or overwrites its
            // tableau before every block has read them
            if (CA > 1) cg::this_cluster().sync();
            __syncthreads();
        }
        if (failed) {
            if (tid == 0 && arank == 0) set_status(d.ctl, kEbs, g);
            return;
        }
        // results go to the member's slot of the side buffer; the state itself
        // is updated after the step's kick, which runs beside this kernel
        if (tid < nm && arank == 0) {
            double* o = d.bsout + (int64_t)kBsOut * (mb + tid);
            for (int c = 0; c < 6; c++) o[c] = S.y[c][tid];
            o[6] = S.m[tid];
            o[7] = S.R[tid];
            o[8] = (double)S.alive[tid];
        }
        if (tid == 0 && arank == 0) {
            d.glost[g] = S.El;
            if (S.nmerge) atomicAdd(&d.ctl->nmerge, S.nmerge);
            atomicAdd(&d.ctl->nsub, (unsigned long long)nsub);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Many groups: the first attempt of each group (the whole step as one
// substep), with one lane per member and many groups to a warp; a group whose
// attempt is rejected goes on the list the lockstep kernels take next.  A warp
// works through the size classes (groups of at most 16, 8, 4, 2 members) in
// turn; its lanes form 32 / Wc segments of Wc lanes, and each segment takes
// groups of the class from a queue, the next one as soon as its group is done.  Every lane runs the same instructions on each pass of the
// loop: one derivative at the member's evaluation point, then the midpoint
// step or, at the end of a sequence, its row of the extrapolation tableau and
// the group's decision.  The sequences n_k run one after another as in the
// sequential method, so a pass does the work of up to 32 members.  What a
// group shares (positions for the forces, the error maximum, contacts) goes
// through shared memory within its segment.
constexpr int kPkWarps = 2;    // warps per block

struct PkWarp {
    double row[kBsRows][6][32];          // each lane's extrapolation tableau (in place)
    double y[6][32];                     // states at a substep's end (contacts, mergers)
    double px[32], py[32], pz[32];       // positions of the current evaluation
    double m[32], R[32], rc[32], prc2[32], pinv[32], pc01[32];
    int alive[32], gid[32];
    int big[32];                         // a big body (a source of force), not a small one
    int seg_g[16];                       // group each segment took from the queue
};

__global__ void __launch_bounds__(32 * kPkWarps) k_bs_packed(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlBsPacked);
    extern __shared__ __align__(16) unsigned char pk_smem[];
    const int lane = threadIdx.x & 31;
    PkWarp& W = reinterpret_cast<PkWarp*>(pk_smem)[threadIdx.x >> 5];
    if (d.ctl->status) return;
    if (d.ctl->ngroups <= kBsManyGroups) return;   // few groups: the lockstep kernels take them
    const Params p = d.p;
    const double tol2 = p.bs_tol * p.bs_tol, dt = p.dt;
    const int cap = p.bs_max_substeps;
    for (int c = 3; c >= 0; c--) {
        const int Wc = 2 << c;                      // 16, 8, 4, 2 lanes a segment
        const int nq = d.ctl->ncls[c];
        const int seg = lane / Wc, sl = lane % Wc, base = seg * Wc;
        const unsigned segmask = (Wc == 32 ? 0xffffffffu : ((1u << Wc) - 1u)) << base;
        int g = -1, sz = 0, mslot = 0;
        double M0g = p.M0, GM0 = p.G * p.M0;   // the star of the segment's group
        double yv[6] = {0, 0, 0, 0, 0, 0}, z0[6] = {0, 0, 0, 0, 0, 0}, z1[6] = {0, 0, 0, 0, 0, 0};
        double t = 0.0, H = 0.0, El = 0.0;
        int k = 0, ms = 0, nsub = 0, last = 0, nmerge = 0;
        bool need = true;
        for (;;) {
            // segments that need a group take the next one of the class
            if (need && sl == 0) {
                const int q = atomicAdd(&d.ctl->qcls[c], 1);
                W.seg_g[seg] = q < nq ? d.gcls[c * d.gcap + q] : -1;
            }
            __syncwarp();
            if (need) {
                need = false;
                g = W.seg_g[seg];
                sz = g >= 0 ? d.goff[g + 1] - d.goff[g] : 0;
                if (g >= 0) {
                    M0g = d.M0s[d.body_sys[d.members[d.goff[g]]]];
                    GM0 = p.G * M0g;
                }
                W.alive[lane] = 0;
                W.big[lane] = 0;
                if (sl < sz) {
                    mslot = d.goff[g] + sl;
                    const int gb = d.members[mslot];
                    W.gid[lane] = gb;
                    yv[0] = d.x0[gb]; yv[1] = d.y0[gb]; yv[2] = d.z0[gb];
                    yv[3] = d.vx0[gb]; yv[4] = d.vy0[gb]; yv[5] = d.vz0[gb];
                    W.m[lane] = d.m[gb];
                    W.R[lane] = d.R[gb];
                    const double rc = d.rc[gb];
                    W.rc[lane] = rc;
                    W.prc2[lane] = rc * rc;
                    W.pc01[lane] = 0.1 * rc;
                    W.pinv[lane] = 1.0 / (0.9 * rc);
                    W.alive[lane] = d.alive[gb];
                    const SysInfo& gs = d.sys[d.body_sys[gb]];
                    W.big[lane] = gb - gs.off < gs.nb;
                }
                t = 0.0;
                H = dt;
                last = 0;
                if (fabs(H) >= fabs(dt - t)) {
                    H = dt - t;
                    last = 1;
                }
                k = 0;
                ms = 0;
                nsub = 0;
                El = 0.0;
                nmerge = 0;
            }
            __syncwarp();
            const bool active = g >= 0;
            if (!__any_sync(0xffffffffu, active)) break;   // the class is done for the whole warp
            const bool live = active && sl < sz;
            // evaluation point: the substep's start (ms == 0) or the midpoint chain
            {
                const bool st = ms == 0;
                W.px[lane] = st ? yv[0] : z1[0];
                W.py[lane] = st ? yv[1] : z1[1];
                W.pz[lane] = st ? yv[2] : z1[2];
            }
            __syncwarp();
            double f[6] = {0, 0, 0, 0, 0, 0};
            if (live && W.alive[lane]) {
                const double P0 = W.px[lane], P1 = W.py[lane], P2 = W.pz[lane];
                const bool st = ms == 0;
                f[0] = st ? yv[3] : z1[3];
                f[1] = st ? yv[4] : z1[4];
                f[2] = st ? yv[5] : z1[5];
                const double r2 = P0 * P0 + P1 * P1 + P2 * P2, ri = rsqrt(r2);
                const double sk = -GM0 * (ri * ri * ri);
                double ax = sk * P0, ay = sk * P1, az = sk * P2;
                for (int j = 0; j < Wc - 1; j++) {   // the j-th other lane of the segment, ascending
                    const int o = base + j + (j >= sl ? 1 : 0);
                    if (!W.alive[o] || !W.big[o]) continue;
                    const int w = gt_nonneg(W.rc[lane], W.rc[o]) ? lane : o;
                    bs_pair(p, P0, P1, P2, W.px[o], W.py[o], W.pz[o], W.m[o], W.rc[w], W.prc2[w], W.pc01[w],
                            W.pinv[w], ax, ay, az);
                }
                f[3] = ax;
                f[4] = ay;
                f[5] = az;
            }
            const int n = 2 * (k + 1);
            const double h = H / n;
            const int stage = ms == 0 ? 0 : (ms < n ? 1 : 2);
            double cur[6] = {0, 0, 0, 0, 0, 0};
            bool pass = true;   // lanes without a live member never hold a segment back
            if (stage < 2) {
                // first step z1 = y + h f; then z0 <- z1, z1 <- z0 + 2 h f
                for (int q = 0; q < 6; q++) {
                    const double b0 = stage == 0 ? yv[q] : z0[q];
                    const double zn = b0 + (stage == 0 ? h : 2.0 * h) * f[q];
                    z0[q] = stage == 0 ? yv[q] : z1[q];
                    z1[q] = zn;
                }
            } else if (live) {
                double dsq_x = 0.0, dsq_v = 0.0, nx = 0.0, nv = 0.0;
                for (int q = 0; q < 6; q++) {
                    double cv = 0.5 * (z1[q] + z0[q] + h * f[q]), pv = 0.0;
                    for (int j = 1; j <= k; j++) {
                        const double up = W.row[j - 1][q][lane];
                        W.row[j - 1][q][lane] = cv;
                        pv = cv;
                        cv = cv + (cv - up) * kNeville[k][j];
                    }
                    W.row[k][q][lane] = cv;
                    cur[q] = cv;
                    const double df = cv - pv;
                    if (q < 3) {
                        dsq_x += df * df;
                        nx += cv * cv;
                    } else {
                        dsq_v += df * df;
                        nv += cv * cv;
                    }
                }
                if (k >= 1 && W.alive[lane]) {
                    // |dX|^2 <= tol^2 |X|^2 and the same for V; a NaN fails it
                    pass = dsq_x <= tol2 * fmax(nx, 2.3e-308) && dsq_v <= tol2 * fmax(nv, 2.3e-308);
                }
            }
            // the segment's members all pass (a ballot: no FP64 work)
            const bool seg_pass = (__ballot_sync(0xffffffffu, pass) & segmask) == segmask;
            // 0: on with the sequence, 1: next sequence, 2: accept row k, 3: reject the substep
            int decision = 0;
            if (active && stage == 2) {
                const bool acc = k >= 1 && seg_pass;
                decision = acc ? 2 : (k == kBsRows - 1 ? 3 : 1);
            }
            if (decision == 2 && live)
                for (int q = 0; q < 6; q++) W.y[q][lane] = cur[q];
            __syncwarp();
            // contacts after an accepted substep: each lane tests its pairs with
            // later members; the segment's first lane merges in the sequential order
            bool touch = false;
            if (decision == 2 && live && W.alive[lane])
                for (int o = lane + 1; o < base + sz; o++) {
                    if (!W.alive[o] || !bs_can_touch(W.m[lane], W.m[o])) continue;
                    const double ddx = cur[0] - W.y[0][o], ddy = cur[1] - W.y[1][o], ddz = cur[2] - W.y[2][o];
                    const double rs = W.R[lane] + W.R[o];
                    if (ddx * ddx + ddy * ddy + ddz * ddz <= rs * rs * (1.0 + 1e-9)) touch = true;
                }
            const unsigned tb = __ballot_sync(0xffffffffu, touch);
            if (decision == 2 && sl == 0 && (tb & segmask)) {
                for (int u = base; u < base + sz; u++)
                    for (int w = u + 1; w < base + sz && W.alive[u]; w++) {
                        if (!W.alive[w] || !bs_can_touch(W.m[u], W.m[w])) continue;
                        const double ddx = W.y[0][w] - W.y[0][u], ddy = W.y[1][w] - W.y[1][u],
                                     ddz = W.y[2][w] - W.y[2][u];
                        if (sqrt(ddx * ddx + ddy * ddy + ddz * ddz) <= W.R[u] + W.R[w])
                            bs_merge(W, p, M0g, u, w, El, nmerge);
                    }
            }
            __syncwarp();
            if (decision == 2 && live)
                for (int q = 0; q < 6; q++) yv[q] = W.y[q][lane];
            // step control (the same on every lane of a segment)
            if (active) {
                if (stage < 2) {
                    ms++;
                } else {
                    ms = 0;
                    if (decision == 1) {
                        k++;
                    } else {
                        nsub++;
                        bool fin = false, failed = false, hard = false;
                        if (decision == 2) {
                            t = last ? dt : t + H;
                            if (last) fin = true;
                            else if (k <= 2) H *= 2.0;
                            else if (k >= 6) H *= 0.5;
                        } else {
                            hard = fin = true;   // first attempt rejected: the lockstep kernels redo the group
                        }
                        if (!fin && nsub >= cap) fin = failed = true;
                        k = 0;
                        if (fin && hard) {
                            if (sl == 0) {
                                const int q = atomicAdd(&d.ctl->nhard, 1);
                                if (q < d.gcap) d.ghard[q] = g;
                                else set_status(d.ctl, kEoverflow, -7);
                            }
                            need = true;
                        } else if (fin) {
                            if (live) {
                                double* o = d.bsout + (int64_t)kBsOut * mslot;
                                for (int q = 0; q < 6; q++) o[q] = yv[q];
                                o[6] = W.m[lane];
                                o[7] = W.R[lane];
                                o[8] = (double)W.alive[lane];
                            }
                            if (sl == 0) {
                                d.glost[g] = El;
                                if (nmerge) atomicAdd(&d.ctl->nmerge, nmerge);
                                atomicAdd(&d.ctl->nsub, (unsigned long long)nsub);
                                if (failed) set_status(d.ctl, kEbs, g);
                            }
                            need = true;
                        } else {
                            last = 0;
                            if (fabs(H) >= fabs(dt - t)) {
                                H = dt - t;
                                last = 1;
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// Groups of up to four members (nearly every encounter): the attempts (step
// sizes H, H/2, H/4, H/8, or H and H/2) are the blocks of a cluster; when
// every one is rejected the next round tries the following halvings, so the
// sizes tried and accepted are those of the sequential scheme.  Inside a
// block, three warps, which the SM issues from three of its schedulers, each
// with its own FP64 unit (on this chip a warp pays about the same for an FP64
// instruction whatever its dependences, so what shortens a round is fewer
// instructions on the warp that waits):
//   warp 0 keeps each (sequence, member) state and takes the midpoint steps,
//          then the extrapolation, acceptance test and decision;
//   warps 1 and 2 evaluate the (1 - K) mutual terms at the even and at the
//          odd evaluation points;
//   warp 3 evaluates the stellar term at every point, in order.
// In the midpoint sequence x_{m+1} = x_{m-1} + 2h v_m, v_{m+1} = v_{m-1} +
// 2h a(x_m), the position x_{m+2} needs a(x_m) but not a(x_{m+1}), so the
// accelerations at two successive points are computed at once: as soon as
// a(x_m) arrives, warp 0 forms v_{m+1} and x_{m+2} and hands x_{m+2} to the
// warp of its parity while the other warp is still on a(x_{m+1}).  The
// arithmetic is that of the sequential scheme, except that a point's
// acceleration is the stellar term plus the sum of the mutual terms (the
// two parts come from different warps).  Four named barriers hand over
// positions and accelerations, one pair per parity, each met by warp 0, the
// mutual warp of its parity and the stellar warp; buffers are doubled by
// parity.  The four warps sit on the SM's four schedulers, each with its
// own FP64 unit.  Lanes: k * nm + b
// (sequence k, member b).  Attempt 0 announces its acceptance to the other
// blocks through distributed shared memory.
struct WsSh {
    static constexpr int M = 4;
    double y[6][M];                      // current state, component-major
    double pos[2][kBsRows][3][M];        // evaluation points, by parity of the round
    double acc[2][kBsRows][3][M];        // mutual terms there
    double sacc[2][kBsRows][3][M];       // stellar terms there
    double row[kBsRows][6][M];           // the last extrapolated row of each member
    double diag[kBsRows][6][M];          // T[k][k] of every finished row
    double raw[6][M];                    // midpoint result of the sequence finishing this round
    double df2[6][M], cur2[6][M];
    double m[M], R[M], rc[M], prc2[M], pinv[M], pc01[M];
    int alive[M], gid[M], big[M], ok[M];
    int kacc;                            // this block's attempt: accepted row, -1 while none
    int stop;                            // warp 0 tells the evaluating warps that the rounds are over
    int decision;                        // the substep number attempt 0 announced
    int dec, gi, collide, nmerge;
    int kq[4];
    double El;
};

constexpr int kWsThreads = 128;
constexpr int kBarPos0 = 1, kBarPos1 = 2;   // named barriers: evaluation points written (warp 0 -> 1 or 2, and 3)
constexpr int kBarAcc0 = 3, kBarAcc1 = 4;   // accelerations written (warp 1 or 2, and 3 -> 0)

// every named barrier is met by three warps
__device__ __forceinline__ void ws_bar_sync(int id) { asm volatile("bar.sync %0, 96;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void ws_bar_arrive(int id) { asm volatile("bar.arrive %0, 96;" ::"r"(id) : "memory"); }

// Attempts a cluster: four when the encounter integrator has the GPU to
// itself (a rejected substep costs no extra round unless all four fail);
// two beside the kick, whose blocks then get the registers the other two
// would hold (measured on the 16384-body disk: the kick and the encounter
// branch end together, and the step is 2-3% shorter than with four).
constexpr int kWsAttemptsAlone = 4, kWsAttemptsBeside = 2;

template <int CA>
__global__ void __launch_bounds__(kWsThreads, 6) k_bs_ws(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlBsWs);
    __shared__ WsSh S;
    __shared__ int s_gi;
    constexpr int M = WsSh::M;
    static_assert(CA >= 1 && CA <= 4, "one to four attempts a cluster");
    cg::cluster_group cl = cg::this_cluster();
    const int arank = (int)cl.block_rank();
    // (no status check: every block of a cluster must take the same path, and
    // another kernel may set the status while the cluster's blocks start)
    const Params p = d.p;
    const bool many = d.ctl->ngroups > kBsManyGroups;
    const int* list = many ? d.ghard : nullptr;
    const int ng = many ? d.ctl->nhard : d.ctl->ngroups;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cap = p.bs_max_substeps;
    const double tol2 = p.bs_tol * p.bs_tol;
    int epoch = 0;
    if (tid == 0) S.decision = -1;
    for (;;) {
        __syncthreads();
        if (arank == 0 && tid == 0) S.gi = atomicAdd(&d.ctl->qlock[0], 1);
        cl.sync();
        if (tid == 0) s_gi = cl.map_shared_rank(&S, 0)->gi;
        cl.sync();
        const int gi = s_gi;
        if (gi >= ng) break;
        const int g = list ? list[gi] : gi;
        const int mb = d.goff[g], nm = d.goff[g + 1] - mb;
        if (nm > M) continue;                // a larger group: the other lockstep kernels'
        const double M0g = d.M0s[d.body_sys[d.members[mb]]], GM0 = p.G * M0g;   // the group's star
        const int k = lane / nm, b = lane % nm;
        const bool act = k < kBsRows;
        if (tid < nm) {
            const int gb = d.members[mb + tid];
            S.gid[tid] = gb;
            S.y[0][tid] = d.x0[gb];
            S.y[1][tid] = d.y0[gb];
            S.y[2][tid] = d.z0[gb];
            S.y[3][tid] = d.vx0[gb];
            S.y[4][tid] = d.vy0[gb];
            S.y[5][tid] = d.vz0[gb];
            S.m[tid] = d.m[gb];
            S.R[tid] = d.R[gb];
            const double rcp = d.rc[gb];
            S.rc[tid] = rcp;
            S.prc2[tid] = rcp * rcp;
            S.pc01[tid] = 0.1 * rcp;
            S.pinv[tid] = 1.0 / (0.9 * rcp);
            S.alive[tid] = d.alive[gb];
            const SysInfo& gs = d.sys[d.body_sys[gb]];
            S.big[tid] = gb - gs.off < gs.nb;
        }
        if (tid == 0) {
            S.El = 0.0;
            S.nmerge = 0;
        }
        __syncthreads();
        const double dt = p.dt;
        const int n = 2 * (k + 1);
        double t = 0.0, H = dt;
        int nsub = 0, failed = 0, finished = 0;
        while (!finished && !failed) {
            double rem = dt - t;
            int last0 = 0;
            if (fabs(H) >= fabs(rem)) {
                H = rem;
                last0 = 1;
            }
            const double h = ldexp(H, -arank) / n;
            epoch++;
            if (warp == 0) {
                // ---- warp 0: states, midpoint steps, extrapolation, decision.  At
                // iteration m a lane holds x_{m-1}, x_m, x_{m+1} and v_{m-1}, v_m.
                double Xm[3], X0[3], X1[3], Vm[3], V0[3];
                if (act)
                    for (int c = 0; c < 3; c++) {
                        X0[c] = Xm[c] = S.y[c][b];
                        V0[c] = Vm[c] = S.y[3 + c][b];
                        S.pos[0][k][c][b] = X0[c];
                        X1[c] = X0[c] + h * V0[c];   // x_1 = x_0 + h v_0
                        S.pos[1][k][c][b] = X1[c];
                    }
                if (lane == 0) {
                    S.kacc = -1;
                    S.stop = 0;
                }
                ws_bar_arrive(kBarPos0);             // points 0 and 1
                ws_bar_arrive(kBarPos1);
                for (int m = 0;; m++) {
                    const int par = m & 1;
                    ws_bar_sync(par ? kBarAcc1 : kBarAcc0);   // a(x_m)
                    if (act && m <= n) {
                        double a[3] = {0.0, 0.0, 0.0};
                        if (S.alive[b])
                            for (int c = 0; c < 3; c++) a[c] = S.sacc[par][k][c][b] + S.acc[par][k][c][b];
                        if (m < n) {
                            double vn[3];
                            for (int c = 0; c < 3; c++) vn[c] = m == 0 ? V0[c] + h * a[c] : Vm[c] + 2.0 * h * a[c];
                            // the point two ahead: x_{m+2} = x_m + 2h v_{m+1}
                            for (int c = 0; c < 3; c++) {
                                const double x2 = X0[c] + 2.0 * h * vn[c];
                                if (m + 2 <= n) S.pos[par][k][c][b] = x2;
                                Xm[c] = X0[c];
                                X0[c] = X1[c];
                                X1[c] = x2;
                                Vm[c] = V0[c];
                                V0[c] = vn[c];
                            }
                        } else {
                            // sequence k done: its midpoint result 1/2 (z_n + z_{n-1} + h f(z_n))
                            for (int c = 0; c < 3; c++) {
                                S.raw[c][b] = 0.5 * (X0[c] + Xm[c] + h * V0[c]);
                                S.raw[3 + c][b] = 0.5 * (V0[c] + Vm[c] + h * a[c]);
                            }
                        }
                    }
                    ws_bar_arrive(par ? kBarPos1 : kBarPos0);   // point m + 2
                    if (m >= 2 && (m & 1) == 0) {
                        // row kr of the tableau: sequence kr finished at this point
                        const int kr = m / 2 - 1;
                        __syncwarp();
                        if (lane < 6 * nm) {
                            const int c = lane / nm, bb = lane % nm;
                            double cur = S.raw[c][bb], prev_col = 0.0;
                            for (int j = 1; j <= kr; j++) {
                                const double up = S.row[j - 1][c][bb];
                                S.row[j - 1][c][bb] = cur;
                                prev_col = cur;
                                cur = cur + (cur - up) * kNeville[kr][j];
                            }
                            S.row[kr][c][bb] = cur;
                            S.diag[kr][c][bb] = cur;
                            const double df = cur - prev_col;
                            S.df2[c][bb] = df * df;
                            S.cur2[c][bb] = cur * cur;
                        }
                        __syncwarp();
                        if (lane < nm) {
                            int pass = 1;
                            if (kr >= 1 && S.alive[lane]) {
                                const double dsq_x = S.df2[0][lane] + S.df2[1][lane] + S.df2[2][lane];
                                const double nx = S.cur2[0][lane] + S.cur2[1][lane] + S.cur2[2][lane];
                                const double dsq_v = S.df2[3][lane] + S.df2[4][lane] + S.df2[5][lane];
                                const double nv = S.cur2[3][lane] + S.cur2[4][lane] + S.cur2[5][lane];
                                pass = dsq_x <= tol2 * fmax(nx, 2.3e-308) && dsq_v <= tol2 * fmax(nv, 2.3e-308);
                            }
                            S.ok[lane] = pass;
                        }
                        __syncwarp();
                        if (lane == 0 && kr >= 1 && S.kacc < 0) {
                            int all = 1;
                            for (int q = 0; q < nm; q++) all &= S.ok[q];
                            if (all) {
                                S.kacc = kr;
                                if (arank == 0)
                                    for (int q = 0; q < CA; q++) cl.map_shared_rank(&S, q)->decision = epoch;
                            }
                        }
                    }
                    // stop: this attempt accepted, attempt 0 announced, or every row done
                    int st = 0;
                    if (lane == 0)
                        st = S.kacc >= 0 || *reinterpret_cast<volatile int*>(&S.decision) == epoch ||
                             m == 2 * kBsRows;
                    if (__shfl_sync(0xffffffffu, st, 0)) {
                        // the evaluations of points m + 1 and m + 2 are under way: take
                        // (and drop) them, then release both warps with the stop flag
                        ws_bar_sync(par ? kBarAcc0 : kBarAcc1);
                        ws_bar_sync(par ? kBarAcc1 : kBarAcc0);
                        if (lane == 0) S.stop = 1;
                        ws_bar_arrive(kBarPos0);
                        ws_bar_arrive(kBarPos1);
                        break;
                    }
                }
            } else if (warp == 3) {
                // ---- warp 3: the stellar term at every point, in order.  At the
                // stop, warp 0 releases both position barriers: this warp meets
                // the second one too, which the other parity's warp waits at.
                for (int m = 0;; m++) {
                    const int par = m & 1;
                    ws_bar_sync(par ? kBarPos1 : kBarPos0);
                    if (*reinterpret_cast<volatile int*>(&S.stop)) {
                        ws_bar_sync(par ? kBarPos0 : kBarPos1);
                        break;
                    }
                    if (act && m <= n && S.alive[b]) {
                        const double px = S.pos[par][k][0][b], py = S.pos[par][k][1][b], pz = S.pos[par][k][2][b];
                        const double r2 = px * px + py * py + pz * pz, ri = rsqrt(r2);
                        const double sk = -GM0 * (ri * ri * ri);
                        S.sacc[par][k][0][b] = sk * px;
                        S.sacc[par][k][1][b] = sk * py;
                        S.sacc[par][k][2][b] = sk * pz;
                    }
                    ws_bar_arrive(par ? kBarAcc1 : kBarAcc0);
                }
            } else {
                // ---- warps 1 and 2: mutual terms at the points of their parity
                const int par = warp - 1;
                for (int m = par;; m += 2) {
                    ws_bar_sync(par ? kBarPos1 : kBarPos0);
                    if (*reinterpret_cast<volatile int*>(&S.stop)) break;
                    if (act && m <= n && S.alive[b]) {
                        const double px = S.pos[par][k][0][b], py = S.pos[par][k][1][b], pz = S.pos[par][k][2][b];
                        double ax = 0.0, ay = 0.0, az = 0.0;
                        for (int j = 0; j < nm - 1; j++) {   // the other members, ascending
                            const int o = j + (j >= b ? 1 : 0);
                            if (!S.alive[o] || !S.big[o]) continue;
                            const int w = gt_nonneg(S.rc[b], S.rc[o]) ? b : o;
                            bs_pair(p, px, py, pz, S.pos[par][k][0][o], S.pos[par][k][1][o], S.pos[par][k][2][o],
                                    S.m[o], S.rc[w], S.prc2[w], S.pc01[w], S.pinv[w], ax, ay, az);
                        }
                        S.acc[par][k][0][b] = ax;
                        S.acc[par][k][1][b] = ay;
                        S.acc[par][k][2][b] = az;
                    }
                    ws_bar_arrive(par ? kBarAcc1 : kBarAcc0);
                }
            }
            __syncthreads();
            // every block is out of its rounds: the first accepted attempt in
            // halving order is taken, the same in every block
            cl.sync();
            if (tid == 0) {
                int dcs = CA;
                for (int q = CA - 1; q >= 0; q--) {
                    S.kq[q] = cl.map_shared_rank(&S, q)->kacc;
                    if (S.kq[q] >= 0) dcs = q;
                }
                S.dec = dcs;
            }
            __syncthreads();
            const int dec = S.dec;
            // replay the sequential control flow over the attempts just made
            for (int q = 0; q < CA; q++) {
                nsub++;
                const double Hq = ldexp(H, -q);
                if (q == dec) {
                    const int kacc = S.kq[q];
                    if (tid < 6 * nm) S.y[tid / nm][tid % nm] = cl.map_shared_rank(&S, q)->diag[kacc][tid / nm][tid % nm];
                    const int lastq = (q == 0) ? last0 : 0;
                    t = lastq ? dt : t + Hq;
                    if (tid == 0) S.collide = 0;
                    __syncthreads();
                    // any pair in contact?  (exact sequential resolution only if so)
                    for (int e = tid; e < nm * nm; e += kWsThreads) {
                        const int u = e / nm, w = e % nm;
                        if (w > u && S.alive[u] && S.alive[w] && bs_can_touch(S.m[u], S.m[w])) {
                            const double dx = S.y[0][w] - S.y[0][u], dy = S.y[1][w] - S.y[1][u],
                                         dz = S.y[2][w] - S.y[2][u];
                            if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[u] + S.R[w]) S.collide = 1;
                        }
                    }
                    __syncthreads();
                    if (S.collide && tid == 0) {
                        for (int u = 0; u < nm; u++)
                            for (int w = u + 1; w < nm && S.alive[u]; w++) {
                                if (!S.alive[w] || !bs_can_touch(S.m[u], S.m[w])) continue;
                                const double dx = S.y[0][w] - S.y[0][u], dy = S.y[1][w] - S.y[1][u],
                                             dz = S.y[2][w] - S.y[2][u];
                                if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[u] + S.R[w])
                                    bs_merge(S, p, M0g, u, w, S.El, S.nmerge);
                            }
                    }
                    __syncthreads();
                    if (lastq) {
                        finished = 1;
                        break;
                    }
                    H = Hq;
                    if (kacc <= 2) H *= 2.0;
                    else if (kacc >= 6) H *= 0.5;
                    if (nsub >= cap) failed = 1;
                    break;
                }
                if (nsub >= cap) {   // attempt q rejected
                    failed = 1;
                    break;
                }
            }
            if (dec == CA && !failed) H = ldexp(H, -CA);   // every attempt rejected
            // no block resets its accepted row or overwrites its tableau before
            // every block has read them
            cl.sync();
        }
        if (failed) {
            if (tid == 0 && arank == 0) set_status(d.ctl, kEbs, g);
            return;
        }
        if (tid < nm && arank == 0) {
            double* o = d.bsout + (int64_t)kBsOut * (mb + tid);
            for (int c = 0; c < 6; c++) o[c] = S.y[c][tid];
            o[6] = S.m[tid];
            o[7] = S.R[tid];
            o[8] = (double)S.alive[tid];
        }
        if (tid == 0 && arank == 0) {
            d.glost[g] = S.El;
            if (S.nmerge) atomicAdd(&d.ctl->nmerge, S.nmerge);
            atomicAdd(&d.ctl->nsub, (unsigned long long)nsub);
        }
    }
}

constexpr int kBsLargeThreads = 256;   // groups of up to 32 members: one attempt
constexpr int kBsLargerThreads = 512;  // groups of up to 64 members: one attempt

cudaError_t bs_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_bs_packed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kPkWarps * sizeof(PkWarp)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_bs<kBsLargeThreads, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(BsSh<kBsLargeThreads, 1>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bs<kBsLargerThreads, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(BsSh<kBsLargerThreads, 1>));
}

void launch_bs_packed(const Dev& d, int nsm, cudaStream_t s) {
    // two warps an SM: FP64 issues about one warp instruction per 17 cycles an
    // SM, so fewer warps sharing it finish their groups' chains sooner
    k_bs_packed<<<nsm, 32 * kPkWarps, kPkWarps * sizeof(PkWarp), s>>>(d);
    prof_mark("bs: many groups, packed");
}

// The lockstep kernels: groups of up to 4 members on s, the larger groups on
// the branch s2 (s2 == s: one after the other).  Within a stream priority,
// blocks are placed in launch order, and a kernel whose blocks do not fit yet
// holds back the kernels launched after it.  small_first (the kick runs
// beside, on a stream of lower priority than s2, which is lower than s): the
// small-group kernel goes first, since beside the kick's blocks only its
// blocks fit (a larger-group block takes half an SM's registers or more).
// Otherwise the larger-group kernels go first, on a branch of the same
// priority, and the small-group blocks fill the room they leave.  The
// small-group clusters hold two attempts beside the kick, four otherwise.
cudaError_t launch_bs_lockstep(const Dev& d, int nsm, cudaStream_t s, cudaStream_t s2, cudaEvent_t fork,
                               cudaEvent_t join, bool small_first) {
    cudaError_t err = cudaSuccess;   // the first failed launch, if any (the cluster and cooperative ones)
    if (s2 != s) {
        cudaEventRecord(fork, s);
        cudaStreamWaitEvent(s2, fork, 0);
    }
    auto larger = [&] {
        k_bs<kBsLargeThreads, 1, 1><<<nsm, kBsLargeThreads, sizeof(BsSh<kBsLargeThreads, 1>), s2>>>(d, 1);
        if (s2 == s) prof_mark("bs: groups of 5-32");
        k_bs<kBsLargerThreads, 1, 1><<<nsm, kBsLargerThreads, sizeof(BsSh<kBsLargerThreads, 1>), s2>>>(d, 2);
        if (s2 == s) prof_mark("bs: groups of 33-64");
        const cudaError_t e = launch_bs_huge(d, nsm, s2);
        if (err == cudaSuccess) err = e;
    };
    if (!small_first) larger();
    {
        // groups of up to 4 members: clusters of two or four blocks, one attempt each
        cudaLaunchConfig_t cfg = {};
        const int ca = small_first ? kWsAttemptsBeside : kWsAttemptsAlone;
        cfg.gridDim = dim3((unsigned)(ca * 2 * nsm));
        cfg.blockDim = dim3(kWsThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = ca;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = ca == kWsAttemptsBeside ? cudaLaunchKernelEx(&cfg, k_bs_ws<kWsAttemptsBeside>, d)
                                                      : cudaLaunchKernelEx(&cfg, k_bs_ws<kWsAttemptsAlone>, d);
        if (err == cudaSuccess) err = e;
    }
    prof_mark("bs: groups <= 4");
    if (small_first) larger();
    if (s2 != s) {
        cudaEventRecord(join, s2);
        cudaStreamWaitEvent(s, join, 0);
    }
    return err;
}

}  // namespace opal
