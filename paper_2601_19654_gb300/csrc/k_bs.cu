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
// One block of four warps per group.  Warp w runs the two midpoint
// sequences n = 2(w+1) and n = 16 - 2w (20 derivative evaluations each, so
// the warps finish together) with one member per lane; then one thread per
// (member, position-or-velocity) extrapolates its three components.  Every
// row the sequential method would compute is computed (the extra rows are
// unused), so the accepted values are those of the sequential method.
#include "opal_internal.cuh"

namespace opal {

constexpr int kM = kBsMaxMembers;
constexpr int kBsThreads = 32 * kBsWarps;

struct BsShared {
    double y[6][kM];               // current state, component-major: X, Y, Z, VX, VY, VZ
    double T0[kBsRows][6][kM];     // midpoint results; overwritten by the diagonal T[k][k]
    double pos[kBsWarps][3][kM];   // positions of the evaluation in progress, per warp
    double m[kM], R[kM], rc[kM];
    int alive[kM], gid[kM];
    double errk[kBsWarps][kBsRows];
    int kacc, collide;
    double El;
    int nmerge;
};

// derivative of the members a lane owns (q = 0, 1 -> member lane + 32 q)
__device__ __forceinline__ void bs_deriv(BsShared& S, const Params& p, int w, int nm, const double (&z)[2][6],
                                         double (&f)[2][6]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        int b = lane + 32 * q;
        if (b < nm) {
            S.pos[w][0][b] = z[q][0];
            S.pos[w][1][b] = z[q][1];
            S.pos[w][2][b] = z[q][2];
        }
    }
    __syncwarp();
    const double G = p.G, M0 = p.M0;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        int b = lane + 32 * q;
        if (b >= nm) continue;
        if (!S.alive[b]) {
#pragma unroll
            for (int c = 0; c < 6; c++) f[q][c] = 0.0;
            continue;
        }
        const double xb = z[q][0], yb = z[q][1], zb = z[q][2];
        double r2 = xb * xb + yb * yb + zb * zb, r = sqrt(r2);
        double s = -G * M0 / (r2 * r);
        double ax = s * xb, ay = s * yb, az = s * zb;
        for (int o = 0; o < nm; o++) {
            if (o == b || !S.alive[o]) continue;
            double dx = S.pos[w][0][o] - xb, dy = S.pos[w][1][o] - yb, dz = S.pos[w][2][o] - zb;
            double dr2 = dx * dx + dy * dy + dz * dz, dr = sqrt(dr2);
            double rcbo = S.rc[b] > S.rc[o] ? S.rc[b] : S.rc[o];
            double wgt = 1.0 - changeover(dr, rcbo, p.changeover);
            if (wgt == 0.0) continue;
            double t = G * S.m[o] * wgt / (dr2 * dr);
            ax += t * dx;
            ay += t * dy;
            az += t * dz;
        }
        f[q][0] = z[q][3];
        f[q][1] = z[q][4];
        f[q][2] = z[q][5];
        f[q][3] = ax;
        f[q][4] = ay;
        f[q][5] = az;
    }
    __syncwarp();
}

// modified midpoint with n steps over H from S.y, result into S.T0[row]
__device__ void bs_mmid(BsShared& S, const Params& p, int w, int nm, double H, int n, int row) {
    const int lane = threadIdx.x & 31;
    double za[2][6], zb[2][6], f[2][6];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        int b = lane + 32 * q;
#pragma unroll
        for (int c = 0; c < 6; c++) za[q][c] = (b < nm) ? S.y[c][b] : 0.0;
    }
    const double h = H / n;
    bs_deriv(S, p, w, nm, za, f);
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) zb[q][c] = za[q][c] + h * f[q][c];
    for (int st = 1; st < n; st++) {
        bs_deriv(S, p, w, nm, zb, f);
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int c = 0; c < 6; c++) {
                double znew = za[q][c] + 2.0 * h * f[q][c];
                za[q][c] = zb[q][c];
                zb[q][c] = znew;
            }
    }
    bs_deriv(S, p, w, nm, zb, f);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        int b = lane + 32 * q;
        if (b < nm)
#pragma unroll
            for (int c = 0; c < 6; c++) S.T0[row][c][b] = 0.5 * (zb[q][c] + za[q][c] + h * f[q][c]);
    }
}

__device__ void bs_merge(BsShared& S, const Params& p, int b, int q) {
    const double G = p.G, M0 = p.M0;
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
    S.El += e_before - e_after;
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
    S.nmerge++;
}

__global__ void __launch_bounds__(kBsThreads) k_bs(Dev d) {
    __shared__ BsShared S;
    if (d.ctl->status) return;
    const Params p = d.p;
    const int ng = d.ctl->ngroups;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int cap = p.bs_max_substeps;
    for (int g = blockIdx.x; g < ng; g += gridDim.x) {
        const int mb = d.goff[g], nm = d.goff[g + 1] - mb;
        if (nm > kM) {
            if (tid == 0) set_status(d.ctl, kEoverflow, 1000000 + g);
            return;
        }
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
            d.undo[3 * (mb + tid)] = d.m[gb];
            d.undo[3 * (mb + tid) + 1] = d.R[gb];
            d.undo[3 * (mb + tid) + 2] = (double)d.alive[gb];
        }
        if (tid == 0) {
            S.El = 0.0;
            S.nmerge = 0;
        }
        __syncthreads();
        const double dt = p.dt, tol = p.bs_tol;
        double t = 0.0, H = dt;
        int nsub = 0, failed = 0;
        for (;;) {
            double rem = dt - t;
            int last = 0;
            if (fabs(H) >= fabs(rem)) {
                H = rem;
                last = 1;
            }
            // all eight midpoint sequences, two per warp
            bs_mmid(S, p, w, nm, H, 2 * (w + 1), w);
            bs_mmid(S, p, w, nm, H, 2 * (kBsRows - w), kBsRows - 1 - w);
            __syncthreads();
            // extrapolation: thread (member b, part pp) owns components 3pp..3pp+2
            double ek[kBsRows];
#pragma unroll
            for (int k = 0; k < kBsRows; k++) ek[k] = 0.0;
            if (tid < 2 * nm) {
                const int b = tid >> 1, pp = tid & 1;
                double dsq[kBsRows], nrm[kBsRows];
#pragma unroll
                for (int k = 0; k < kBsRows; k++) dsq[k] = nrm[k] = 0.0;
                for (int c = 3 * pp; c < 3 * pp + 3; c++) {
                    double prev[kBsRows], cur[kBsRows];
#pragma unroll
                    for (int k = 0; k < kBsRows; k++) {
                        cur[0] = S.T0[k][c][b];
#pragma unroll
                        for (int j = 1; j <= k; j++) {
                            double ratio = (double)(k + 1) / (double)(k - j + 1);
                            double den = ratio * ratio - 1.0;
                            cur[j] = cur[j - 1] + (cur[j - 1] - prev[j - 1]) / den;
                        }
                        if (k >= 1) {
                            double df = cur[k] - cur[k - 1];
                            dsq[k] += df * df;
                        }
                        nrm[k] += cur[k] * cur[k];
                        S.T0[k][c][b] = cur[k];
#pragma unroll
                        for (int j = 0; j <= k; j++) prev[j] = cur[j];
                    }
                }
                if (S.alive[b]) {
#pragma unroll
                    for (int k = 1; k < kBsRows; k++) {
                        double sc = sqrt(nrm[k]);
                        if (sc < 1e-300) sc = 1e-300;
                        double e = sqrt(dsq[k]) / sc;
                        ek[k] = (e <= 1.7e308) ? e : HUGE_VAL;   // NaN counts as not converged
                    }
                }
            }
#pragma unroll
            for (int k = 1; k < kBsRows; k++) {
                double v = ek[k];
                for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
                if (lane == 0) S.errk[w][k] = v;
            }
            __syncthreads();
            if (tid == 0) {
                int kacc = -1;
                for (int k = 1; k < kBsRows && kacc < 0; k++) {
                    double e = S.errk[0][k];
                    for (int ww = 1; ww < kBsWarps; ww++) e = fmax(e, S.errk[ww][k]);
                    if (e <= tol) kacc = k;
                }
                S.kacc = kacc;
            }
            __syncthreads();
            const int kacc = S.kacc;
            nsub++;
            if (kacc >= 0) {
                for (int e = tid; e < 6 * nm; e += kBsThreads) {
                    int c = e / nm, b = e % nm;
                    S.y[c][b] = S.T0[kacc][c][b];
                }
                t = last ? dt : t + H;
                if (tid == 0) S.collide = 0;
                __syncthreads();
                // any pair in contact?  (exact sequential resolution only if so)
                for (int e = tid; e < nm * nm; e += kBsThreads) {
                    int b = e / nm, q = e % nm;
                    if (q > b && S.alive[b] && S.alive[q]) {
                        double dx = S.y[0][q] - S.y[0][b], dy = S.y[1][q] - S.y[1][b], dz = S.y[2][q] - S.y[2][b];
                        if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[b] + S.R[q]) S.collide = 1;
                    }
                }
                __syncthreads();
                if (S.collide && tid == 0) {
                    for (int b = 0; b < nm; b++)
                        for (int q = b + 1; q < nm && S.alive[b]; q++) {
                            if (!S.alive[q]) continue;
                            double dx = S.y[0][q] - S.y[0][b], dy = S.y[1][q] - S.y[1][b],
                                   dz = S.y[2][q] - S.y[2][b];
                            if (sqrt(dx * dx + dy * dy + dz * dz) <= S.R[b] + S.R[q]) bs_merge(S, p, b, q);
                        }
                }
                __syncthreads();
                if (last) break;
                if (kacc <= 2) H *= 2.0;
                else if (kacc >= 6) H *= 0.5;
            } else {
                H *= 0.5;
            }
            if (nsub >= cap) {
                failed = 1;
                break;
            }
        }
        if (failed) {
            if (tid == 0) set_status(d.ctl, kEbs, g);
            return;
        }
        if (tid < nm) {
            int gb = S.gid[tid];
            double x = S.y[0][tid], y = S.y[1][tid], z = S.y[2][tid];
            d.x[gb] = x; d.y[gb] = y; d.z[gb] = z;
            d.vx[gb] = S.y[3][tid]; d.vy[gb] = S.y[4][tid]; d.vz[gb] = S.y[5][tid];
            d.m[gb] = S.m[tid];
            d.R[gb] = S.R[tid];
            d.alive[gb] = S.alive[tid];
            if (S.alive[tid]) kick_floats(d, gb, x, y, z, S.m[tid], d.rc[gb]);
            else park_floats(d, gb);
            d.label[gb] = -1;
        }
        if (tid == 0) {
            d.glost[g] = S.El;
            if (S.nmerge) atomicAdd(&d.ctl->nmerge, S.nmerge);
            atomicAdd(&d.ctl->nsub, (unsigned long long)nsub);
        }
        __syncthreads();
    }
}

void launch_bs(const Dev& d, int grid, cudaStream_t s) { k_bs<<<grid, kBsThreads, 0, s>>>(d); }

}  // namespace opal
