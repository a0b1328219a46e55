// Close-encounter scan (Sec. 3.1, mce_snif block): flag every pair i < j of
// live bodies of a system whose minimum separation over the step is <= the
// critical distance max(rc_i, rc_j); then gather the flagged pairs into
// groups (connected components) for the encounter integrator.
//
// The minimum is taken over the cubic Hermite path of the relative motion
// built from the saved start-of-drift state (x0, V0) and the state after
// the drift (x1, V1).  Three stages, each a superset of the next:
//   1. FP32, on bodies sorted by the cell of their path midpoint c and tile
//      pairs culled by boxes: |c_j - c_i| < s_i + s_j, where s bounds how far
//      a body's path strays from its midpoint (plus rc);
//   2. FP32, on the list of pairs that pass, one thread per pair: distance
//      from the origin to the chord d0 -> d1 minus a bound on the path's
//      deviation from the chord;
//   3. the minimum on the survivors: the sign of g = d.d' on 16 equal
//      intervals and a bracketed Newton search for each - to + change, both
//      in FP32, then the path, d' and d'' at the root found taken in FP64
//      and the minimum there as the local quadratic's, |d|^2 - g^2 / g'
//      (an FP32 root is off by ~1e-7 of the step, which leaves errors of
//      order its square: the minimum agrees with an FP64 search to ~1e-13).
// Stages 1-2 carry margins far above FP32 rounding, so they never drop a
// pair stage 3 would flag; the flagged set is that of stage 3 alone.
#include "opal_internal.cuh"

namespace opal {

// ---------------------------------------------------------------- stage 2
__device__ __noinline__ bool chord_bound_passes(const Dev& d, int64_t i, int64_t j, float T) {
    float4 a0 = d.sc0[i], b0 = d.sc0[j], a0l = d.sc1[i], b0l = d.sc1[j];
    float4 a1 = d.kh[i], b1 = d.kh[j], a1l = d.kl[i], b1l = d.kl[j];
    float4 av0 = d.sv0[i], bv0 = d.sv0[j], av1 = d.sv1[i], bv1 = d.sv1[j];
    float d0x = (b0.x - a0.x) + (b0l.x - a0l.x), d0y = (b0.y - a0.y) + (b0l.y - a0l.y),
          d0z = (b0.z - a0.z) + (b0l.z - a0l.z);
    float d1x = (b1.x - a1.x) + (b1l.x - a1l.x), d1y = (b1.y - a1.y) + (b1l.y - a1l.y),
          d1z = (b1.z - a1.z) + (b1l.z - a1l.z);
    float u0x = bv0.x - av0.x, u0y = bv0.y - av0.y, u0z = bv0.z - av0.z;
    float u1x = bv1.x - av1.x, u1y = bv1.y - av1.y, u1z = bv1.z - av1.z;
    float wx = d1x - d0x, wy = d1y - d0y, wz = d1z - d0z;
    float ww = wx * wx + wy * wy + wz * wz;
    float t = 0.0f;
    if (ww > 0.0f) t = fminf(fmaxf(-(d0x * wx + d0y * wy + d0z * wz) / ww, 0.0f), 1.0f);
    float cx = d0x + t * wx, cy = d0y + t * wy, cz = d0z + t * wz;
    float cd = sqrtf(cx * cx + cy * cy + cz * cz);
    float nu0 = sqrtf(u0x * u0x + u0y * u0y + u0z * u0z), nu1 = sqrtf(u1x * u1x + u1y * u1y + u1z * u1z);
    float aT = fabsf(T);
    // |path - chord| <= (sqrt 3 / 18)|d1 - d0| + (4/27)|T|(|u0| + |u1|), constants rounded up
    float E = 0.0962251f * sqrtf(ww) + 0.1481482f * aT * (nu0 + nu1);
    float rcij = fmaxf(d.rcf[i], d.rcf[j]);
    float n0 = sqrtf(d0x * d0x + d0y * d0y + d0z * d0z), n1 = sqrtf(d1x * d1x + d1y * d1y + d1z * d1z);
    float margin = 1e-4f * (n0 + n1 + E + rcij) + 1e-6f * aT * (av0.w + bv0.w + av1.w + bv1.w);
    return cd - E <= rcij + margin;
}

// ---------------------------------------------------------------- stage 1
// A body's Hermite path stays within s of its midpoint c, so a pair can come
// within the critical distance only if |c_j - c_i| < s_i + s_j.  Each step
// the bodies of a system are counting-sorted by the row-major cell of c on a
// grid fitted to the system's box of midpoints (a few bodies per cell), so
// that 64 consecutive bodies of the sorted order lie close together; a tile
// of 64 gets the box of its intervals c +- s, and only tile pairs whose boxes
// overlap are tested pair by pair (a pair passing the test has overlapping
// intervals on every axis, so no such pair is skipped).

struct SortGrid {
    float lo[3];
    float inv_h;
    int nx, ny, nz;
};

// a grid over the system's box of midpoints: cells of side h, about 8 of the
// nbody bodies per cell in the two widest directions, at most nbuck cells.
// FP32 throughout: the grid only orders the bodies (any grid gives a valid
// sorted order, and the same inputs give the same grid on every run), and
// one thread's chain of FP64 operations here would hold every block of the
// kernel for microseconds.
__device__ void sort_grid(const Dev& d, int sys, float nbody, int64_t nbuck, SortGrid& g) {
    float lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = fordinv(d.sbox[3 * sys + k]);
        hi[k] = fordinv(d.sbox[3 * d.nsys + 3 * sys + k]);
        if (!(hi[k] >= lo[k])) lo[k] = hi[k] = 0.0f;   // no live body
        g.lo[k] = lo[k];
    }
    float W[3];
    for (int k = 0; k < 3; k++) W[k] = fmaxf(hi[k] - lo[k], 1e-20f);
    const float a = fmaxf(W[0], W[1]), b = fminf(W[0], W[1]);
    const float wmax = fmaxf(a, W[2]), wmid = W[2] > a ? a : (W[2] > b ? W[2] : b);
    const float cells = fmaxf(1.0f, nbody / 8.0f);
    float inv_h = sqrtf(cells) * rsqrtf(wmax) * rsqrtf(wmid);   // finite down to W = 1e-20
    const float nb = (float)max((int64_t)1, nbuck);
    float n[3];
    for (int it = 0; it < 400; it++) {
        for (int k = 0; k < 3; k++) n[k] = fminf(floorf(W[k] * inv_h) + 1.0f, 1.0e6f);
        if (n[0] * n[1] * n[2] <= nb) break;
        inv_h *= 0.8f;
    }
    // grid_index clamps to these counts, so every key stays in the grid's buckets
    g.inv_h = inv_h;
    g.nx = (int)n[0];
    g.ny = (int)n[1];
    g.nz = (int)n[2];
    while ((double)g.nx * g.ny * g.nz > (double)nb) {   // only if 400 shrinks were not enough
        if (g.nx >= g.ny && g.nx >= g.nz) g.nx = max(1, g.nx / 2);
        else if (g.ny >= g.nz) g.ny = max(1, g.ny / 2);
        else g.nz = max(1, g.nz / 2);
    }
}

// The system's cap / 4 buckets: the big bodies' grid first, then the small
// bodies' (each sized to its own count, so both sorted runs are compact), the
// last bucket for dead and padding bodies.  The sorted order is thus: live
// big bodies, live small bodies, dead ones; the kick's sources and the scan's
// big tiles are its first nb places.
__device__ __forceinline__ int64_t big_buckets(const SysInfo& si) {
    const int64_t nbk = si.cap / kBucketDiv - 1;   // buckets of live bodies
    if (si.nb >= si.n) return nbk;
    if (si.nb == 0) return 0;
    return min(nbk - 1, max((int64_t)1, (si.nb * nbk + si.n - 1) / si.n));
}

__device__ __forceinline__ int grid_index(float c, float lo, float inv_h, int n) {
    float q = floorf((c - lo) * inv_h);
    q = fminf(fmaxf(q, 0.0f), (float)(n - 1));
    return (int)q;
}

__global__ void __launch_bounds__(kBodyThreads) k_sort_count(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlSortCount);
    if (d.ctl->status) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int sys = d.body_sys[(int64_t)blockIdx.x * kBodyThreads];
    const SysInfo si = d.sys[sys];
    __shared__ SortGrid grid[2];                   // big bodies, small bodies
    const int64_t nbb = big_buckets(si);
    if (threadIdx.x == 0) sort_grid(d, sys, (float)si.nb, nbb, grid[0]);
    if (threadIdx.x == 32) sort_grid(d, sys, (float)(si.n - si.nb), si.cap / kBucketDiv - 1 - nbb, grid[1]);
    __syncthreads();
    const int64_t base = si.off / kBucketDiv;      // the system's buckets: cap / 4 from off / 4
    int key;
    if (d.alive[b]) {
        const bool big = b - si.off < si.nb;
        const SortGrid& g = grid[big ? 0 : 1];
        const float4 c = d.cen[b];
        int ix = grid_index(c.x, g.lo[0], g.inv_h, g.nx), iy = grid_index(c.y, g.lo[1], g.inv_h, g.ny),
            iz = grid_index(c.z, g.lo[2], g.inv_h, g.nz);
        if (iy & 1) ix = g.nx - 1 - ix;            // serpentine rows keep row ends together
        key = (int)(base + (big ? 0 : nbb) + ((int64_t)iz * g.ny + iy) * g.nx + ix);
    } else {
        key = (int)(base + si.cap / kBucketDiv - 1);   // dead and padding bodies last
    }
    d.ckey[b] = key;
    atomicAdd(&d.cstart[key], 1);
}

// exclusive prefix sum of the bucket counts (one block): each pass, every
// thread loads 16 consecutive counts at once (vector loads), the block scans
// the per-thread sums, and a carry runs from pass to pass
__global__ void __launch_bounds__(1024) k_sort_prefix(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlSortPrefix);
    constexpr int PER = 16;
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (d.ctl->status) return;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < d.ncell; base += 1024 * PER) {
        const int k0 = base + threadIdx.x * PER;
        int v[PER];
        if (k0 + PER <= d.ncell) {
            const int4* src = reinterpret_cast<const int4*>(d.cstart + k0);
#pragma unroll
            for (int u = 0; u < PER / 4; u++) {
                const int4 q = src[u];
                v[4 * u] = q.x; v[4 * u + 1] = q.y; v[4 * u + 2] = q.z; v[4 * u + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < PER; u++) v[u] = k0 + u < d.ncell ? d.cstart[k0 + u] : 0;
        }
        int sum = 0;
#pragma unroll
        for (int u = 0; u < PER; u++) sum += v[u];
        int x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = warp_sum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        int excl = carry + x - sum + (warp > 0 ? warp_sum[warp - 1] : 0);
        const int last = excl + sum;
#pragma unroll
        for (int u = 0; u < PER; u++) {
            if (k0 + u < d.ncell) d.ccursor[k0 + u] = excl;
            excl += v[u];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = last;
        __syncthreads();
    }
}

// scatter into the buckets (in whatever order the atomics give)
__global__ void __launch_bounds__(kBodyThreads) k_sort_scatter(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlSortScatter);
    if (d.ctl->status) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int key = d.ckey[b];
    const int pos = atomicAdd(&d.ccursor[key], 1);
    d.cscratch[pos] = make_int2((int)b, d.alive[b] ? key : -1);
}

// ascending ids within each bucket, so the order (and every sum taken in it)
// is the same on every run; each body's midpoint record goes beside it.
// A body's new place is its bucket's start plus the number of bucket mates
// with smaller ids.  The dead bodies' bucket (last of each system) keeps its
// order: it follows every live body, and dead bodies add nothing to any sum.
__global__ void __launch_bounds__(kBodyThreads) k_sort_order(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlSortOrder);
    if (d.ctl->status) return;
    const int64_t p = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int2 bk = d.cscratch[p];   // (body, bucket; -1 for a dead body)
    const int b = bk.x;
    int64_t out = p;
    if (bk.y >= 0) {
        const int e = d.ccursor[bk.y], s = e - d.cstart[bk.y];
        int rank = 0;
#pragma unroll 4
        for (int q = s; q < e; q++) rank += d.cscratch[q].x < b ? 1 : 0;
        out = s + rank;
    }
    d.csorted[out] = b;
    d.cen_sorted[out] = d.cen[b];
}

// box of c +- s over the live bodies of each 64-body tile of the sorted order
__global__ void __launch_bounds__(kSeg) k_tile_box(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlTileBox);
    if (d.ctl->status) return;
    const int64_t t = blockIdx.x;
    const int64_t pos = t * kSeg + threadIdx.x;
    const float4 c = d.cen_sorted[pos];
    const bool live = d.alive[d.csorted[pos]] != 0;
    float v[6];
    v[0] = live ? __fsub_rd(c.x, c.w) : 3.0e38f;
    v[1] = live ? __fsub_rd(c.y, c.w) : 3.0e38f;
    v[2] = live ? __fsub_rd(c.z, c.w) : 3.0e38f;
    v[3] = live ? __fadd_ru(c.x, c.w) : -3.0e38f;
    v[4] = live ? __fadd_ru(c.y, c.w) : -3.0e38f;
    v[5] = live ? __fadd_ru(c.z, c.w) : -3.0e38f;
    __shared__ float red[2][6];
    for (int k = 0; k < 6; k++) {
        float x = v[k];
        for (int o = 16; o >= 1; o >>= 1) {
            float y = __shfl_xor_sync(0xffffffffu, x, o);
            x = k < 3 ? fminf(x, y) : fmaxf(x, y);
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        d.tbox[6 * t + k] = k < 3 ? fminf(red[0][k], red[1][k]) : fmaxf(red[0][k], red[1][k]);
    }
}

__device__ __forceinline__ bool boxes_overlap(const float* a, const float* b) {
    return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

// The tile pairs whose boxes overlap, listed (one thread a tile pair, one
// atomic a warp); the list's order is the schedule's, and nothing after it
// depends on that order.
__global__ void __launch_bounds__(256) k_tile_cull(Dev d, const PairTile* __restrict__ tiles, int64_t ntiles) {
    OPAL_TIMELINE_SCOPE(kTlTileCull);
    if (d.ctl->status) return;
    const int lane = threadIdx.x & 31;
    for (int64_t it0 = (int64_t)blockIdx.x * blockDim.x; it0 < ntiles; it0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t it = it0 + threadIdx.x;
        bool ov = false;
        if (it < ntiles) {
            const PairTile tl = tiles[it];
            ov = boxes_overlap(d.tbox + 6 * (tl.i0 / kSeg), d.tbox + 6 * (tl.j0 / kSeg));
        }
        const unsigned m = __ballot_sync(0xffffffffu, ov);
        if (m == 0) continue;
        int base = 0;
        if (lane == 0) base = atomicAdd(&d.ctl->ntov, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ov) d.tov[base + __popc(m & ((1u << lane) - 1u))] = (int)it;
    }
}

// The listed tile pairs (A, B >= A): pairs that pass |c_j - c_i| < s_i + s_j
// go to a list for stage 2.  The tile list has a big tile as A (the big
// bodies sort first); pairs of two small bodies in it are dropped here.
__global__ void __launch_bounds__(kSeg) k_scan_tiles(Dev d, const PairTile* __restrict__ tiles) {
    OPAL_TIMELINE_SCOPE(kTlScanTiles);
    __shared__ float4 sj[kSeg];
    __shared__ int gj[kSeg];
    __shared__ unsigned smask[kSeg / 32][kSeg];
    if (d.ctl->status) return;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nov = d.ctl->ntov;
    for (int q = blockIdx.x; q < nov; q += gridDim.x) {
        {
            const PairTile tl = tiles[d.tov[q]];
            const int64_t pi = tl.i0 + threadIdx.x;
            const float4 ci = d.cen_sorted[pi];
            const int gi = d.csorted[pi];
            const int64_t big_end = d.sys[tl.sys].off + d.sys[tl.sys].nb;   // ids below are big bodies
            const bool ibig = gi < big_end;
            __syncthreads();
            sj[threadIdx.x] = d.cen_sorted[tl.j0 + threadIdx.x];
            gj[threadIdx.x] = d.csorted[tl.j0 + threadIdx.x];
            __syncthreads();
            const bool diag = tl.i0 == tl.j0;
            // pass 1: each warp's ballots of the tile pair, and their total; pass 2:
            // one atomic reserves the warp's room in the list, then every passing
            // lane writes its pair (one atomic per warp and tile pair, not per column)
            int cnt = 0;
#pragma unroll 4
            for (int jj = 0; jj < kSeg; jj++) {
                const float4 cj = sj[jj];
                float dx = cj.x - ci.x, dy = cj.y - ci.y, dz = cj.z - ci.z;
                float r2 = dx * dx + dy * dy + dz * dz;
                float Ts = ci.w + cj.w;
                // two small bodies never interact
                bool pass = (!diag || jj > (int)threadIdx.x) && (r2 < Ts * Ts) && (ibig || gj[jj] < big_end);
                const unsigned mask = __ballot_sync(0xffffffffu, pass);
                if (lane == 0) smask[warp][jj] = mask;
                cnt += __popc(mask);
            }
            if (cnt == 0) continue;                     // the same for the whole warp
            int base = 0;
            if (lane == 0) base = atomicAdd(&d.ctl->nnear, cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
            __syncwarp();
            const unsigned below = (1u << lane) - 1u;
            for (int jj = 0; jj < kSeg; jj++) {
                const unsigned mask = smask[warp][jj];
                if ((mask >> lane) & 1u) {
                    const int idx = base + __popc(mask & below);
                    const int b2 = gj[jj];
                    if (idx < d.near_cap) d.near[idx] = make_int2(min(gi, b2), max(gi, b2));
                }
                base += __popc(mask);
            }
        }
    }
}

// stage 2 on the stage-1 list, one thread per pair
__global__ void __launch_bounds__(256) k_chord(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlChord);
    if (d.ctl->status) return;
    const int nn = d.ctl->nnear;
    if (nn > d.near_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.ctl, kEoverflow, -4);
        return;
    }
    const float T = (float)d.p.dt;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x; base < nn; base += gridDim.x * blockDim.x) {
        const int k = base + threadIdx.x;
        bool pass = false;
        int2 pr = make_int2(0, 0);
        if (k < nn) {
            pr = d.near[k];
            pass = d.alive[pr.x] && d.alive[pr.y] && chord_bound_passes(d, pr.x, pr.y, T);
        }
        unsigned mask = __ballot_sync(0xffffffffu, pass);
        if (mask) {
            int leader = __ffs(mask) - 1;
            int b0 = 0;
            if (lane == leader) b0 = atomicAdd(&d.ctl->ncand, __popc(mask));
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (pass) {
                int idx = b0 + __popc(mask & ((1u << lane) - 1u));
                if (idx < d.cand_cap) d.cand[idx] = pr;
            }
        }
    }
}

// ---------------------------------------------------------------- stage 3
// Relative position and its first and second s-derivatives on the cubic
// Hermite path, s in [0, 1], T = dt (same operation order as the oracle).
__device__ __forceinline__ void hermite_rel(double s, double T, const double* d0, const double* u0,
                                            const double* d1, const double* u1, double* dd, double* dp,
                                            double* d2) {
    double s2 = s * s, s3 = s2 * s;
    double h00 = 2.0 * s3 - 3.0 * s2 + 1.0, h10 = s3 - 2.0 * s2 + s;
    double h01 = -2.0 * s3 + 3.0 * s2, h11 = s3 - s2;
    double p00 = 6.0 * s2 - 6.0 * s, p10 = 3.0 * s2 - 4.0 * s + 1.0;
    double p01 = -6.0 * s2 + 6.0 * s, p11 = 3.0 * s2 - 2.0 * s;
    double q00 = 12.0 * s - 6.0, q10 = 6.0 * s - 4.0, q01 = -12.0 * s + 6.0, q11 = 6.0 * s - 2.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dd[k] = h00 * d0[k] + h10 * T * u0[k] + h01 * d1[k] + h11 * T * u1[k];
        dp[k] = p00 * d0[k] + p10 * T * u0[k] + p01 * d1[k] + p11 * T * u1[k];
        d2[k] = q00 * d0[k] + q10 * T * u0[k] + q01 * d1[k] + q11 * T * u1[k];
    }
}

__device__ __forceinline__ double dot3p(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// The same path in FP32 for the root search: relative position and its
// first and second s-derivatives (T u folded into the tangents).
__device__ __forceinline__ void hermite_rel_f(float s, const float* d0, const float* tu0, const float* d1,
                                              const float* tu1, float* dd, float* dp, float* d2) {
    const float s2 = s * s, s3 = s2 * s;
    const float h00 = 2.0f * s3 - 3.0f * s2 + 1.0f, h10 = s3 - 2.0f * s2 + s;
    const float h01 = -2.0f * s3 + 3.0f * s2, h11 = s3 - s2;
    const float p00 = 6.0f * s2 - 6.0f * s, p10 = 3.0f * s2 - 4.0f * s + 1.0f;
    const float p01 = -6.0f * s2 + 6.0f * s, p11 = 3.0f * s2 - 2.0f * s;
    const float q00 = 12.0f * s - 6.0f, q10 = 6.0f * s - 4.0f, q01 = -12.0f * s + 6.0f, q11 = 6.0f * s - 2.0f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dd[k] = h00 * d0[k] + h10 * tu0[k] + h01 * d1[k] + h11 * tu1[k];
        dp[k] = p00 * d0[k] + p10 * tu0[k] + p01 * d1[k] + p11 * tu1[k];
        d2[k] = q00 * d0[k] + q10 * tu0[k] + q01 * d1[k] + q11 * tu1[k];
    }
}

// Stage 3, 16 lanes per candidate pair: lane k looks at interval k of the
// 16, and where g = d.d' changes sign from - to + on it, finds the root of g
// (the minimum of |d|^2) by Newton from the secant point, kept inside the
// bracket by bisection.  The bracket tests and the root search run in FP32
// (one warp's FP64 instruction takes the FP64 unit for many cycles, and the
// search is a long dependent chain).  At the root found, the path and its
// derivatives are taken in FP64 with the oracle's arithmetic, and the minimum
// is that of the local quadratic, |d|^2 - g^2 / g': a root off by ds leaves
// an error of order ds^3, and an FP32 root is off by about 1e-7 (the minimum
// then agrees with the oracle's to about 1e-13 relative, 1e-11 for near
// head-on passes).  A sign of g that FP32 gets wrong at an interval's end
// moves the bracket to the neighbouring interval, whose root is then that end.  The minimum over the lanes and the path's two ends is
// the sequential result (a minimum does not depend on the order its terms
// are visited in).
__device__ double interval_min2(double T, int k, const double* d0, const double* u0, const double* d1,
                                const double* u1) {
    float f0[3], f1[3], tu0[3], tu1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        f0[c] = (float)d0[c];
        f1[c] = (float)d1[c];
        tu0[c] = (float)(T * u0[c]);
        tu1[c] = (float)(T * u1[c]);
    }
    float dd[3], dp[3], d2[3];
    const float lo0 = k / 16.0f, hi0 = (k + 1) / 16.0f;
    hermite_rel_f(lo0, f0, tu0, f1, tu1, dd, dp, d2);
    const float ga = dd[0] * dp[0] + dd[1] * dp[1] + dd[2] * dp[2];
    hermite_rel_f(hi0, f0, tu0, f1, tu1, dd, dp, d2);
    const float gb = dd[0] * dp[0] + dd[1] * dp[1] + dd[2] * dp[2];
    if (!(ga < 0.0f && gb >= 0.0f)) return HUGE_VAL;
    float lo = lo0, hi = hi0;
    float s = lo + (hi - lo) * (ga / (ga - gb));
    if (!(s > lo && s < hi)) s = 0.5f * (lo + hi);
    for (int it = 0; it < 60; it++) {
        hermite_rel_f(s, f0, tu0, f1, tu1, dd, dp, d2);
        const float g = dd[0] * dp[0] + dd[1] * dp[1] + dd[2] * dp[2];
        const float gp = dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2] + dd[0] * d2[0] + dd[1] * d2[1] + dd[2] * d2[2];
        if (g < 0.0f) lo = s;
        else hi = s;
        float sn = s - g / gp;
        if (!(gp > 0.0f && sn > lo && sn < hi)) sn = 0.5f * (lo + hi);
        const float step = sn - s;
        s = sn;
        if (fabsf(step) <= 1e-7f || hi - lo <= 2e-7f) break;
    }
    // FP64 at the root found: |d|^2 less g^2 / g', the minimum of the local
    // quadratic (one Newton step's worth)
    double ddd[3], dpd[3], d2d[3];
    hermite_rel((double)s, T, d0, u0, d1, u1, ddd, dpd, d2d);
    const double g = dot3p(ddd, dpd), gp = dot3p(dpd, dpd) + dot3p(ddd, d2d);
    double D = dot3p(ddd, ddd);
    if (gp > 0.0) D -= g * g / gp;
    return fmax(D, 0.0);
}

__global__ void __launch_bounds__(256) k_confirm(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlConfirm);
    if (d.ctl->status) return;
    const int ncand = d.ctl->ncand;
    if (ncand > d.cand_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.ctl, kEoverflow, -1);
        return;
    }
    const double T = d.p.dt;
    const int lane = threadIdx.x & 31, sub = lane & 15;
    const unsigned half = 0xffffu << (lane & 16);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the two halves of a warp take two pairs; every lane runs every pass
    for (int64_t kk = 2 * warp; kk < ncand; kk += 2 * nwarp) {
        const int64_t k = kk + (lane >> 4);
        bool live = k < ncand;
        int2 pr = make_int2(0, 0);
        if (live) {
            pr = d.cand[k];
            live = d.alive[pr.x] && d.alive[pr.y];
        }
        double D = HUGE_VAL, rcij = 0.0;
        if (live) {
            const int i = pr.x, j = pr.y;
            double d0[3] = {d.x0[j] - d.x0[i], d.y0[j] - d.y0[i], d.z0[j] - d.z0[i]};
            double u0[3] = {d.vx0[j] - d.vx0[i], d.vy0[j] - d.vy0[i], d.vz0[j] - d.vz0[i]};
            double d1[3] = {d.x[j] - d.x[i], d.y[j] - d.y[i], d.z[j] - d.z[i]};
            double u1[3] = {d.vx[j] - d.vx[i], d.vy[j] - d.vy[i], d.vz[j] - d.vz[i]};
            rcij = fmax(d.rc[i], d.rc[j]);
            D = fmin(dot3p(d0, d0), dot3p(d1, d1));
            D = fmin(D, interval_min2(T, sub, d0, u0, d1, u1));
        }
#pragma unroll
        for (int o = 8; o >= 1; o >>= 1) D = fmin(D, __shfl_xor_sync(half, D, o));
        if (live && sub == 0 && D <= rcij * rcij) {
            int idx = atomicAdd(&d.ctl->nflag, 1);
            if (idx < d.flag_cap) {
                d.flag[idx] = pr;
                d.label[pr.x] = pr.x;   // both ends become members (their own union-find roots)
                d.label[pr.y] = pr.y;
            } else {
                set_status(d.ctl, kEoverflow, -2);
            }
        }
    }
}

// ---------------------------------------------------------------- groups
// Connected components of the flagged pairs, for any number of pairs:
//   k_confirm marks both ends of a flagged pair (label = its own index);
//   k_group_link joins the ends of every pair in a lock-free union-find that
//     always hooks the larger root under the smaller, so the root of a
//     component is its lowest body;
//   k_group_count points every member at its root and counts each group;
//   k_group_offsets (one block) scans the counts in body order, so groups
//     come in ascending root order, each with its range in the member list;
//   k_group_place puts every member into its group's range;
//   k_group_order sorts each range ascending (one block per group) and lists
//     the groups the small-group encounter kernel leaves to the large one.
constexpr int kUfSteps = 1 << 20;         // bound on any one union-find walk
constexpr int kGroupSortMax = 8192;       // members one block sorts in shared memory

// root of x, halving the path on the way; -1 if the walk runs past its bound
__device__ __forceinline__ int uf_root(int* parent, int x) {
    for (int it = 0; it < kUfSteps; it++) {
        const int p = __ldcg(&parent[x]);
        if (p == x) return x;
        const int gp = __ldcg(&parent[p]);
        if (gp != p) atomicCAS(&parent[x], p, gp);
        x = gp;
    }
    return -1;
}

__global__ void __launch_bounds__(256) k_group_link(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlGroupLink);
    if (d.ctl->status) return;
    const int nf = d.ctl->nflag;
    if (nf > d.flag_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(d.ctl, kEoverflow, -3);
        return;
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nf; p += gridDim.x * blockDim.x) {
        const int2 pr = d.flag[p];
        bool done = false;
        for (int it = 0; it < kUfSteps && !done; it++) {
            int ra = uf_root(d.label, pr.x), rb = uf_root(d.label, pr.y);
            if (ra < 0 || rb < 0) break;
            if (ra == rb) {
                done = true;
                break;
            }
            if (ra > rb) {
                const int t = ra;
                ra = rb;
                rb = t;
            }
            done = atomicCAS(&d.label[rb], rb, ra) == rb;   // the larger root goes under the smaller
        }
        if (!done) set_status(d.ctl, kEoverflow, -5);
    }
}

__global__ void __launch_bounds__(kBodyThreads) k_group_count(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlGroupCount);
    if (d.ctl->status || d.ctl->nflag == 0) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    if (__ldcg(&d.label[b]) < 0) return;
    const int r = uf_root(d.label, (int)b);
    if (r < 0) {
        set_status(d.ctl, kEoverflow, -5);
        return;
    }
    d.label[b] = r;
    atomicAdd(&d.gcount[r], 1);
}

// one block: exclusive scans, in body order, of the group sizes (member
// offsets) and of the root flags (group indices), 16 counts per thread a pass
__global__ void __launch_bounds__(1024) k_group_offsets(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlGroupOffsets);
    constexpr int PER = 16;
    __shared__ long long warp_sum[32];
    __shared__ long long carry;
    if (d.ctl->status || d.ctl->nflag == 0) return;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t N = d.ntot;
    for (int64_t base = 0; base < N; base += 1024 * PER) {
        const int64_t k0 = base + (int64_t)threadIdx.x * PER;
        int v[PER];
        if (k0 + PER <= N) {
            const int4* src = reinterpret_cast<const int4*>(d.gcount + k0);
#pragma unroll
            for (int u = 0; u < PER / 4; u++) {
                const int4 q = src[u];
                v[4 * u] = q.x; v[4 * u + 1] = q.y; v[4 * u + 2] = q.z; v[4 * u + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < PER; u++) v[u] = k0 + u < N ? d.gcount[k0 + u] : 0;
        }
        // low 32 bits: members; high 32 bits: groups (roots have a nonzero count)
        long long sum = 0;
#pragma unroll
        for (int u = 0; u < PER; u++) sum += (long long)v[u] + (v[u] > 0 ? (1LL << 32) : 0LL);
        long long x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            long long w = warp_sum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        long long excl = carry + x - sum + (warp > 0 ? warp_sum[warp - 1] : 0);
        const long long last = excl + sum;
#pragma unroll
        for (int u = 0; u < PER; u++) {
            if (v[u] > 0) {
                const int gi = (int)(excl >> 32), off = (int)(excl & 0xffffffffLL);
                d.gofs[k0 + u] = off;
                d.goff[gi] = off;
                d.gidx[k0 + u] = gi;
            }
            excl += (long long)v[u] + (v[u] > 0 ? (1LL << 32) : 0LL);
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = last;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int ng = (int)(carry >> 32), nm = (int)(carry & 0xffffffffLL);
        d.goff[ng] = nm;
        d.ctl->ngroups = ng;
        d.ctl->ninvolved = nm;
    }
}

__global__ void __launch_bounds__(kBodyThreads) k_group_place(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlGroupPlace);
    if (d.ctl->status || d.ctl->nflag == 0) return;
    const int64_t b = (int64_t)blockIdx.x * kBodyThreads + threadIdx.x;
    const int r = d.label[b];
    if (r >= 0) {
        // the count goes back to zero as the range fills, ready for the next step
        const int pos = d.gofs[r] + atomicSub(&d.gcount[r], 1) - 1;
        d.members[pos] = (int)b;
        // the mixed kick beside the encounter integrator leaves the members
        // out as sources (mass 0 in its float copy; k_kick_apply writes the
        // new copy with the mass), so the fix-up adds their new terms only
        if (d.overlap && d.p.precision == 1) d.kh[b].w = 0.0f;
    }
    // big members counted (the cost of patching the kick after the encounters)
    const SysInfo& si = d.sys[d.body_sys[(int64_t)blockIdx.x * kBodyThreads]];
    const unsigned bm = __ballot_sync(0xffffffffu, r >= 0 && b - si.off < si.nb);
    if ((threadIdx.x & 31) == 0 && bm) atomicAdd(&d.ctl->ninv_big, __popc(bm));
}

__global__ void __launch_bounds__(256) k_group_order(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlGroupOrder);
    __shared__ int v[kGroupSortMax];
    if (d.ctl->status || d.ctl->nflag == 0) return;
    const int ng = d.ctl->ngroups;
    for (int g = blockIdx.x; g < ng; g += gridDim.x) {
        const int m0 = d.goff[g], n = d.goff[g + 1] - m0;
        if (threadIdx.x == 0 && n > 64) {
            // the whole-GPU kernel's, one after another
            if (n <= d.hb.cap) d.ghuge[atomicAdd(&d.ctl->nhuge, 1)] = g;
            else set_status(d.ctl, kEoverflow, 2000000 + g);
        } else if (threadIdx.x == 0) {
            if (ng > kBsManyGroups) {
                // many groups: up to 16 members to the packed kernel's class lists, larger
                // ones straight to the lockstep kernels
                if (n <= 16) {
                    const int c = n <= 2 ? 0 : (n <= 4 ? 1 : (n <= 8 ? 2 : 3));
                    d.gcls[c * d.gcap + atomicAdd(&d.ctl->ncls[c], 1)] = g;
                } else {
                    const int q = atomicAdd(&d.ctl->nhard, 1);
                    if (q < d.gcap) d.ghard[q] = g;
                    else set_status(d.ctl, kEoverflow, -7);
                }
            } else if (n > 4) {
                d.glarge[atomicAdd(&d.ctl->nlarge, 1)] = g;
            }
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            d.undo[3 * (m0 + k) + 2] = -1.0;
            d.bsout[(int64_t)kBsOut * (m0 + k) + 8] = -1.0;   // no result yet (the BS kernels write one)
        }
        if (n <= 1) continue;
        if (n == 2) {
            if (threadIdx.x == 0) {
                const int a = d.members[m0], b = d.members[m0 + 1];
                if (a > b) {
                    d.members[m0] = b;
                    d.members[m0 + 1] = a;
                }
            }
            continue;
        }
        if (n > kGroupSortMax) {
            if (threadIdx.x == 0) set_status(d.ctl, kEoverflow, 2000000 + g);
            return;
        }
        int np2 = 1;
        while (np2 < n) np2 <<= 1;
        __syncthreads();
        for (int k = threadIdx.x; k < np2; k += blockDim.x) v[k] = k < n ? d.members[m0 + k] : 0x7fffffff;
        __syncthreads();
        for (int size = 2; size <= np2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int k = threadIdx.x; k < np2; k += blockDim.x) {
                    const int q = k ^ stride;
                    if (q > k) {
                        const bool up = (k & size) == 0;
                        const int x = v[k], y = v[q];
                        if ((x > y) == up) {
                            v[k] = y;
                            v[q] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int k = threadIdx.x; k < n; k += blockDim.x) d.members[m0 + k] = v[k];
    }
}

void launch_sort_bodies(const Dev& d, cudaStream_t s) {
    const unsigned nb = (unsigned)(d.ntot / kBodyThreads);
    k_sort_count<<<nb, kBodyThreads, 0, s>>>(d);
    prof_mark("scan: sort count");
    k_sort_prefix<<<1, 1024, 0, s>>>(d);
    prof_mark("scan: sort prefix");
    k_sort_scatter<<<nb, kBodyThreads, 0, s>>>(d);
    prof_mark("scan: sort scatter");
    k_sort_order<<<nb, kBodyThreads, 0, s>>>(d);
    prof_mark("scan: sort order");
}

void launch_scan(const Dev& d, const PairTile* tiles, int64_t ntiles, int grid, cudaStream_t s) {
    launch_sort_bodies(d, s);
    k_tile_box<<<(unsigned)(d.ntot / kSeg), kSeg, 0, s>>>(d);
    prof_mark("scan: tile boxes");
    const int64_t cb = (ntiles + 255) / 256;
    k_tile_cull<<<(unsigned)(cb < 152 * 8 ? cb : 152 * 8), 256, 0, s>>>(d, tiles, ntiles);
    prof_mark("scan: tile boxes culled");
    k_scan_tiles<<<grid, kSeg, 0, s>>>(d, tiles);
    prof_mark("scan: tile pairs");
    k_chord<<<152 * 4, 256, 0, s>>>(d);
    prof_mark("scan: chord bound");
}
void launch_confirm(const Dev& d, int grid, cudaStream_t s) {
    k_confirm<<<grid, 256, 0, s>>>(d);
    prof_mark("confirm (FP64)");
}

void launch_group(const Dev& d, int nsm, cudaStream_t s) {
    const unsigned nb = (unsigned)(d.ntot / kBodyThreads);
    k_group_link<<<nsm * 2, 256, 0, s>>>(d);
    prof_mark("group: link");
    k_group_count<<<nb, kBodyThreads, 0, s>>>(d);
    prof_mark("group: count");
    k_group_offsets<<<1, 1024, 0, s>>>(d);
    prof_mark("group: offsets");
    k_group_place<<<nb, kBodyThreads, 0, s>>>(d);
    prof_mark("group: place");
    k_group_order<<<nsm * 2, 256, 0, s>>>(d);
    prof_mark("group: order");
}

}  // namespace opal
