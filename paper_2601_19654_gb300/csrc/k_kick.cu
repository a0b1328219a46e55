// The kick's pair kernel: a_i = sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
// (Sec. 3.1, force block, LOOP 2, with the changeover weight K of the hybrid
// integrator).  G is applied when the partials are reduced.
//
// Work is a list of items (i-tile of 128 bodies x a j-range of the same
// system) that the blocks of a persistent grid take from a queue; each item
// writes its partial sums to its own row of a buffer that k_kick_rows
// reduces in a fixed order, so results do not depend on the schedule.
// j-bodies are staged through shared memory and read by every thread of the
// block (broadcast).  Pairs closer than 2 (rc_i + rc_max) take a slow path
// that handles the changeover, the self pair and exact coincidence; all
// other pairs take the plain Newtonian fast path.
//
// Mixed form: FP32 separations of the hi parts of a hi/lo float split of the
// FP64 positions (the lo parts are added on the slow path), MUFU rsqrt, FP32
// sums over each 256-body j-tile (the even and the odd j in the two lanes of
// a packed accumulator), written to the tile's partial row as the float pair
// (hi, lo) that TwoSum makes of the two lanes, which holds their sum
// exactly; k_kick_rows adds a body's rows in float-float arithmetic and
// converts the total to FP64.  FP64 form: the same in doubles, rows summed
// in FP64.
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
__device__ __noinline__ float4 slow_pair_f(float4 li, float4 lj, float dx, float dy, float dz, float mj,
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

// ---------------------------------------------------------------------------
// Staging, before each mixed kick: the float copies of the kick's bodies in
// the scan's spatial order (position p holds body csorted[p]) as separate
// arrays, so that a j-tile is a contiguous run of records, and for every
// 128-position tile the box of its live positions and its largest near
// threshold (2 (rc + rc_max))^2, so that the kick reads a tile's box instead
// of reducing it (also for every 256 positions, the j-tiles and the larger
// i-tiles).  Parked bodies (dead or padding, at kFar) stay out of the boxes;
// an empty tile gets lo > hi.
__global__ void __launch_bounds__(2 * kKickBox) k_kick_stage(Dev d) {
    OPAL_TIMELINE_SCOPE(kTlKickStage);
    if (d.gated && !d.ctl->reprime) return;   // the re-evaluation after a removal, with none
    if (d.ctl->status) return;
    constexpr int W = 2 * kKickBox / 32;      // warps of the block (8)
    __shared__ int red[7][W];
    const int64_t p = (int64_t)blockIdx.x * 2 * kKickBox + threadIdx.x;   // grid: ntot / 256 blocks
    const int b = d.csorted[p];
    const float4 h = d.kh[b];
    const float rc = d.rcf[b];
    d.ks_x[p] = h.x;
    d.ks_y[p] = h.y;
    d.ks_z[p] = h.z;
    d.ks_m[p] = h.w;
    d.ks_lo[p] = d.kl[b];
    d.ks_rc[p] = rc;
    const bool live = h.x < 0.5f * kFar;
    const float t = 2.0f * (rc + d.rcmax[d.body_sys[b]]);
    const float thr = fmaxf(t * t, 1e-30f);
    const float c[3] = {h.x, h.y, h.z};
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int lo = __reduce_min_sync(0xffffffffu, live ? ford(c[k]) : 0x7fffffff);
        const int hi = __reduce_max_sync(0xffffffffu, live ? ford(c[k]) : (int)0x80000000);
        if (lane == 0) {
            red[k][wq] = lo;
            red[3 + k][wq] = hi;
        }
    }
    // thresholds are >= 0: their bits order as their values
    const int tm = __reduce_max_sync(0xffffffffu, live ? __float_as_int(thr) : 0);
    if (lane == 0) red[6][wq] = tm;
    __syncthreads();
    // thread 0: the first 128 positions, thread 1: the second, thread 2: all 256
    if (threadIdx.x < 3) {
        const int w0 = threadIdx.x == 1 ? W / 2 : 0, w1 = threadIdx.x == 0 ? W / 2 : W;
        int v[7];
        for (int k = 0; k < 7; k++) {
            v[k] = red[k][w0];
            for (int w = w0 + 1; w < w1; w++) v[k] = (k < 3) ? min(v[k], red[k][w]) : max(v[k], red[k][w]);
        }
        const float4 lo = make_float4(fordinv(v[0]), fordinv(v[1]), fordinv(v[2]), __int_as_float(v[6]));
        const float4 hi = make_float4(fordinv(v[3]), fordinv(v[4]), fordinv(v[5]), 0.0f);
        float4* o = threadIdx.x < 2 ? d.kbox + 2 * (2 * (int64_t)blockIdx.x + threadIdx.x)
                                    : d.kbox2 + 2 * (int64_t)blockIdx.x;
        o[0] = lo;
        o[1] = hi;
    }
}

// Far j-tile (no pair can be near): plain Newtonian terms in packed FP32
// pairs.  Each 16-byte shared load brings four j records' x (or y, z, m);
// each packed instruction takes two j at once against one i, the two lanes
// of the packed accumulators holding the even and the odd j.  The arithmetic
// of each lane is the scalar fast path's: x_j + (-x_i) is x_j - x_i exactly.
template <int NI>
__device__ __forceinline__ void far_tile(const float* sx, const float* sy, const float* sz, const float* sm,
                                         const float2 (&nx)[NI], const float2 (&ny)[NI], const float2 (&nz)[NI],
                                         float2 (&ax)[NI], float2 (&ay)[NI], float2 (&az)[NI]) {
    const float4* px = reinterpret_cast<const float4*>(sx);
    const float4* py = reinterpret_cast<const float4*>(sy);
    const float4* pz = reinterpret_cast<const float4*>(sz);
    const float4* pm = reinterpret_cast<const float4*>(sm);
#pragma unroll 4
    for (int jq = 0; jq < kJTile / 4; jq++) {
        const float4 x4 = px[jq], y4 = py[jq], z4 = pz[jq], m4 = pm[jq];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float2 xj = h ? make_float2(x4.z, x4.w) : make_float2(x4.x, x4.y);
            const float2 yj = h ? make_float2(y4.z, y4.w) : make_float2(y4.x, y4.y);
            const float2 zj = h ? make_float2(z4.z, z4.w) : make_float2(z4.x, z4.y);
            const float2 mj = h ? make_float2(m4.z, m4.w) : make_float2(m4.x, m4.y);
#pragma unroll
            for (int q = 0; q < NI; q++) {
                const float2 dx = __fadd2_rn(xj, nx[q]), dy = __fadd2_rn(yj, ny[q]), dz = __fadd2_rn(zj, nz[q]);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                const float2 sv = __fmul2_rn(__fmul2_rn(mj, ri), __fmul2_rn(ri, ri));
                ax[q] = __ffma2_rn(sv, dx, ax[q]);
                ay[q] = __ffma2_rn(sv, dy, ay[q]);
                az[q] = __ffma2_rn(sv, dz, az[q]);
            }
        }
    }
}

// Near j-tile: the packed loop, with every pair closer than the i-body's
// threshold left out (its term set to zero) and its j noted in the lane's
// own list in shared memory; then the lanes take the slow path (lo parts,
// changeover) for their listed pairs side by side, each adding its own in
// j order, so the warp runs as many slow-path rounds as its longest list
// holds rather than one for every j where any lane has a near pair.  A list
// that could overflow is worked off first (a warp-uniform test).  The
// i-body's lo parts, rc and threshold are read here (near tiles are few).
constexpr int kNearList = 32;   // listed near pairs per lane and i-body before a flush

template <int T, int NI>
__device__ __forceinline__ void near_flush(const float* sx, const float* sy, const float* sz, const float* sm,
                                           const float4* sl, const float* src, const unsigned char* lst,
                                           const int (&cnt)[NI], const float2 (&nx)[NI], const float2 (&ny)[NI],
                                           const float2 (&nz)[NI], const float4 (&li)[NI], const float (&rci)[NI],
                                           int form, float2 (&ax)[NI], float2 (&ay)[NI], float2 (&az)[NI]) {
#pragma unroll
    for (int q = 0; q < NI; q++) {
        int most = cnt[q];
        for (int o = 16; o >= 1; o >>= 1) most = max(most, __shfl_xor_sync(0xffffffffu, most, o));
        for (int k = 0; k < most; k++) {
            if (k < cnt[q]) {
                const int jj = lst[(k * NI + q) * T + threadIdx.x];
                const float4 r = slow_pair_f(li[q], sl[jj], sx[jj] + nx[q].x, sy[jj] + ny[q].x, sz[jj] + nz[q].x,
                                             sm[jj], rci[q], src[jj], form);
                ax[q].x = fmaf(r.x, r.y, ax[q].x);
                ay[q].x = fmaf(r.x, r.z, ay[q].x);
                az[q].x = fmaf(r.x, r.w, az[q].x);
            }
        }
    }
}

template <int T, int NI>
__device__ __forceinline__ void near_tile(const Dev& d, int64_t i0, float rcm, const float* sx, const float* sy,
                                          const float* sz, const float* sm, const float4* sl, const float* src,
                                          unsigned char* lst, const float2 (&nx)[NI], const float2 (&ny)[NI],
                                          const float2 (&nz)[NI], int form, float2 (&ax)[NI], float2 (&ay)[NI],
                                          float2 (&az)[NI]) {
    float4 li[NI];
    float rci[NI], thr[NI];
    int cnt[NI];
#pragma unroll
    for (int q = 0; q < NI; q++) {
        const int64_t p = i0 + q * T + threadIdx.x;
        li[q] = d.ks_lo[p];
        rci[q] = d.ks_rc[p];
        const float t = 2.0f * (rci[q] + rcm);
        thr[q] = fmaxf(t * t, 1e-30f);
        cnt[q] = 0;
    }
    const float4* px = reinterpret_cast<const float4*>(sx);
    const float4* py = reinterpret_cast<const float4*>(sy);
    const float4* pz = reinterpret_cast<const float4*>(sz);
    const float4* pm = reinterpret_cast<const float4*>(sm);
#pragma unroll 1
    for (int jq = 0; jq < kJTile / 4; jq++) {
        // room for the four pairs of this quad in every lane's list, or work it off
        bool full = false;
#pragma unroll
        for (int q = 0; q < NI; q++) full |= cnt[q] > kNearList - 4;
        if (__any_sync(0xffffffffu, full)) {
            near_flush<T, NI>(sx, sy, sz, sm, sl, src, lst, cnt, nx, ny, nz, li, rci, form, ax, ay, az);
#pragma unroll
            for (int q = 0; q < NI; q++) cnt[q] = 0;
        }
        const float4 x4 = px[jq], y4 = py[jq], z4 = pz[jq], m4 = pm[jq];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float2 xj = h ? make_float2(x4.z, x4.w) : make_float2(x4.x, x4.y);
            const float2 yj = h ? make_float2(y4.z, y4.w) : make_float2(y4.x, y4.y);
            const float2 zj = h ? make_float2(z4.z, z4.w) : make_float2(z4.x, z4.y);
            const float2 mj = h ? make_float2(m4.z, m4.w) : make_float2(m4.x, m4.y);
#pragma unroll
            for (int q = 0; q < NI; q++) {
                const float2 dx = __fadd2_rn(xj, nx[q]), dy = __fadd2_rn(yj, ny[q]), dz = __fadd2_rn(zj, nz[q]);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                float2 sv = __fmul2_rn(__fmul2_rn(mj, ri), __fmul2_rn(ri, ri));
                const int j = 4 * jq + 2 * h;
                if (r2.x < thr[q]) {
                    sv.x = 0.0f;
                    lst[(cnt[q]++ * NI + q) * T + threadIdx.x] = (unsigned char)j;
                }
                if (r2.y < thr[q]) {
                    sv.y = 0.0f;
                    lst[(cnt[q]++ * NI + q) * T + threadIdx.x] = (unsigned char)(j + 1);
                }
                ax[q] = __ffma2_rn(sv, dx, ax[q]);
                ay[q] = __ffma2_rn(sv, dy, ay[q]);
                az[q] = __ffma2_rn(sv, dz, az[q]);
            }
        }
    }
    near_flush<T, NI>(sx, sy, sz, sm, sl, src, lst, cnt, nx, ny, nz, li, rci, form, ax, ay, az);
}

// Items index the system's bodies in the order the encounter scan sorted
// them (cells of the path midpoints, so a 128-body tile is compact); the
// staging kernel has copied them there.  An item is one j-tile of 256
// sources, staged in shared memory once, against a run of i-tiles of
// T x NI bodies (every istep-th position: a run's tiles are spread over the
// system, so that the few near ones fall into different items); each thread
// takes NI i-bodies of each i-tile, and the next i-tile's positions and box
// are loaded while the current one runs.  An
// i-tile whose box is farther from the j-tile's box than the i-tile's
// largest threshold allows cannot hold a near pair and runs the packed loop
// with no per-pair test.  Records past the item's j-range are parked (kFar,
// zero mass): they add exact zeros.  Each (i-tile, j-tile) sum goes to the
// j-tile's partial row, at the i-body's sorted position; k_kick_rows adds the
// rows in order.
template <int T, int NI, int MINB>
__global__ void __launch_bounds__(T, MINB) k_kick_mixed(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    OPAL_TIMELINE_SCOPE(kTlKick);
    if (d.gated && !d.ctl->reprime) return;   // the re-evaluation after a removal, with none
    constexpr int JPT = kJTile / T;           // j records each thread stages (2 or 4)
    constexpr int IT = T * NI;                // bodies of an i-tile: 128 or 256, one staged box
    static_assert(JPT == 2 || JPT == 4, "the kick stages 2 or 4 records a thread");
    static_assert(IT == kKickBox || IT == 2 * kKickBox, "an i-tile is one staged box");
    const float4* ibox = IT == kKickBox ? d.kbox : d.kbox2;
    __shared__ __align__(16) float sx[kJTile], sy[kJTile], sz[kJTile], sm[kJTile];
    __shared__ float4 sl[kJTile];     // lo parts and 4 rc^2 of the j-tile (the near path's)
    __shared__ float src[kJTile];
    __shared__ KickItem s_w;          // the block's item
    __shared__ float s_jbox[6];       // its j-tile's box (lo xyz, hi xyz)
    __shared__ unsigned char s_near[kNearList * NI * T];   // near pairs' j, per lane and i-body
    if (d.ctl->status) return;
    const int form = d.p.changeover;
    for (;;) {
        // items are taken in list order (largest first) by whichever block is free
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t it = atomicAdd(&d.ctl->kick_next, 1);
            s_w.sys = -1;
            if (it < nitems) s_w = items[it];
        }
        __syncthreads();
        if (s_w.sys < 0) break;
        const KickItem w = s_w;
        const int nj = (int)(w.j1 - w.j0);
        const float rcm = d.rcmax[w.sys];
        // stage the j-tile: contiguous records, past nj parked
        {
            const int k0 = threadIdx.x * JPT;
            float vx[JPT], vy[JPT], vz[JPT], vm[JPT];
            if (k0 + JPT <= nj) {
                if (JPT == 2) {
                    const float2 a = *reinterpret_cast<const float2*>(d.ks_x + w.j0 + k0);
                    const float2 b = *reinterpret_cast<const float2*>(d.ks_y + w.j0 + k0);
                    const float2 c = *reinterpret_cast<const float2*>(d.ks_z + w.j0 + k0);
                    const float2 e = *reinterpret_cast<const float2*>(d.ks_m + w.j0 + k0);
                    vx[0] = a.x; vx[1] = a.y; vy[0] = b.x; vy[1] = b.y;
                    vz[0] = c.x; vz[1] = c.y; vm[0] = e.x; vm[1] = e.y;
                } else {
                    const float4 a = *reinterpret_cast<const float4*>(d.ks_x + w.j0 + k0);
                    const float4 b = *reinterpret_cast<const float4*>(d.ks_y + w.j0 + k0);
                    const float4 c = *reinterpret_cast<const float4*>(d.ks_z + w.j0 + k0);
                    const float4 e = *reinterpret_cast<const float4*>(d.ks_m + w.j0 + k0);
                    vx[0] = a.x; vx[1] = a.y; vx[JPT - 2] = a.z; vx[JPT - 1] = a.w;
                    vy[0] = b.x; vy[1] = b.y; vy[JPT - 2] = b.z; vy[JPT - 1] = b.w;
                    vz[0] = c.x; vz[1] = c.y; vz[JPT - 2] = c.z; vz[JPT - 1] = c.w;
                    vm[0] = e.x; vm[1] = e.y; vm[JPT - 2] = e.z; vm[JPT - 1] = e.w;
                }
            } else {
#pragma unroll
                for (int u = 0; u < JPT; u++) {
                    const bool in = k0 + u < nj;
                    vx[u] = in ? d.ks_x[w.j0 + k0 + u] : kFar;
                    vy[u] = in ? d.ks_y[w.j0 + k0 + u] : kFar;
                    vz[u] = in ? d.ks_z[w.j0 + k0 + u] : kFar;
                    vm[u] = in ? d.ks_m[w.j0 + k0 + u] : 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < JPT; u++) {
                sx[k0 + u] = vx[u];
                sy[k0 + u] = vy[u];
                sz[k0 + u] = vz[u];
                sm[k0 + u] = vm[u];
                sl[k0 + u] = k0 + u < nj ? d.ks_lo[w.j0 + k0 + u] : make_float4(0.0f, 0.0f, 0.0f, 1e-30f);
                src[k0 + u] = k0 + u < nj ? d.ks_rc[w.j0 + k0 + u] : 0.0f;
            }
            if (threadIdx.x == 0) {
                // the j-tile's box: its whole 256 positions (any records past nj
                // are padding or small bodies, and a larger box only sends more
                // i-tiles to the near path)
                const float4 lo = d.kbox2[2 * (w.j0 / kJTile)], hi = d.kbox2[2 * (w.j0 / kJTile) + 1];
                s_jbox[0] = lo.x; s_jbox[1] = lo.y; s_jbox[2] = lo.z;
                s_jbox[3] = hi.x; s_jbox[4] = hi.y; s_jbox[5] = hi.z;
            }
        }
        __syncthreads();
        const SysInfo si = d.sys[w.sys];
        const int64_t base = si.slot0 + (int64_t)w.chunk * si.cap - si.off;
        // the first i-tile's positions and box
        float px[NI], py[NI], pz[NI];
        float4 pb[2];
#pragma unroll
        for (int q = 0; q < NI; q++) {
            const int64_t p = w.i0 + q * T + threadIdx.x;
            px[q] = d.ks_x[p];
            py[q] = d.ks_y[p];
            pz[q] = d.ks_z[p];
        }
        pb[0] = ibox[2 * (w.i0 / IT)];
        pb[1] = ibox[2 * (w.i0 / IT) + 1];
        for (int64_t ib = w.i0; ib < w.i1; ib += w.istep) {
            float2 nx[NI], ny[NI], nz[NI];
#pragma unroll
            for (int q = 0; q < NI; q++) {
                nx[q] = make_float2(-px[q], -px[q]);
                ny[q] = make_float2(-py[q], -py[q]);
                nz[q] = make_float2(-pz[q], -pz[q]);
            }
            // near test of this i-tile against the j-tile (block-uniform)
            bool near;
            {
                const float lo[3] = {pb[0].x, pb[0].y, pb[0].z}, hi[3] = {pb[1].x, pb[1].y, pb[1].z};
                float g2 = 0.0f;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float g = fmaxf(0.0f, fmaxf(s_jbox[k] - hi[k], lo[k] - s_jbox[3 + k]));
                    g2 = fmaf(g, g, g2);
                }
                near = g2 < pb[0].w * 1.001f;
            }
            // the next i-tile's positions and box, in flight during this one
            const int64_t nb0 = ib + w.istep < w.i1 ? ib + w.istep : ib;
#pragma unroll
            for (int q = 0; q < NI; q++) {
                const int64_t p = nb0 + q * T + threadIdx.x;
                px[q] = d.ks_x[p];
                py[q] = d.ks_y[p];
                pz[q] = d.ks_z[p];
            }
            pb[0] = ibox[2 * (nb0 / IT)];
            pb[1] = ibox[2 * (nb0 / IT) + 1];
            float2 ax[NI], ay[NI], az[NI];
#pragma unroll
            for (int q = 0; q < NI; q++) ax[q] = ay[q] = az[q] = make_float2(0.0f, 0.0f);
            if (near) near_tile<T, NI>(d, ib, rcm, sx, sy, sz, sm, sl, src, s_near, nx, ny, nz, form, ax, ay, az);
            else far_tile<NI>(sx, sy, sz, sm, nx, ny, nz, ax, ay, az);
            // partial rows by sorted position (coalesced), each the exact float
            // pair of the two lanes' sums; k_kick_rows sums them by position
#pragma unroll
            for (int q = 0; q < NI; q++) {
                const int64_t slot = base + ib + q * T + threadIdx.x;
                reinterpret_cast<float2*>(d.pacc_x)[slot] = two_sum(ax[q].x, ax[q].y);
                reinterpret_cast<float2*>(d.pacc_y)[slot] = two_sum(ay[q].x, ay[q].y);
                reinterpret_cast<float2*>(d.pacc_z)[slot] = two_sum(az[q].x, az[q].y);
            }
        }
    }
    queue_done(d);
}

template <int T>
__global__ void __launch_bounds__(T) k_kick_fp64(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    OPAL_TIMELINE_SCOPE(kTlKick);
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
        for (int64_t ib = w.i0; ib < w.i1; ib += w.istep) {
        const int64_t i = ib + threadIdx.x;
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
    }
    queue_done(d);
}

// ---------------------------------------------------------------------------
// After the encounter integrator.  k_kick_apply puts each member's BS result
// into the state, keeping the old float copies and position.  When the kick
// ran beside the BS (overlap), on the state after the drift, its partial rows
// leave the group members out as sources (k_group_place set their mass to 0
// in the kick's float copy; overlap runs in the mixed form only), and
// k_kick_fix then
//   - recomputes the full row of each member at its new place, in kFixParts
//     runs of the sources (one block a run; k_close adds them in order),
//   - adds the members' new terms to every other body's row,
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
    OPAL_TIMELINE_SCOPE(kTlApply);
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
        if (o[6] != d.m[g]) d.hcb[g] = cbrt(o[6] / (3.0 * d.M0s[s]));   // a merger changed the mass
        d.m[g] = o[6];
        d.R[g] = o[7];
        const int al = (int)o[8];
        d.alive[g] = al;
        if (al) kick_floats(d, g, o[0], o[1], o[2], o[6], d.rc[g]);
        else park_floats(d, g);
    }
}

constexpr int kFixThreads = kBodyThreads;

__global__ void __launch_bounds__(kFixThreads) k_kick_fix(Dev d, int nbody_blocks) {
    OPAL_TIMELINE_SCOPE(kTlFix);
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
            system_total(d, d.pP_close, d.sys[s], s, d.pcnt + d.nsys, d.Ptot + 3 * (d.nsys + s),
                         d.Pjump + 3 * (d.nsys + s));
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
                // the kick left the members out as sources: their new terms
                // only, two members a packed instruction in the kick's far-path
                // arithmetic; when either pair is nearer than the threshold,
                // both take term_f, each in its own lane
                const float2 nx2 = make_float2(-hi.x, -hi.x), ny2 = make_float2(-hi.y, -hi.y),
                             nz2 = make_float2(-hi.z, -hi.z);
                float2 tx2 = make_float2(0.0f, 0.0f), ty2 = tx2, tz2 = tx2;
                int q = 0;
                for (; q + 1 < n; q += 2) {
                    const float4 a = snh[q], c = snh[q + 1];
                    const float2 dx = __fadd2_rn(make_float2(a.x, c.x), nx2), dy = __fadd2_rn(make_float2(a.y, c.y), ny2),
                                 dz = __fadd2_rn(make_float2(a.z, c.z), nz2);
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                    if (r2.x < thrf || r2.y < thrf) {
                        const float3 ta = term_f(hi, li, rci, thrf, a, snl[q], snr[q], form);
                        const float3 tc = term_f(hi, li, rci, thrf, c, snl[q + 1], snr[q + 1], form);
                        tx2.x += ta.x; ty2.x += ta.y; tz2.x += ta.z;
                        tx2.y += tc.x; ty2.y += tc.y; tz2.y += tc.z;
                    } else {
                        const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                        const float2 sv = __fmul2_rn(__fmul2_rn(make_float2(a.w, c.w), ri), __fmul2_rn(ri, ri));
                        tx2 = __ffma2_rn(sv, dx, tx2);
                        ty2 = __ffma2_rn(sv, dy, ty2);
                        tz2 = __ffma2_rn(sv, dz, tz2);
                    }
                }
                if (q < n) {
                    const float3 t = term_f(hi, li, rci, thrf, snh[q], snl[q], snr[q], form);
                    tx2.x += t.x; ty2.x += t.y; tz2.x += t.z;
                }
                fold(hx, lx, tx2.x);
                fold(hx, lx, tx2.y);
                fold(hy, ly, ty2.x);
                fold(hy, ly, ty2.y);
                fold(hz, lz, tz2.x);
                fold(hz, lz, tz2.y);
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
    // member rows, a block per (member, part) task at a time: part q takes
    // the q-th of kFixParts runs of the sources and its sum goes to part q
    if (!d.overlap) return;
    const int first = nbody_blocks * kFixParts;
    for (int task = (int)blockIdx.x - first; task < nm * kFixParts; task += (int)gridDim.x - first) {
        const int k = task / kFixParts, part = task % kFixParts;
        const int g = d.members[k];
        const int s = d.body_sys[g];
        const SysInfo si = d.sys[s];
        const int64_t span = (si.nb + kFixParts - 1) / kFixParts;
        const int64_t jlo = si.off + part * span;
        const int64_t jhi = si.off + (si.nb < (part + 1) * span ? si.nb : (part + 1) * span);
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
                // float sums of 8 terms at a time, folded into hi/lo pairs
                float hx = 0.0f, hy = 0.0f, hz = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
                const float2 nx2 = make_float2(-hi.x, -hi.x), ny2 = make_float2(-hi.y, -hi.y),
                             nz2 = make_float2(-hi.z, -hi.z);
                const int64_t jend = jhi;   // sources: this part's run of the big bodies
                for (int64_t j0 = jlo + threadIdx.x; j0 < jend; j0 += 8 * kFixThreads) {
                    // eight records loaded together (their latencies overlap); lo parts
                    // and rc only for the rare pair that takes the slow path
                    float4 hj[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int64_t j = j0 + (int64_t)u * kFixThreads;
                        hj[u] = (j < jend && j != g) ? d.kh[j] : make_float4(kFar, kFar, kFar, 0.0f);
                    }
                    // two sources a packed instruction (the kick's far-path
                    // arithmetic); a pair of sources with either one near takes
                    // the scalar path, each in its own lane
                    float2 tx2 = make_float2(0.0f, 0.0f), ty2 = tx2, tz2 = tx2;
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const float2 dx = __fadd2_rn(make_float2(hj[u].x, hj[u + 1].x), nx2),
                                     dy = __fadd2_rn(make_float2(hj[u].y, hj[u + 1].y), ny2),
                                     dz = __fadd2_rn(make_float2(hj[u].z, hj[u + 1].z), nz2);
                        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                        if (r2.x < thrf || r2.y < thrf) {
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const int64_t j = j0 + (int64_t)(u + h) * kFixThreads;
                                const float4 hh = hj[u + h];
                                float ex = hh.x - hi.x, ey = hh.y - hi.y, ez = hh.z - hi.z;
                                const float rs = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                                float sv;
                                if (rs < thrf) {
                                    const float4 r = slow_pair_f(li, d.kl[j], ex, ey, ez, hh.w, rci, d.rcf[j], form);
                                    sv = r.x;
                                    ex = r.y;
                                    ey = r.z;
                                    ez = r.w;
                                } else {
                                    const float ri = rsqrt_approx(rs);
                                    sv = (hh.w * ri) * (ri * ri);
                                }
                                if (h == 0) {
                                    tx2.x += sv * ex; ty2.x += sv * ey; tz2.x += sv * ez;
                                } else {
                                    tx2.y += sv * ex; ty2.y += sv * ey; tz2.y += sv * ez;
                                }
                            }
                        } else {
                            const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                            const float2 sv = __fmul2_rn(__fmul2_rn(make_float2(hj[u].w, hj[u + 1].w), ri),
                                                         __fmul2_rn(ri, ri));
                            tx2 = __ffma2_rn(sv, dx, tx2);
                            ty2 = __ffma2_rn(sv, dy, ty2);
                            tz2 = __ffma2_rn(sv, dz, tz2);
                        }
                    }
                    fold(hx, lx, tx2.x);
                    fold(hx, lx, tx2.y);
                    fold(hy, ly, ty2.x);
                    fold(hy, ly, ty2.y);
                    fold(hz, lz, tz2.x);
                    fold(hz, lz, tz2.y);
                }
                ax = (double)hx + (double)lx;
                ay = (double)hy + (double)ly;
                az = (double)hz + (double)lz;
            } else for (int64_t j = jlo + threadIdx.x; j < jhi; j += kFixThreads) {
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
            const int64_t o = (int64_t)part * d.ntot + g;
            d.cfx[o] = red[0][0];
            d.cfy[o] = red[1][0];
            d.cfz[o] = red[2][0];
        }
    }
}

void launch_bs_apply(const Dev& d, int nsm, cudaStream_t s) {
    k_kick_apply<<<nsm, 256, 0, s>>>(d);
    prof_mark("apply BS results");
}

void launch_kick_fix(const Dev& d, int nsm, cudaStream_t s) {
    const int nb = (int)(d.ntot / kFixThreads);
    k_kick_fix<<<nb * kFixParts + 4 * nsm, kFixThreads, 0, s>>>(d, nb);
    prof_mark("kick fix: member rows and corrections");
}

// Kick variants the autotuner picks from: (threads, i-bodies per thread,
// minimum resident blocks); an item's i-tile is threads x i-bodies (128 or
// 256 bodies, a divisor of the system padding).
struct KickVariant {
    const char* name;
    int threads;
    int ni;           // i-bodies per thread: an item's i-tile is threads x ni bodies
    bool jmajor;      // items: a j-tile against a run of i-tiles (else an i-tile against a j-chunk)
    void (*launch)(const Dev&, const KickItem*, int64_t, int, cudaStream_t);
    int (*occupancy)();
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
    {"mixed t128 i1", 128, 1, true, launch_mixed<128, 1, 7>, occ_mixed<128, 1, 7>},
    {"mixed t128 i1 6", 128, 1, true, launch_mixed<128, 1, 6>, occ_mixed<128, 1, 6>},
    {"mixed t128 i1 8", 128, 1, true, launch_mixed<128, 1, 8>, occ_mixed<128, 1, 8>},
    {"mixed t64 i2", 64, 2, true, launch_mixed<64, 2, 8>, occ_mixed<64, 2, 8>},
    {"mixed t128 i2", 128, 2, true, launch_mixed<128, 2, 5>, occ_mixed<128, 2, 5>},
};
static const KickVariant kFp64[] = {
    {"fp64 t128", 128, 1, false, launch_fp64<128>, occ_fp64<128>},
};

int kick_num_variants(int precision) {
    return precision == 1 ? (int)(sizeof(kMixed) / sizeof(kMixed[0])) : (int)(sizeof(kFp64) / sizeof(kFp64[0]));
}
const char* kick_variant_name(int precision, int v) { return precision == 1 ? kMixed[v].name : kFp64[v].name; }
bool kick_jmajor(int precision, int v) { return precision == 1 ? kMixed[v].jmajor : kFp64[v].jmajor; }
int kick_itile(int precision, int v) {
    const KickVariant& k = precision == 1 ? kMixed[v] : kFp64[v];
    return k.threads * k.ni;
}
int kick_occupancy(int precision, int v) { return precision == 1 ? kMixed[v].occupancy() : kFp64[v].occupancy(); }
int kick_threads(int precision, int v) { return precision == 1 ? kMixed[v].threads : kFp64[v].threads; }
void launch_kick(const Dev& d, const KickItem* items, int64_t nitems, int grid, int precision, int v,
                 cudaStream_t s) {
    if (precision == 1) kMixed[v].launch(d, items, nitems, grid, s);
    else kFp64[v].launch(d, items, nitems, grid, s);
    prof_mark("kick");
}

void launch_kick_stage(const Dev& d, int precision, cudaStream_t s) {
    if (precision != 1) return;   // the FP64 kick reads the state itself
    k_kick_stage<<<(unsigned)(d.ntot / (2 * kKickBox)), 2 * kKickBox, 0, s>>>(d);
    prof_mark("kick: sorted copies and tile boxes");
}

}  // namespace opal
