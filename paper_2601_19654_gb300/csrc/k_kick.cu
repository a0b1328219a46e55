// The kick's pair kernel: a_i = sum_{j != i} m_j K(r_ij; rc_ij) (x_j - x_i) / r_ij^3
// (Sec. 3.1, force block, LOOP 2, with the changeover weight K of the hybrid
// integrator).  G is applied when the partials are reduced.
//
// Work is a list of items (i-tile of 128 bodies x a j-range of the same
// system) spread round-robin over a persistent grid; each item writes its
// partial sums to its own row of a buffer that the closing kernel reduces in
// a fixed order, so results do not depend on the schedule.  j-bodies are
// staged through shared memory and read by every thread of the block
// (broadcast).  Pairs closer than 2 (rc_i + rc_max) take a slow path that
// handles the changeover, the self pair and exact coincidence; all other
// pairs take the plain Newtonian fast path.
//
// Mixed form: FP32 separations of the hi parts of a hi/lo float split of the
// FP64 positions (the lo parts are added on the slow path), MUFU rsqrt, FP32
// sums over each 128-body j-tile folded into a float hi/lo pair with Knuth's
// TwoSum, converted to FP64 at the end.  FP64 form: the same in doubles.
#include "opal_internal.cuh"

namespace opal {

constexpr int kJTile = 128;

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
__device__ __forceinline__ float4 slow_pair_f(const Dev& d, int64_t i, int64_t j, float dx, float dy, float dz,
                                              float mj, float rci, int form) {
    float4 li = d.kl[i], lj = d.kl[j];
    dx += lj.x - li.x;
    dy += lj.y - li.y;
    dz += lj.z - li.z;
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float s = 0.0f;
    if (r2 > 0.0f) {
        float r = sqrtf(r2);
        float rcij = fmaxf(rci, d.rcf[j]);
        float K = changeover_f(r, rcij, form);
        s = mj * K / (r2 * r);
    }
    return make_float4(s, dx, dy, dz);
}

__device__ __forceinline__ double slow_pair_d(const Dev& d, int64_t j, double r2, double mj, double rci, int form) {
    if (!(r2 > 0.0)) return 0.0;
    double r = sqrt(r2);
    double rcij = fmax(rci, d.rc[j]);
    double K = changeover(r, rcij, form);
    return mj * K / (r2 * r);
}

// Fixed-order sum of m V over the tile's kSeg-body segments (chunk 0 only):
// the momentum the closing jump needs, after any encounter changes.
template <int T, int NI>
__device__ void tile_momentum(const Dev& d, int64_t i0) {
    __shared__ double red[3][T * NI];
    for (int q = 0; q < NI; q++) {
        int64_t i = i0 + q * T + threadIdx.x;
        double m = d.alive[i] ? d.m[i] : 0.0;
        red[0][q * T + threadIdx.x] = m * d.vx[i];
        red[1][q * T + threadIdx.x] = m * d.vy[i];
        red[2][q * T + threadIdx.x] = m * d.vz[i];
    }
    __syncthreads();
    if (threadIdx.x < 3 * (T * NI / kSeg)) {
        int c = threadIdx.x % 3, sgl = threadIdx.x / 3;
        double s = 0.0;
        for (int k = 0; k < kSeg; k++) s += red[c][sgl * kSeg + k];
        d.pP_close[c * d.nseg_tot + i0 / kSeg + sgl] = s;
    }
    __syncthreads();
}

template <int T, int NI, int MINB>
__global__ void __launch_bounds__(T, MINB) k_kick_mixed(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    __shared__ float4 sj[kJTile];
    if (d.ctl->status) return;
    const int form = d.p.changeover;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const KickItem w = items[it];
        const SysInfo si = d.sys[w.sys];
        const float rcm = d.rcmax[w.sys];
        float xi[NI], yi[NI], zi[NI], thr[NI], rci[NI];
        float hx[NI], hy[NI], hz[NI], lx[NI], ly[NI], lz[NI];
#pragma unroll
        for (int q = 0; q < NI; q++) {
            int64_t i = w.i0 + q * T + threadIdx.x;
            float4 h = d.kh[i];
            xi[q] = h.x; yi[q] = h.y; zi[q] = h.z;
            rci[q] = d.rcf[i];
            float t = 2.0f * (rci[q] + rcm);
            thr[q] = fmaxf(t * t, 1e-30f);
            hx[q] = hy[q] = hz[q] = lx[q] = ly[q] = lz[q] = 0.0f;
        }
        for (int64_t jb = w.j0; jb < w.j1; jb += kJTile) {
            const int nj = (int)min((int64_t)kJTile, w.j1 - jb);
            __syncthreads();
            for (int k = threadIdx.x; k < nj; k += T) sj[k] = d.kh[jb + k];
            __syncthreads();
            float tx[NI], ty[NI], tz[NI];
#pragma unroll
            for (int q = 0; q < NI; q++) tx[q] = ty[q] = tz[q] = 0.0f;
#pragma unroll 4
            for (int jj = 0; jj < nj; jj++) {
                const float4 pj = sj[jj];
#pragma unroll
                for (int q = 0; q < NI; q++) {
                    float dx = pj.x - xi[q], dy = pj.y - yi[q], dz = pj.z - zi[q];
                    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    float s;
                    if (r2 < thr[q]) {
                        float4 r = slow_pair_f(d, w.i0 + q * T + threadIdx.x, jb + jj, dx, dy, dz, pj.w, rci[q], form);
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
#pragma unroll
            for (int q = 0; q < NI; q++) {
                fold(hx[q], lx[q], tx[q]);
                fold(hy[q], ly[q], ty[q]);
                fold(hz[q], lz[q], tz[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NI; q++) {
            int64_t i = w.i0 + q * T + threadIdx.x;
            int64_t slot = si.slot0 + (int64_t)w.chunk * si.cap + (i - si.off);
            d.pacc_x[slot] = (double)hx[q] + (double)lx[q];
            d.pacc_y[slot] = (double)hy[q] + (double)ly[q];
            d.pacc_z[slot] = (double)hz[q] + (double)lz[q];
        }
        if (w.chunk == 0) tile_momentum<T, NI>(d, w.i0);
    }
}

template <int T>
__global__ void __launch_bounds__(T) k_kick_fp64(Dev d, const KickItem* __restrict__ items, int64_t nitems) {
    __shared__ D4 sj[kJTile];
    if (d.ctl->status) return;
    const int form = d.p.changeover;
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
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
                    s = slow_pair_d(d, jb + jj, r2, pj.w, rci, form);
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
        if (w.chunk == 0) tile_momentum<T, 1>(d, w.i0);
    }
}

// Kick variants the autotuner picks from: (threads, i-bodies per thread,
// minimum resident blocks); every variant covers a 128-body i-tile.
struct KickVariant {
    const char* name;
    int threads;
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
    {"mixed t128 i1", 128, launch_mixed<128, 1, 8>, occ_mixed<128, 1, 8>},
    {"mixed t64 i2", 64, launch_mixed<64, 2, 12>, occ_mixed<64, 2, 12>},
    {"mixed t64 i2 r", 64, launch_mixed<64, 2, 16>, occ_mixed<64, 2, 16>},
    {"mixed t32 i4", 32, launch_mixed<32, 4, 16>, occ_mixed<32, 4, 16>},
    {"mixed t128 i1 r", 128, launch_mixed<128, 1, 4>, occ_mixed<128, 1, 4>},
};
static const KickVariant kFp64[] = {
    {"fp64 t128", 128, launch_fp64<128>, occ_fp64<128>},
};

int kick_num_variants(int precision) {
    return precision == 1 ? (int)(sizeof(kMixed) / sizeof(kMixed[0])) : (int)(sizeof(kFp64) / sizeof(kFp64[0]));
}
const char* kick_variant_name(int precision, int v) { return precision == 1 ? kMixed[v].name : kFp64[v].name; }
int kick_occupancy(int precision, int v) { return precision == 1 ? kMixed[v].occupancy() : kFp64[v].occupancy(); }
void launch_kick(const Dev& d, const KickItem* items, int64_t nitems, int grid, int precision, int v,
                 cudaStream_t s) {
    if (precision == 1) kMixed[v].launch(d, items, nitems, grid, s);
    else kFp64[v].launch(d, items, nitems, grid, s);
    prof_mark("kick");
}

}  // namespace opal
