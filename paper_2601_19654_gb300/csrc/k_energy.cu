// Energy, angular momentum and momentum of each system in democratic
// heliocentric variables (Sec. 2.1.1 item (7), mxx_en; the Hamiltonian split
// is footnote 1 of Sec. 2.1.1):
//   E = sum 1/2 m |V|^2 - sum G M0 m / |x| + |P|^2 / (2 M0) - sum_{i<j} G m_i m_j / r_ij,
//   P = sum m V,  L = sum m x x V.
// FP64 throughout; every partial is summed in a fixed order.
#include <cuda.h>   // driver types only: cuCtxGetCurrent / cuCtxGetId are reached through the runtime
#include <cmath>
#include <mutex>

#include "opal_internal.cuh"

namespace opal {

constexpr int kEnThreads = 128;

// body terms: per 128-body block, 7 sums (kinetic + central, P, L)
__global__ void __launch_bounds__(kEnThreads) k_energy_body(Dev d, double* body_part) {
    __shared__ double red[7][kEnThreads];
    const int64_t b = (int64_t)blockIdx.x * kEnThreads + threadIdx.x;
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (d.alive[b]) {
        double m = d.m[b], x = d.x[b], y = d.y[b], z = d.z[b], vx = d.vx[b], vy = d.vy[b], vz = d.vz[b];
        v[0] = 0.5 * m * (vx * vx + vy * vy + vz * vz) - d.p.G * d.M0s[d.body_sys[b]] * m / sqrt(x * x + y * y + z * z);
        v[1] = m * vx;
        v[2] = m * vy;
        v[3] = m * vz;
        v[4] = m * (y * vz - z * vy);
        v[5] = m * (z * vx - x * vz);
        v[6] = m * (x * vy - y * vx);
    }
    for (int c = 0; c < 7; c++) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = kEnThreads / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 7; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 7) body_part[(int64_t)blockIdx.x * 7 + threadIdx.x] = red[threadIdx.x][0];
}

// pair potential: one kSeg x kSeg tile (j-tile at or above the i-tile) per item
__global__ void __launch_bounds__(kSeg) k_energy_pair(Dev d, const PairTile* tiles, int64_t ntiles,
                                                      double* pair_part) {
    __shared__ D4 sj[kSeg];
    __shared__ double red[kSeg];
    for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x) {
        const PairTile tl = tiles[it];
        const int64_t i = tl.i0 + threadIdx.x;
        __syncthreads();
        {
            int64_t j = tl.j0 + threadIdx.x;
            sj[threadIdx.x] = D4{d.x[j], d.y[j], d.z[j], d.alive[j] ? d.m[j] : 0.0};
        }
        __syncthreads();
        double e = 0.0;
        if (d.alive[i]) {
            const double xi = d.x[i], yi = d.y[i], zi = d.z[i], mi = d.m[i];
            for (int jj = 0; jj < kSeg; jj++) {
                if (tl.j0 + jj <= i) continue;
                D4 pj = sj[jj];
                if (pj.w == 0.0) continue;
                double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
                e -= mi * pj.w / sqrt(dx * dx + dy * dy + dz * dz);
            }
        }
        red[threadIdx.x] = e;
        __syncthreads();
        for (int w = kSeg / 2; w >= 1; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) pair_part[it] = d.p.G * red[0];
    }
}

// one block per system: fixed-order sums of its partials
__global__ void k_energy_final(Dev d, const double* body_part, const double* pair_part, const int64_t* tile_off,
                               double* out) {
    const int s = blockIdx.x;
    const SysInfo si = d.sys[s];
    __shared__ double red[8][256];
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t b0 = si.off / kEnThreads, nb = si.cap / kEnThreads;
    for (int64_t k = threadIdx.x; k < nb; k += blockDim.x)
        for (int c = 0; c < 7; c++) v[c] += body_part[(b0 + k) * 7 + c];
    for (int64_t k = tile_off[s] + threadIdx.x; k < tile_off[s + 1]; k += blockDim.x) v[7] += pair_part[k];
    for (int c = 0; c < 8; c++) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 8; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double Px = red[1][0], Py = red[2][0], Pz = red[3][0];
        double E = red[0][0] + (Px * Px + Py * Py + Pz * Pz) / (2.0 * d.M0s[s]) + red[7][0];
        double* o = out + 8 * s;
        o[0] = E;
        o[1] = red[4][0]; o[2] = red[5][0]; o[3] = red[6][0];
        o[4] = Px; o[5] = Py; o[6] = Pz;
        o[7] = d.E_lost[s];
    }
}

void launch_energy(const Dev& d, const PairTile* tiles, int64_t ntiles, const int64_t* tile_off,
                   double* pair_part, double* body_part, double* out, int grid, cudaStream_t s) {
    k_energy_body<<<(unsigned)(d.ntot / kEnThreads), kEnThreads, 0, s>>>(d, body_part);
    k_energy_pair<<<grid, kSeg, 0, s>>>(d, tiles, ntiles, pair_part);
    k_energy_final<<<d.nsys, 256, 0, s>>>(d, body_part, pair_part, tile_off, out);
}

// ---------------------------------------------------------------------------
// The same energy, L and P from caller-owned device arrays of one system,
// with no allocation: the per-block partial sums live in a file-scope device
// array of fixed size, found once per device with cudaGetSymbolAddress.
// Inputs are heliocentric x and v; with u = sum m v / (M0 + sum m) the
// barycentric velocities are V = v - u, so
//   sum 1/2 m |V|^2 = sum 1/2 m |v|^2 - u . sum m v + 1/2 |u|^2 sum m,
//   P = sum m v - u sum m,  L = sum m x x v - (sum m x) x u,
// which lets one pass over the bodies gather every term.

constexpr int kNaThreads = 128;
constexpr int kNaMaxBlocks = 1024;
constexpr int64_t kNaMaxBodies = (int64_t)kNaThreads * kNaMaxBlocks;   // 131072
constexpr int kNaSums = 13;   // 1/2 m v^2, m v (3), m, m/|x|, m x (3), m x x v (3), sum_j m_i m_j / r_ij
constexpr int kNaMaxDevices = 64;

// Every slot a call reads is written earlier in the same call (block b writes
// row b; the final kernel reads rows 0 .. nb-1), so nothing here has to start
// at zero.
static __device__ __align__(256) double g_na_part[kNaMaxBlocks * kNaSums];

__global__ void __launch_bounds__(kNaThreads) k_energy_na_part(int64_t n, const double* __restrict__ m,
                                                               const double* __restrict__ x,
                                                               const double* __restrict__ v,
                                                               double* __restrict__ part) {
    __shared__ D4 sj[kNaThreads];
    __shared__ double red[kNaSums][kNaThreads];
    const int64_t i = (int64_t)blockIdx.x * kNaThreads + threadIdx.x;
    double s[kNaSums];
    for (int c = 0; c < kNaSums; c++) s[c] = 0.0;
    double xi = 0.0, yi = 0.0, zi = 0.0, mi = 0.0;
    if (i < n) {
        mi = m[i];
        xi = x[3 * i];
        yi = x[3 * i + 1];
        zi = x[3 * i + 2];
        const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
        if (mi != 0.0) {
            s[0] = 0.5 * mi * (vx * vx + vy * vy + vz * vz);
            s[1] = mi * vx;
            s[2] = mi * vy;
            s[3] = mi * vz;
            s[4] = mi;
            s[5] = mi / sqrt(xi * xi + yi * yi + zi * zi);
            s[6] = mi * xi;
            s[7] = mi * yi;
            s[8] = mi * zi;
            s[9] = mi * (yi * vz - zi * vy);
            s[10] = mi * (zi * vx - xi * vz);
            s[11] = mi * (xi * vy - yi * vx);
        }
    }
    // sum over every j != i of m_j / r_ij (each pair counted from both ends)
    double e = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += kNaThreads) {
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        sj[threadIdx.x] = j < n ? D4{x[3 * j], x[3 * j + 1], x[3 * j + 2], m[j]} : D4{0.0, 0.0, 0.0, 0.0};
        __syncthreads();
        if (mi != 0.0) {
            const int nj = (int)min((int64_t)kNaThreads, n - j0);
            for (int jj = 0; jj < nj; jj++) {
                const D4 pj = sj[jj];
                if (j0 + jj == i || pj.w == 0.0) continue;
                const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
                e += pj.w / sqrt(dx * dx + dy * dy + dz * dz);
            }
        }
    }
    s[12] = mi * e;
    for (int c = 0; c < kNaSums; c++) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = kNaThreads / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < kNaSums; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kNaSums) part[(int64_t)blockIdx.x * kNaSums + threadIdx.x] = red[threadIdx.x][0];
}

// one block: fixed-order sums of the nb partial rows, then E, L, P
__global__ void __launch_bounds__(256) k_energy_na_final(int nb, double G, double M0,
                                                         const double* __restrict__ part,
                                                         double* __restrict__ out) {
    __shared__ double red[kNaSums][256];
    double s[kNaSums];
    for (int c = 0; c < kNaSums; c++) s[c] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int c = 0; c < kNaSums; c++) s[c] += part[(int64_t)b * kNaSums + c];
    for (int c = 0; c < kNaSums; c++) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < kNaSums; c++) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double kin = red[0][0], mv[3] = {red[1][0], red[2][0], red[3][0]}, msum = red[4][0];
        const double pot_sun = red[5][0], mx[3] = {red[6][0], red[7][0], red[8][0]};
        const double lh[3] = {red[9][0], red[10][0], red[11][0]}, pair = red[12][0];
        double u[3], P[3];
        for (int k = 0; k < 3; k++) {
            u[k] = mv[k] / (M0 + msum);
            P[k] = mv[k] - u[k] * msum;
        }
        const double kinV = kin - (u[0] * mv[0] + u[1] * mv[1] + u[2] * mv[2]) +
                            0.5 * msum * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        out[0] = kinV - G * M0 * pot_sun + (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) / (2.0 * M0) -
                 0.5 * G * pair;
        out[1] = lh[0] - (mx[1] * u[2] - mx[2] * u[1]);
        out[2] = lh[1] - (mx[2] * u[0] - mx[0] * u[2]);
        out[3] = lh[2] - (mx[0] * u[1] - mx[1] * u[0]);
        out[4] = P[0];
        out[5] = P[1];
        out[6] = P[2];
    }
}

namespace {

std::mutex g_na_mu;
// per device: the scratch's device address and the context it belongs to
struct NaScratch {
    unsigned long long ctx_id;
    double* ptr;
};
NaScratch g_na[kNaMaxDevices] = {};
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// unique id of the current context (0 if none is current yet); caller holds g_na_mu
opal_status na_context_id(unsigned long long* id) {
    if (!g_ctx_current || !g_ctx_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            set_thread_error("the driver's context queries (cuCtxGetCurrent, cuCtxGetId) are unavailable");
            return OPAL_ECUDA;
        }
        g_ctx_current = (CtxGetCurrentFn)f1;
        g_ctx_id = (CtxGetIdFn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) {
        set_thread_error("cuCtxGetCurrent failed");
        return OPAL_ECUDA;
    }
    *id = 0;
    if (ctx && g_ctx_id(ctx, id) != CUDA_SUCCESS) {
        set_thread_error("cuCtxGetId failed");
        return OPAL_ECUDA;
    }
    return OPAL_OK;
}

// the device address of g_na_part in the current device's context, looked up
// once per device and context (a device reset or a new primary context makes
// the module load again at another address, so the lookup is redone)
opal_status na_scratch(double** out) {
    int dev = -1;
    cudaError_t rc = cudaGetDevice(&dev);
    if (rc != cudaSuccess) {
        set_thread_error("cudaGetDevice failed: %s", cudaGetErrorString(rc));
        return OPAL_ECUDA;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_thread_error("device ordinal %d is beyond the %d devices this path supports", dev, kNaMaxDevices);
        return OPAL_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_na_mu);
    unsigned long long id = 0;
    opal_status st = na_context_id(&id);
    if (st != OPAL_OK) return st;
    if (!g_na[dev].ptr || id == 0 || g_na[dev].ctx_id != id) {
        void* p = nullptr;
        rc = cudaGetSymbolAddress(&p, g_na_part);
        if (rc != cudaSuccess || !p) {
            set_thread_error("cudaGetSymbolAddress of the energy scratch failed on device %d: %s", dev,
                             cudaGetErrorString(rc));
            return OPAL_ECUDA;
        }
        st = na_context_id(&id);   // the lookup made the primary context current if none was
        if (st != OPAL_OK) return st;
        g_na[dev].ctx_id = id;
        g_na[dev].ptr = (double*)p;
    }
    *out = g_na[dev].ptr;
    return OPAL_OK;
}

// a pointer the kernels may read or write: device (or managed) memory of the
// current device, aligned for doubles
opal_status na_check_ptr(const void* p, const char* name) {
    if (!p) {
        set_thread_error("%s is NULL", name);
        return OPAL_EINVAL;
    }
    if (((uintptr_t)p & 7u) != 0) {
        set_thread_error("%s is not 8-byte aligned", name);
        return OPAL_EINVAL;
    }
    cudaPointerAttributes a{};
    cudaError_t rc = cudaPointerGetAttributes(&a, p);
    if (rc != cudaSuccess) {
        cudaGetLastError();
        set_thread_error("%s: cudaPointerGetAttributes failed: %s", name, cudaGetErrorString(rc));
        return OPAL_EINVAL;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (!((a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged)) {
        set_thread_error("%s is not device memory of the current device %d", name, dev);
        return OPAL_EINVAL;
    }
    return OPAL_OK;
}

}  // namespace

}  // namespace opal

using namespace opal;

extern "C" opal_status opal_energy_momentum_noalloc(int64_t n, double G, double M0, const double* m,
                                                    const double* x, const double* v, double* out,
                                                    void* stream) {
    if (n < 0) {
        set_thread_error("n = %lld < 0", (long long)n);
        return OPAL_EINVAL;
    }
    if (n > kNaMaxBodies) {
        set_thread_error("n = %lld exceeds the %lld-body limit of opal_energy_momentum_noalloc (its fixed scratch "
                         "holds %d blocks of %d bodies); use opal_energy_momentum",
                         (long long)n, (long long)kNaMaxBodies, kNaMaxBlocks, kNaThreads);
        return OPAL_EINVAL;
    }
    if (!(std::isfinite(G) && G > 0.0) || !(std::isfinite(M0) && M0 > 0.0)) {
        set_thread_error("G and M0 must be finite and > 0");
        return OPAL_EINVAL;
    }
    opal_status st = na_check_ptr(out, "out");
    if (st == OPAL_OK && n > 0) st = na_check_ptr(m, "m");
    if (st == OPAL_OK && n > 0) st = na_check_ptr(x, "x");
    if (st == OPAL_OK && n > 0) st = na_check_ptr(v, "v");
    if (st != OPAL_OK) return st;
    double* part = nullptr;
    st = na_scratch(&part);
    if (st != OPAL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + kNaThreads - 1) / kNaThreads);
    if (nb > 0) k_energy_na_part<<<nb, kNaThreads, 0, s>>>(n, m, x, v, part);
    k_energy_na_final<<<1, 256, 0, s>>>(nb, G, M0, part, out);
    cudaError_t rc = cudaGetLastError();
    if (rc != cudaSuccess) {
        set_thread_error("launch of the energy kernels failed: %s", cudaGetErrorString(rc));
        return OPAL_ECUDA;
    }
    return OPAL_OK;
}
