// Energy, angular momentum and momentum of each system in democratic
// heliocentric variables (Sec. 2.1.1 item (7), mxx_en; the Hamiltonian split
// is footnote 1 of Sec. 2.1.1):
//   E = sum 1/2 m |V|^2 - sum G M0 m / |x| + |P|^2 / (2 M0) - sum_{i<j} G m_i m_j / r_ij,
//   P = sum m V,  L = sum m x x V.
// FP64 throughout; every partial is summed in a fixed order.
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
        v[0] = 0.5 * m * (vx * vx + vy * vy + vz * vz) - d.p.G * d.p.M0 * m / sqrt(x * x + y * y + z * z);
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
        double E = red[0][0] + (Px * Px + Py * Py + Pz * Pz) / (2.0 * d.p.M0) + red[7][0];
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

}  // namespace opal
