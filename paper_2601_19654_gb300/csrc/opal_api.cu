// Host side of the C ABI (include/opal.h): validation, device layout, work
// lists, the per-step CUDA graph, and the copies across the boundary.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "../../include/opal.h"
#include "../../include/opal_testing.h"
#include "opal_internal.cuh"

using namespace opal;

namespace {

thread_local char g_err[512];

}  // namespace

namespace opal {
thread_local ProfRec* g_prof = nullptr;
}

namespace {

void set_err(char* buf, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (buf != g_err) std::memcpy(g_err, buf, 512);
}

}  // namespace

void opal::set_thread_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {

const char* status_name(int s) {
    switch (s) {
        case kOk: return "ok";
        case kEinval: return "invalid argument";
        case kEnomem: return "out of memory";
        case kEcuda: return "CUDA error";
        case kEkepler: return "Kepler drift did not converge";
        case kEbs: return "Bulirsch-Stoer substep cap reached";
        case kEoverflow: return "encounter list or group capacity exceeded";
        case kEnonfinite: return "non-finite value in the state";
    }
    return "unknown";
}

}  // namespace

struct opal_sim {
    Dev d{};
    int dev = 0;
    int nsm = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;             // the kick's branch of the step graph
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaStream_t side2 = nullptr;            // the large-group BS kernels' branch (in order)
    cudaStream_t side3 = nullptr;            // the same beside the kick, one priority lower
    cudaEvent_t fork2_ev = nullptr, join2_ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<SysInfo> sys;
    std::vector<int64_t> n_per_sys;
    std::vector<KickItem> items;
    std::vector<PairTile> tiles;
    std::vector<int64_t> tile_off;
    KickItem* d_items = nullptr;
    PairTile* d_tiles = nullptr;
    int64_t* d_tile_off = nullptr;
    int kick_grid = 1, scan_grid = 1, confirm_grid = 1, bs_grid = 1, energy_grid = 1;
    int kick_variant = 0;
    char kick_desc[256] = {0};
    int time_kick = 0;                       // graph records events around the kick
    cudaError_t launch_err = cudaSuccess;    // the first failed cluster or cooperative launch of a capture
    int64_t last_involved = 0;               // bodies in encounters in the last step
    int64_t last_inv_big = 0;                // of them big bodies (sources of force)
    int64_t n_big = 0;                       // big bodies of all systems
    cudaEvent_t kick_ev[2] = {nullptr, nullptr};
    double* d_rec = nullptr;       // get_state: one record of 8 doubles a body, the largest system
    int* d_ralive = nullptr;       // get_state: live flags
    double* d_exP = nullptr;       // get_state: the system's momentum
    int* d_excnt = nullptr;        // get_state: blocks done with their segments, a system
    double* h_rec = nullptr;       // pinned host copies of the two (allocated at the first get_state)
    int* h_ralive = nullptr;
    double* d_en_body = nullptr;
    double* d_en_pair = nullptr;
    double* d_en_out = nullptr;
    std::vector<void*> allocs;
    char err[512] = {0};
    int64_t n_total = 0;
};

namespace {

template <class T>
opal_status dalloc(opal_sim* s, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_err(s->err, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? OPAL_ENOMEM : OPAL_ECUDA;
    }
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return OPAL_OK;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            set_err(s->err, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return OPAL_ECUDA;                                                                \
        }                                                                                     \
    } while (0)

#define TRY(call)                          \
    do {                                   \
        opal_status st_ = (call);          \
        if (st_ != OPAL_OK) return st_;    \
    } while (0)

bool finite_all(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// The kick's work list.  Only a system's first nb places (its big bodies)
// are sources: j runs over them (small bodies follow them, in storage and in
// the sorted order alike); i runs over all cap places.  Items are taken from
// a queue, largest first.
//  - i-major (jmajor false): an i-tile of itile bodies against a j-chunk,
//    chunk edges on whole j-tiles, about eight items per resident block;
//    the chunk's partial row.
//  - j-major: one j-tile (staged once) against a run of i-tiles; the j-tile
//    index is the partial row.  The (i-tile, j-tile) units are grouped into
//    runs of 4 while more than four grids' worth of units remain (slots =
//    the blocks of the launch), then of 2 while more than two remain, then
//    single units, so that the queue ends on the smallest items.
void build_kick_items(opal_sim* s, int slots, int itile, bool jmajor) {
    double work = 0;
    for (auto& si : s->sys) work += (double)si.cap * (double)si.nb;
    const double target = std::max(1.0, work / (8.0 * std::max(1, slots)));
    s->items.clear();
    int64_t slot = 0, units = 0;
    for (auto& si : s->sys) units += (si.cap / itile) * ((si.nb + kKickJTile - 1) / kKickJTile);
    int64_t left = units;
    for (size_t k = 0; k < s->sys.size(); k++) {
        SysInfo& si = s->sys[k];
        const int64_t itiles = si.cap / itile;
        const int64_t jtiles = (si.nb + kKickJTile - 1) / kKickJTile;
        if (jmajor) {
            si.nchunk = (int32_t)std::max<int64_t>(1, jtiles);
            si.slot0 = slot;
            slot += (int64_t)si.nchunk * si.cap;
            for (int64_t t = 0; t < jtiles; t++) {
                const int64_t j0 = si.off + t * kKickJTile, j1 = si.off + std::min(si.nb, (t + 1) * kKickJTile);
                for (int64_t a = 0; a < itiles;) {
                    int64_t run = left > 4 * (int64_t)slots ? 4 : (left > 2 * (int64_t)slots ? 2 : 1);
                    run = std::min(run, itiles - a);
                    // the run's i-tiles a + u * S (u < run) for a block of run * S tiles,
                    // S = the block's stride: spatial neighbours go to different items
                    const int64_t span = std::min(itiles - a, (itiles - a) / run * run);
                    const int64_t S = std::max<int64_t>(1, span / run);
                    for (int64_t b = 0; b < S; b++) {
                        KickItem it{};
                        it.sys = (int32_t)k;
                        it.chunk = (int32_t)t;
                        it.i0 = si.off + (a + b) * itile;
                        it.istep = S * itile;
                        it.i1 = it.i0 + run * S * itile;
                        it.j0 = j0;
                        it.j1 = j1;
                        s->items.push_back(it);
                        left -= run;
                    }
                    a += run * S;
                }
            }
            if (jtiles == 0) {
                // no sources: one empty item per i-tile still writes the zero partial row
                for (int64_t a = 0; a < itiles; a++) {
                    KickItem it{};
                    it.sys = (int32_t)k;
                    it.chunk = 0;
                    it.i0 = si.off + a * itile;
                    it.i1 = it.i0 + itile;
                    it.istep = itile;
                    it.j0 = it.j1 = si.off;
                    s->items.push_back(it);
                }
            }
            continue;
        }
        const double w_tile = (double)itile * (double)si.nb;
        int64_t nchunk = (int64_t)std::llround(w_tile / target);
        nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, jtiles));
        si.nchunk = (int32_t)nchunk;
        si.slot0 = slot;
        slot += nchunk * si.cap;
        for (int64_t c = 0; c < nchunk; c++) {
            const int64_t t0 = jtiles * c / nchunk, t1 = jtiles * (c + 1) / nchunk;
            const int64_t j0 = si.off + t0 * kKickJTile, j1 = si.off + std::min(si.nb, t1 * kKickJTile);
            for (int64_t t = 0; t < itiles; t++) {
                KickItem it{};
                it.sys = (int32_t)k;
                it.chunk = (int32_t)c;
                it.i0 = si.off + t * itile;
                it.i1 = it.i0 + itile;
                it.istep = itile;
                it.j0 = j0;
                it.j1 = j1;
                s->items.push_back(it);
            }
        }
    }
    std::stable_sort(s->items.begin(), s->items.end(), [](const KickItem& a, const KickItem& b) {
        return (a.i1 - a.i0) * (a.j1 - a.j0) > (b.i1 - b.i0) * (b.j1 - b.j0);
    });
}

void build_pair_tiles(opal_sim* s) {
    s->tiles.clear();
    s->tile_off.assign(1, 0);
    for (size_t k = 0; k < s->sys.size(); k++) {
        const SysInfo& si = s->sys[k];
        // tile pairs (A, B >= A) with a big body in A: every pair with a big
        // member (pairs of two small bodies never interact)
        const int64_t nt = (si.n + kSeg - 1) / kSeg, ntb = (si.nb + kSeg - 1) / kSeg;
        for (int64_t a = 0; a < ntb; a++)
            for (int64_t b = a; b < nt; b++) {
                PairTile t{};
                t.sys = (int32_t)k;
                t.i0 = si.off + a * kSeg;
                t.j0 = si.off + b * kSeg;
                s->tiles.push_back(t);
            }
        s->tile_off.push_back((int64_t)s->tiles.size());
    }
}

opal_status validate(const opal_params* p, char* err) {
    if (!p) return set_err(err, "params is NULL"), OPAL_EINVAL;
    if (!(std::isfinite(p->G) && p->G > 0)) return set_err(err, "G must be finite and > 0"), OPAL_EINVAL;
    if (!(std::isfinite(p->M0) && p->M0 > 0)) return set_err(err, "M0 must be finite and > 0"), OPAL_EINVAL;
    if (!(std::isfinite(p->dt) && p->dt != 0)) return set_err(err, "dt must be finite and nonzero"), OPAL_EINVAL;
    if (!(std::isfinite(p->rcrit_hill) && p->rcrit_hill >= 0))
        return set_err(err, "rcrit_hill must be finite and >= 0"), OPAL_EINVAL;
    if (!(std::isfinite(p->bs_tol) && p->bs_tol > 0)) return set_err(err, "bs_tol must be > 0"), OPAL_EINVAL;
    if (p->precision != 0 && p->precision != 1) return set_err(err, "precision must be 0 or 1"), OPAL_EINVAL;
    if (!(std::isfinite(p->r_star) && p->r_star >= 0)) return set_err(err, "r_star must be finite and >= 0"), OPAL_EINVAL;
    if (!(std::isfinite(p->r_eject) && p->r_eject >= 0))
        return set_err(err, "r_eject must be finite and >= 0"), OPAL_EINVAL;
    if (p->eject_every < 0 || (p->r_eject > 0 && p->eject_every < 1))
        return set_err(err, "eject_every must be >= 1 when r_eject > 0"), OPAL_EINVAL;
    if (p->changeover != 0 && p->changeover != 1) return set_err(err, "changeover must be 0 or 1"), OPAL_EINVAL;
    if (p->kepler_max_iter < 0 || p->bs_max_substeps < 0 || p->encounter_capacity < 0)
        return set_err(err, "caps must be >= 0"), OPAL_EINVAL;
    return OPAL_OK;
}

opal_status capture_graph(opal_sim* s);

void reset_scan_order(opal_sim* s);

opal_status create_impl(const opal_params* p, int32_t nsys, const int64_t* nps, const double* m, const double* x,
                        const double* v, const double* R, opal_sim** out) {
    if (!out) return set_err(g_err, "out is NULL"), OPAL_EINVAL;
    *out = nullptr;
    TRY(validate(p, g_err));
    if (nsys <= 0 || !nps) return set_err(g_err, "need at least one system"), OPAL_EINVAL;
    int64_t ntot = 0;
    for (int32_t k = 0; k < nsys; k++) {
        if (nps[k] <= 0) return set_err(g_err, "system %d has n = %lld <= 0", k, (long long)nps[k]), OPAL_EINVAL;
        ntot += nps[k];
    }
    if (ntot > (int64_t)1 << 30) return set_err(g_err, "too many bodies"), OPAL_EINVAL;
    if (!m || !x || !v || !R) return set_err(g_err, "NULL body array"), OPAL_EINVAL;
    if (!finite_all(m, ntot) || !finite_all(x, 3 * ntot) || !finite_all(v, 3 * ntot) || !finite_all(R, ntot))
        return set_err(g_err, "non-finite value in the bodies"), OPAL_EINVAL;
    for (int64_t i = 0; i < ntot; i++) {
        if (m[i] < 0) return set_err(g_err, "body %lld has negative mass", (long long)i), OPAL_EINVAL;
        if (R[i] < 0) return set_err(g_err, "body %lld has negative radius", (long long)i), OPAL_EINVAL;
        if (x[3 * i] == 0 && x[3 * i + 1] == 0 && x[3 * i + 2] == 0)
            return set_err(g_err, "body %lld sits on the star", (long long)i), OPAL_EINVAL;
    }
    // small (zero-mass) bodies follow every big body of their system
    for (int64_t k = 0, i0 = 0; k < nsys; i0 += nps[k], k++)
        for (int64_t i = i0 + 1; i < i0 + nps[k]; i++)
            if (m[i] > 0 && m[i - 1] == 0)
                return set_err(g_err, "body %lld has mass but follows a small (zero-mass) body of its system",
                               (long long)i),
                       OPAL_EINVAL;
    opal_sim* s = new (std::nothrow) opal_sim();
    if (!s) return set_err(g_err, "host allocation failed"), OPAL_ENOMEM;
    opal_status st = OPAL_OK;
    auto fail = [&](opal_status code) {
        std::memcpy(g_err, s->err, sizeof(g_err));
        opal_destroy(s);
        return code;
    };
#define CKF(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            set_err(s->err, "%s failed: %s", #call, cudaGetErrorString(e_));                    \
            return fail(OPAL_ECUDA);                                                            \
        }                                                                                       \
    } while (0)
#define TRYF(call)                        \
    do {                                  \
        opal_status st_ = (call);         \
        if (st_ != OPAL_OK) return fail(st_); \
    } while (0)
    CKF(cudaGetDevice(&s->dev));
    CKF(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev));
    // the encounter kernels' streams outrank the kick's: when both are ready
    // (the fork of the step graph) the encounter blocks, which hold the
    // critical path, are placed first and the kick fills the rest.  Beside
    // the kick the larger-group branch runs one priority below the main
    // stream, so that its blocks, which wait for room, hold back no
    // small-group block.
    int prio_lo = 0, prio_hi = 0;
    CKF(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    const int prio_mid = prio_hi < prio_lo ? prio_hi + 1 : prio_hi;
    CKF(cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, prio_hi));
    CKF(cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, prio_lo));
    CKF(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
    CKF(cudaEventCreateWithFlags(&s->join_ev, cudaEventDisableTiming));
    CKF(cudaStreamCreateWithPriority(&s->side2, cudaStreamNonBlocking, prio_hi));
    CKF(cudaStreamCreateWithPriority(&s->side3, cudaStreamNonBlocking, prio_mid));
    CKF(cudaEventCreateWithFlags(&s->fork2_ev, cudaEventDisableTiming));
    CKF(cudaEventCreateWithFlags(&s->join2_ev, cudaEventDisableTiming));
    CKF(bs_setup());

    // parameters
    Params& P = s->d.p;
    P.G = p->G; P.M0 = p->M0; P.dt = p->dt; P.rcrit_hill = p->rcrit_hill; P.bs_tol = p->bs_tol;
    P.precision = p->precision; P.changeover = p->changeover;
    P.kepler_max_iter = p->kepler_max_iter > 0 ? p->kepler_max_iter : 50;
    P.bs_max_substeps = p->bs_max_substeps > 0 ? p->bs_max_substeps : (1 << 20);
    P.encounter_capacity = p->encounter_capacity > 0 ? p->encounter_capacity : std::max<int64_t>(4096, 4 * ntot);
    P.r_star = p->r_star;
    P.r_eject = p->r_eject;
    P.eject_every = p->eject_every;

    // layout
    int64_t off = 0, in0 = 0;
    for (int32_t k = 0; k < nsys; k++) {
        SysInfo si{};
        si.off = off;
        si.n = nps[k];
        si.nb = 0;
        while (si.nb < si.n && m[in0 + si.nb] > 0) si.nb++;
        in0 += nps[k];
        si.cap = (nps[k] + kPad - 1) / kPad * kPad;
        si.seg0 = off / kSeg;
        si.nseg = si.cap / kSeg;
        s->sys.push_back(si);
        s->n_per_sys.push_back(nps[k]);
        s->n_big += si.nb;
        off += si.cap;
    }
    const int64_t N = off;
    s->n_total = ntot;
    Dev& d = s->d;
    d.ntot = N;
    d.nsys = nsys;
    d.huge_wait_ns = kHugeWaitNs;
    d.huge_hold = 0;
    d.nseg_tot = N / kSeg;
    // kick variants: the work list of each, and the largest partial buffer any needs
    const int nvar = kick_num_variants(p->precision);
    std::vector<std::vector<KickItem>> var_items(nvar);
    std::vector<std::vector<SysInfo>> var_sys(nvar);
    std::vector<int> var_grid(nvar);
    int64_t max_slots = 0;
    for (int v = 0; v < nvar; v++) {
        int occ = std::max(1, kick_occupancy(p->precision, v));
        build_kick_items(s, s->nsm * occ, kick_itile(p->precision, v), kick_jmajor(p->precision, v));
        var_items[v] = s->items;
        var_sys[v] = s->sys;
        var_grid[v] = (int)std::min<int64_t>((int64_t)s->items.size(), (int64_t)s->nsm * occ);
        int64_t sl = 0;
        for (auto& si : s->sys) sl += (int64_t)si.nchunk * si.cap;
        max_slots = std::max(max_slots, sl);
    }
    build_pair_tiles(s);
    const int64_t nt = std::max<int64_t>(1, (int64_t)s->tiles.size());
    s->scan_grid = (int)std::min<int64_t>(nt, (int64_t)s->nsm * 16);
    s->energy_grid = (int)std::min<int64_t>(nt, (int64_t)s->nsm * 16);
    s->confirm_grid = s->nsm * 2;
    s->bs_grid = s->nsm * 4;
    const int64_t slots = max_slots;

    double** f64[] = {&d.x, &d.y, &d.z, &d.vx, &d.vy, &d.vz, &d.ax, &d.ay, &d.az, &d.x0, &d.y0, &d.z0,
                      &d.vx0, &d.vy0, &d.vz0, &d.xs, &d.ys, &d.zs, &d.vxs, &d.vys, &d.vzs, &d.rcs,
                      &d.m, &d.R, &d.rc, &d.hcb};
    for (auto pp : f64) TRYF(dalloc(s, pp, N));
    TRYF(dalloc(s, &d.alive, N));
    TRYF(dalloc(s, &d.body_sys, N));
    TRYF(dalloc(s, &d.label, N));
    float4** f4[] = {&d.kh, &d.kl, &d.cen, &d.sc0, &d.sc1, &d.sv0, &d.sv1};
    for (auto pp : f4) TRYF(dalloc(s, pp, N));
    TRYF(dalloc(s, &d.rcf, N));
    float** ksf[] = {&d.ks_x, &d.ks_y, &d.ks_z, &d.ks_m, &d.ks_rc};
    for (auto pp : ksf) TRYF(dalloc(s, pp, N));
    TRYF(dalloc(s, &d.ks_lo, N));
    TRYF(dalloc(s, &d.ksum, 3 * N));
#ifdef OPAL_TIMELINE
    TRYF(dalloc(s, &d.timeline, 2 * (size_t)kTlCount));
#endif
    TRYF(dalloc(s, &d.kbox, 2 * (N / kKickBox)));
    TRYF(dalloc(s, &d.kbox2, 2 * (N / (2 * kKickBox))));
    d.ncell = (int)(N / kBucketDiv);
    TRYF(dalloc(s, &d.sbox, 6 * nsys));
    TRYF(dalloc(s, &d.ckey, N));
    TRYF(dalloc(s, &d.cstart, d.ncell));
    TRYF(dalloc(s, &d.ccursor, d.ncell));
    TRYF(dalloc(s, &d.csorted, N));
    TRYF(dalloc(s, &d.cscratch, N));
    TRYF(dalloc(s, &d.cen_sorted, N));
    TRYF(dalloc(s, &d.tbox, 6 * (N / kSeg)));
    TRYF(dalloc(s, &d.rcmax, nsys));
    TRYF(dalloc(s, &d.pacc_x, slots));
    TRYF(dalloc(s, &d.pacc_y, slots));
    TRYF(dalloc(s, &d.pacc_z, slots));
    TRYF(dalloc(s, &d.pP_close, 3 * d.nseg_tot));
    TRYF(dalloc(s, &d.pP_open, 3 * d.nseg_tot));
    TRYF(dalloc(s, &d.Ptot, 6 * (int64_t)nsys));
    TRYF(dalloc(s, &d.Pjump, 6 * (int64_t)nsys));
    TRYF(dalloc(s, &d.pcnt, 2 * (int64_t)nsys));
    CKF(cudaMemsetAsync(d.pcnt, 0, 2 * nsys * sizeof(int), s->stream));
    d.flag_cap = P.encounter_capacity;
    d.cand_cap = std::max<int64_t>(1 << 16, 8 * d.flag_cap);
    d.near_cap = std::max<int64_t>(1 << 20, 64 * N);
    TRYF(dalloc(s, &d.cand, d.cand_cap));
    TRYF(dalloc(s, &d.near, d.near_cap));
    TRYF(dalloc(s, &d.flag, d.flag_cap));
    TRYF(dalloc(s, &d.members, 2 * d.flag_cap + 2));
    TRYF(dalloc(s, &d.goff, 2 * d.flag_cap + 2));
    TRYF(dalloc(s, &d.glarge, 2 * d.flag_cap + 2));
    d.gcap = std::min<int64_t>(d.flag_cap + 1, N / 2 + 1);   // a group has two members at least
    TRYF(dalloc(s, &d.gcls, 4 * d.gcap));
    TRYF(dalloc(s, &d.ghard, d.gcap));
    TRYF(dalloc(s, &d.ghuge, d.gcap));
    {
        // buffers of the whole-GPU encounter kernel, for groups of up to min(N, kHugeMax)
        HugeBuf& H = d.hb;
        H.cap = std::min<int64_t>(N, kHugeMax);
        const int64_t nch = (H.cap + 63) / 64;
        // the midpoint sequences advance in lockstep: chains, evaluation points
        // and pair sums for each of the kBsRows sequences
        TRYF(dalloc(s, &H.y, 6 * H.cap));
        TRYF(dalloc(s, &H.z0, (int64_t)kBsRows * 6 * H.cap));
        TRYF(dalloc(s, &H.z1, (int64_t)kBsRows * 6 * H.cap));
        TRYF(dalloc(s, &H.row, (int64_t)kBsRows * 6 * H.cap));
        TRYF(dalloc(s, &H.pos, (int64_t)kBsRows * 3 * H.cap));
        TRYF(dalloc(s, &H.posf, (int64_t)kBsRows * H.cap));
        TRYF(dalloc(s, &H.part, (int64_t)kBsRows * 3 * H.cap * nch));
        TRYF(dalloc(s, &H.m, H.cap));
        TRYF(dalloc(s, &H.R, H.cap));
        TRYF(dalloc(s, &H.rc, H.cap));
        TRYF(dalloc(s, &H.pinv, H.cap));
        TRYF(dalloc(s, &H.alive, H.cap));
        TRYF(dalloc(s, &H.gid, H.cap));
        TRYF(dalloc(s, &H.perm, H.cap));
        TRYF(dalloc(s, &H.wide, H.cap));
        TRYF(dalloc(s, &H.key, H.cap));
        TRYF(dalloc(s, &H.cbox, (int64_t)2 * kBsRows * nch * 2));
        TRYF(dalloc(s, &d.hctl, 1));
        CKF(cudaMemsetAsync(d.hctl, 0, sizeof(HugeCtl), s->stream));
    }
    TRYF(dalloc(s, &d.glost, 2 * d.flag_cap + 2));
    TRYF(dalloc(s, &d.undo, 3 * (2 * d.flag_cap + 2)));
    {
        const int64_t mcap = std::min<int64_t>(2 * d.flag_cap + 2, N + 2);   // members are distinct bodies
        TRYF(dalloc(s, &d.bsout, kBsOut * mcap));
        TRYF(dalloc(s, &d.okx, mcap));
    }
    TRYF(dalloc(s, &d.gcount, N));
    TRYF(dalloc(s, &d.gofs, N));
    TRYF(dalloc(s, &d.gidx, N));
    CKF(cudaMemsetAsync(d.gcount, 0, N * sizeof(int), s->stream));
    TRYF(dalloc(s, &d.mlo, nsys));
    TRYF(dalloc(s, &d.mhi, nsys));
    TRYF(dalloc(s, &d.cfx, kFixParts * N));
    TRYF(dalloc(s, &d.cfy, kFixParts * N));
    TRYF(dalloc(s, &d.cfz, kFixParts * N));
    TRYF(dalloc(s, &d.E_lost, nsys));
    TRYF(dalloc(s, &d.M0s, nsys));
    {
        std::vector<double> m0(nsys, p->M0);
        CKF(cudaMemcpyAsync(d.M0s, m0.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        CKF(cudaStreamSynchronize(s->stream));
    }
    TRYF(dalloc(s, &d.accf, N));
    CKF(cudaMemsetAsync(d.accf, 0, N * sizeof(int), s->stream));
    TRYF(dalloc(s, &d.ctl, 1));
    TRYF(dalloc(s, &d.sys, nsys));
    size_t max_items = 0;
    for (auto& it : var_items) max_items = std::max(max_items, it.size());
    TRYF(dalloc(s, &s->d_items, max_items));
    TRYF(dalloc(s, &s->d_tiles, s->tiles.size()));
    TRYF(dalloc(s, &d.tov, std::max<size_t>(1, s->tiles.size())));
    TRYF(dalloc(s, &s->d_tile_off, s->tile_off.size()));
    {
        int64_t maxcap = 0;
        for (auto& si : s->sys) maxcap = std::max(maxcap, si.cap);
        TRYF(dalloc(s, &s->d_rec, 8 * maxcap));
        TRYF(dalloc(s, &s->d_ralive, maxcap));
        TRYF(dalloc(s, &s->d_exP, 3));
        TRYF(dalloc(s, &s->d_excnt, nsys));
    }
    TRYF(dalloc(s, &s->d_en_body, 7 * (N / 128)));
    TRYF(dalloc(s, &s->d_en_pair, s->tiles.size()));
    TRYF(dalloc(s, &s->d_en_out, 8 * nsys));

    // host staging in the padded SoA layout
    std::vector<double> hx(N), hy(N), hz(N), hvx(N, 0.0), hvy(N, 0.0), hvz(N, 0.0), hm(N, 0.0), hR(N, 0.0);
    std::vector<int32_t> halive(N, 0), hsys(N, 0), hlabel(N, -1);
    int64_t src = 0;
    for (int32_t k = 0; k < nsys; k++) {
        const SysInfo& si = s->sys[k];
        for (int64_t t = 0; t < si.cap; t++) {
            int64_t b = si.off + t;
            hsys[b] = k;
            if (t < si.n) {
                hx[b] = x[3 * src]; hy[b] = x[3 * src + 1]; hz[b] = x[3 * src + 2];
                hvx[b] = v[3 * src]; hvy[b] = v[3 * src + 1]; hvz[b] = v[3 * src + 2];
                hm[b] = m[src];
                hR[b] = R[src];
                halive[b] = 1;
                src++;
            } else {   // ghost: massless, parked far away
                hx[b] = 1.0e6 + (double)b; hy[b] = 0.0; hz[b] = 0.0;
            }
        }
    }
    auto up = [&](void* dst, const void* srcp, size_t bytes) {
        return cudaMemcpyAsync(dst, srcp, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    CKF(up(d.x, hx.data(), N * 8)); CKF(up(d.y, hy.data(), N * 8)); CKF(up(d.z, hz.data(), N * 8));
    CKF(up(d.vx, hvx.data(), N * 8)); CKF(up(d.vy, hvy.data(), N * 8)); CKF(up(d.vz, hvz.data(), N * 8));
    CKF(up(d.m, hm.data(), N * 8)); CKF(up(d.R, hR.data(), N * 8));
    CKF(up(d.alive, halive.data(), N * 4)); CKF(up(d.body_sys, hsys.data(), N * 4));
    CKF(up(d.label, hlabel.data(), N * 4));
    CKF(up(s->d_tiles, s->tiles.data(), s->tiles.size() * sizeof(PairTile)));
    CKF(up(s->d_tile_off, s->tile_off.data(), s->tile_off.size() * sizeof(int64_t)));
    CKF(cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), s->stream));
    CKF(cudaMemsetAsync(d.E_lost, 0, nsys * 8, s->stream));
    CKF(cudaMemsetAsync(d.ax, 0, N * 8, s->stream));
    CKF(cudaMemsetAsync(d.ay, 0, N * 8, s->stream));
    CKF(cudaMemsetAsync(d.az, 0, N * 8, s->stream));
    CKF(cudaMemsetAsync(d.rcmax, 0, nsys * 4, s->stream));
    // democratic heliocentric velocities, critical radii (offsets and
    // capacities are the same in every variant's system table)
    CKF(up(d.sys, var_sys[0].data(), nsys * sizeof(SysInfo)));
    launch_to_dh(d, s->stream);
    launch_prime(d, s->stream);
    // a spatially sorted body order for the kick (each step's scan sorts again)
    reset_scan_order(s);
    launch_order_prep(d, s->stream);
    launch_sort_bodies(d, s->stream);
    // pick the kick variant: timed on this simulation's own positions
    {
        // blocks of variant v an SM in the step graph: as many as fit.  Beside
        // the encounter integrator some of them wait for room, and take it as
        // the encounter blocks finish (measured on the 16384-body disk: with
        // room left for one encounter block an SM the kick took 162 us in the
        // graph, with every block it fits 144 us, the encounter kernel the same)
        auto graph_blocks = [&](int v) { return std::max(1, kick_occupancy(p->precision, v)); };
        int best = 0;
        const char* force = getenv("OPAL_KICK_VARIANT");
        double work = 0;
        for (auto& si : s->sys) work += (double)si.cap * (double)si.n;
        double best_ms = -1;
        std::vector<double> var_ms(nvar, -1.0);
        if (force) {
            best = std::max(0, std::min(nvar - 1, atoi(force)));
        } else if (nvar > 1 && work >= 4.0e6) {
            launch_kick_stage(d, P.precision, s->stream);
            cudaEvent_t e0, e1;
            CKF(cudaEventCreate(&e0));
            CKF(cudaEventCreate(&e1));
            for (int v = 0; v < nvar; v++) {
                CKF(up(d.sys, var_sys[v].data(), nsys * sizeof(SysInfo)));
                CKF(up(s->d_items, var_items[v].data(), var_items[v].size() * sizeof(KickItem)));
                const int reps = work >= 1e8 ? 3 : 10;
                launch_kick(d, s->d_items, (int64_t)var_items[v].size(), var_grid[v], P.precision, v, s->stream);
                CKF(cudaEventRecord(e0, s->stream));
                for (int r = 0; r < reps; r++)
                    launch_kick(d, s->d_items, (int64_t)var_items[v].size(), var_grid[v], P.precision, v, s->stream);
                CKF(cudaEventRecord(e1, s->stream));
                CKF(cudaEventSynchronize(e1));
                float ms = 0;
                CKF(cudaEventElapsedTime(&ms, e0, e1));
                var_ms[v] = ms / reps;
                if (best_ms < 0 || ms / reps < best_ms) {
                    best_ms = ms / reps;
                    best = v;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            // timed alone, the variants come within a few per cent of each
            // other; in the step graph the kick shares the SMs with the
            // encounter integrator, and the variant with the most warps
            // resident there hides the latencies best.  Among those within
            // 3% of the fastest alone, take the one with the most warps.
            int best_w = graph_blocks(best) * kick_threads(p->precision, best) / 32;
            for (int v = 0; v < nvar; v++) {
                const int w = graph_blocks(v) * kick_threads(p->precision, v) / 32;
                if (var_ms[v] > 0 && var_ms[v] <= 1.03 * best_ms && w > best_w) {
                    best = v;
                    best_w = w;
                }
            }
        }
        s->kick_variant = best;
        s->kick_grid = (int)std::min<int64_t>((int64_t)var_items[best].size(), (int64_t)s->nsm * graph_blocks(best));
        // the chosen shape's work list, its item sizes scheduled for the blocks it runs with
        build_kick_items(s, s->kick_grid, kick_itile(p->precision, best), kick_jmajor(p->precision, best));
        s->kick_grid = (int)std::min<int64_t>((int64_t)s->items.size(), (int64_t)s->nsm * graph_blocks(best));
        snprintf(s->kick_desc, sizeof(s->kick_desc), "%s, grid %d, %zu items, %d j-chunks (system 0)%s",
                 kick_variant_name(p->precision, best), s->kick_grid, s->items.size(), s->sys[0].nchunk,
                 force ? ", forced" : (best_ms >= 0 ? ", autotuned" : ""));
        CKF(up(d.sys, s->sys.data(), nsys * sizeof(SysInfo)));
        CKF(up(s->d_items, s->items.data(), s->items.size() * sizeof(KickItem)));
    }
    {
        // warps a position takes in the row sums: eight rows a warp, at most eight warps
        int32_t maxc = 1;
        for (auto& si : s->sys) maxc = std::max(maxc, si.nchunk);
        d.rows_g = 1;
        while (d.rows_g < 8 && d.rows_g * 8 < maxc) d.rows_g *= 2;
    }
    launch_kick_stage(d, P.precision, s->stream);
    launch_kick(d, s->d_items, (int64_t)s->items.size(), s->kick_grid, P.precision, s->kick_variant, s->stream);
    launch_kick_rows(d, s->stream);
    launch_first_accel_finish(d, s->stream);
    CKF(cudaGetLastError());
    CKF(cudaStreamSynchronize(s->stream));
    Ctl c{};
    CKF(cudaMemcpy(&c, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (c.status) {
        set_err(s->err, "initial accelerations: %s (body %d)", status_name(c.status), c.detail);
        return fail((opal_status)c.status);
    }
    st = capture_graph(s);
    if (st != OPAL_OK) return fail(st);
    *out = s;
    return OPAL_OK;
#undef CKF
#undef TRYF
}

// bucket counts to zero; midpoint boxes to (+huge, -huge) in the order map
void reset_scan_order(opal_sim* s) {
    const Dev& d = s->d;
    cudaMemsetAsync(d.cstart, 0, (size_t)d.ncell * sizeof(int), s->stream);
    cudaMemsetAsync(d.sbox, 0x7f, 3 * d.nsys * sizeof(int), s->stream);
    cudaMemsetAsync(d.sbox + 3 * d.nsys, 0x80, 3 * d.nsys * sizeof(int), s->stream);
}

// the kernels of one step; names for profiling
const char* kKernelNames[] = {"counters", "open(kick+jump+drift)", "scan", "confirm", "group", "bs", "kick",
                              "apply bs", "kick fix", "close(jump+kick)", "finish", "accelerations afresh",
                              "removals"};
constexpr int kNumKernels = 13;
constexpr int kStageReprime = 11, kStageRemove = 12;
constexpr int kStageBs = 5, kStageKick = 6, kStageApply = 7;

// keep the first error of a cluster or cooperative launch, for the capture to report
void note_launch(opal_sim* s, cudaError_t e) {
    if (e != cudaSuccess && s->launch_err == cudaSuccess) s->launch_err = e;
}

// stage k of a step on stream st
// the kick and its row sums; the timing events (when on) bracket the kick
// kernel alone, not its staging
void launch_kick_timed(opal_sim* s, cudaStream_t st) {
    const Dev& d = s->d;
    if (s->time_kick) cudaEventRecordWithFlags(s->kick_ev[0], st, cudaEventRecordExternal);
    launch_kick(d, s->d_items, (int64_t)s->items.size(), s->kick_grid, d.p.precision, s->kick_variant, st);
    if (s->time_kick) cudaEventRecordWithFlags(s->kick_ev[1], st, cudaEventRecordExternal);
    launch_kick_rows(d, st);
}

void launch_stage(opal_sim* s, int k, cudaStream_t st) {
    const Dev& d = s->d;
    switch (k) {
        case 0: launch_step_reset(d, s->nsm, st); break;
        case 1: launch_open(d, st); break;
        case 2: launch_scan(d, s->d_tiles, (int64_t)s->tiles.size(), s->scan_grid, st); break;
        case 3: launch_confirm(d, s->confirm_grid, st); break;
        case 4: launch_group(d, s->nsm, st); break;
        case kStageBs:
            // the lockstep kernels on parallel branches (one stream when profiling)
            launch_bs_packed(d, s->nsm, st);
            note_launch(s, launch_bs_lockstep(d, s->nsm, st, g_prof ? st : s->side2, s->fork2_ev, s->join2_ev,
                                              false));
            break;
        case kStageKick:
            launch_kick_stage(d, d.p.precision, st);
            launch_kick_timed(s, st);
            break;
        case kStageApply: launch_bs_apply(d, s->nsm, st); break;
        case 8: launch_kick_fix(d, s->nsm, st); break;
        case 9: launch_close(d, st); break;
        case 10: launch_finish(d, st); break;
        case kStageReprime: {
            // after a removal: critical radii, kick and accelerations at the current
            // positions (each kernel returns at once when nothing was removed)
            Dev g = d;
            g.gated = 1;
            launch_prime(g, st);
            launch_kick_stage(g, d.p.precision, st);
            launch_kick(g, s->d_items, (int64_t)s->items.size(), s->kick_grid, d.p.precision, s->kick_variant, st);
            launch_kick_rows(g, st);
            launch_first_accel_finish(g, st);
            prof_mark("accelerations afresh after a removal");
            break;
        }
        case kStageRemove: launch_remove(d, st); break;
    }
}
void launch_stage(opal_sim* s, int k) { launch_stage(s, k, s->stream); }

// Order of the stages.  Overlap: the kick runs beside the BS on the state
// after the drift and the fix puts the members right afterwards.  In order:
// the BS results are applied first and the kick sees them (the fix only sums
// the momentum), which is cheaper when many bodies are in encounters.
// With star collisions or ejections on, the step ends with the removals and
// starts with the accelerations afresh (both return at once when idle).
int stage_order(const opal_sim* s, int* out) {
    static const int ov[] = {0, 1, 2, 3, 4, kStageBs, kStageKick, kStageApply, 8, 9, 10};
    static const int sq[] = {0, 1, 2, 3, 4, kStageBs, kStageApply, kStageKick, 8, 9, 10};
    const int* o = s->d.overlap ? ov : sq;
    const bool removals = s->d.p.r_star > 0 || s->d.p.r_eject > 0;
    int n = 0;
    for (int k = 0; k < 11; k++) {
        out[n++] = o[k];
        if (removals && o[k] == 0) out[n++] = kStageReprime;
    }
    if (removals) out[n++] = kStageRemove;
    return n;
}

opal_status capture_graph(opal_sim* s) {
    if (s->exec) {
        CK(cudaGraphExecDestroy(s->exec));
        s->exec = nullptr;
    }
    if (s->graph) {
        CK(cudaGraphDestroy(s->graph));
        s->graph = nullptr;
    }
    int order[kNumKernels];
    const int ns = stage_order(s, order);
    s->launch_err = cudaSuccess;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < ns; q++) {
        const int k = order[q];
        if (s->d.overlap && k == kStageKick) continue;
        if (s->d.overlap && k == kStageBs) {
            // fork: the kick on the side stream, the encounter integrator here; join before the fix.
            // The packed kernel (many groups; at once done otherwise) runs before the fork: its
            // blocks do not fit beside the kick's, and the lockstep kernels wait for it.
            launch_bs_packed(s->d, s->nsm, s->stream);
            CK(cudaEventRecord(s->fork_ev, s->stream));
            CK(cudaStreamWaitEvent(s->side, s->fork_ev, 0));
            launch_stage(s, kStageKick, s->side);
            CK(cudaEventRecord(s->join_ev, s->side));
            note_launch(s, launch_bs_lockstep(s->d, s->nsm, s->stream, s->side3, s->fork2_ev, s->join2_ev, true));
            CK(cudaStreamWaitEvent(s->stream, s->join_ev, 0));
            continue;
        }
        launch_stage(s, k);
    }
    cudaError_t e = cudaStreamEndCapture(s->stream, &s->graph);
    if (s->launch_err != cudaSuccess) {
        set_err(s->err, "launch of an encounter kernel (a cluster of attempt blocks, or the cooperative whole-GPU "
                        "kernel) refused: %s", cudaGetErrorString(s->launch_err));
        if (s->graph) {
            cudaGraphDestroy(s->graph);
            s->graph = nullptr;
        }
        return OPAL_ECUDA;
    }
    if (e != cudaSuccess) {
        set_err(s->err, "graph capture failed: %s", cudaGetErrorString(e));
        return OPAL_ECUDA;
    }
    CK(cudaGraphInstantiate(&s->exec, s->graph, 0));
    return OPAL_OK;
}

// Overlap (kick beside the encounter integrator, then patched) or in order.
// The patch costs about 2 x bodies x big members involved pair terms against
// the kick's bodies x big bodies, so the share that decides is that of the
// big bodies (sources) in encounters.  The FP64 form always runs in order:
// its kick is bound by the FP64 pipes the encounter integrator needs, and
// beside it both slow down by more than the encounter integrator takes alone.
opal_status choose_mode(opal_sim* s) {
    const double share = s->n_big > 0 ? (double)s->last_inv_big / (double)s->n_big : 0.0;
    int want = s->d.overlap;
    if (share < 0.03) want = 1;
    else if (share > 0.08) want = 0;
    if (s->d.p.precision == 0) want = 0;
    // OPAL_STEP_ORDER=overlap or inorder forces one (the mixed form; the FP64 form is always in order)
    const char* force = getenv("OPAL_STEP_ORDER");
    if (force && s->d.p.precision == 1) {
        if (!strcmp(force, "overlap")) want = 1;
        else if (!strcmp(force, "inorder")) want = 0;
    }
    if (want == s->d.overlap && s->exec) return OPAL_OK;
    s->d.overlap = want;
    return capture_graph(s);
}

opal_status finish_steps(opal_sim* s, int64_t before) {
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    Ctl c{};
    CK(cudaMemcpy(&c, s->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    s->last_involved = c.ninvolved;
    s->last_inv_big = c.ninv_big;
    if (c.status) {
        if (c.status == kEbs && c.detail >= kHugeAbortDetail)
            set_err(s->err, "step %lld: whole-GPU encounter kernel: a grid-barrier wait ran out (detail %d)",
                    (long long)(c.steps_done + 1), c.detail);
        else
            set_err(s->err, "step %lld: %s (detail %d)", (long long)(c.steps_done + 1), status_name(c.status),
                    c.detail);
        int zero[2] = {0, 0};
        CK(cudaMemcpy(s->d.ctl, zero, sizeof(zero), cudaMemcpyHostToDevice));
        return (opal_status)c.status;
    }
    (void)before;
    return OPAL_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

void opal_default_params(opal_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->G = 1.0;
    p->M0 = 1.0;
    p->dt = 2.0 * M_PI * 0.01;
    p->rcrit_hill = 3.0;
    p->bs_tol = 1e-12;
    p->precision = 1;
    p->changeover = 0;
}

opal_status opal_create(const opal_params* p, int64_t n, const double* m, const double* x, const double* v,
                        const double* radius, opal_sim** out) {
    return create_impl(p, 1, &n, m, x, v, radius, out);
}

opal_status opal_ensemble_create(const opal_params* p, int32_t nsys, const int64_t* n_per_sys, const double* m,
                                 const double* x, const double* v, const double* radius, opal_sim** out) {
    return create_impl(p, nsys, n_per_sys, m, x, v, radius, out);
}

opal_status opal_step(opal_sim* s, int64_t nsteps) {
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    if (nsteps < 0) return set_err(s->err, "nsteps < 0"), OPAL_EINVAL;
    TRY(choose_mode(s));
    for (int64_t k = 0; k < nsteps; k++) CK(cudaGraphLaunch(s->exec, s->stream));
    return finish_steps(s, 0);
}

opal_status opal_step_async(opal_sim* s, int64_t nsteps) {
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    if (nsteps < 0) return set_err(s->err, "nsteps < 0"), OPAL_EINVAL;
    TRY(choose_mode(s));
    for (int64_t k = 0; k < nsteps; k++) CK(cudaGraphLaunch(s->exec, s->stream));
    return OPAL_OK;
}

opal_status opal_wait(opal_sim* s) {
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    return finish_steps(s, 0);
}

int32_t opal_num_systems(const opal_sim* s) { return s ? s->d.nsys : 0; }
int64_t opal_num_bodies(const opal_sim* s) { return s ? s->n_total : 0; }

int64_t opal_steps_done(const opal_sim* s) {
    if (!s) return -1;
    long long v = 0;
    cudaStreamSynchronize(s->stream);
    cudaMemcpy(&v, reinterpret_cast<char*>(s->d.ctl) + offsetof(Ctl, steps_done), sizeof(v),
               cudaMemcpyDeviceToHost);
    return v;
}

opal_status opal_get_state(const opal_sim* cs, int32_t sys, int64_t* n_alive, int64_t* ids, double* m, double* x,
                           double* v, double* radius) {
    opal_sim* s = const_cast<opal_sim*>(cs);
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    if (sys < 0 || sys >= s->d.nsys) return set_err(s->err, "no system %d", sys), OPAL_EINVAL;
    const SysInfo si = s->sys[sys];
    const int64_t n = si.n;
    if (!s->h_rec) {   // pinned staging for the largest system, kept until destroy
        int64_t maxcap = 0;
        for (auto& q : s->sys) maxcap = std::max(maxcap, q.cap);
        CK(cudaHostAlloc(reinterpret_cast<void**>(&s->h_rec), std::max<int64_t>(1, 8 * maxcap) * 8, 0));
        CK(cudaHostAlloc(reinterpret_cast<void**>(&s->h_ralive), std::max<int64_t>(1, maxcap) * 4, 0));
    }
    CK(cudaMemsetAsync(s->d_excnt, 0, s->d.nsys * sizeof(int), s->stream));
    launch_export(s->d, sys, si.cap, s->d_exP, s->d_excnt, s->d_rec, s->d_ralive, s->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(s->h_rec, s->d_rec, n * 8 * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->h_ralive, s->d_ralive, n * 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!s->h_ralive[i]) continue;
        const double* r = s->h_rec + 8 * i;
        if (ids) ids[k] = i;
        if (m) m[k] = r[6];
        if (radius) radius[k] = r[7];
        if (x) { x[3 * k] = r[0]; x[3 * k + 1] = r[1]; x[3 * k + 2] = r[2]; }
        if (v) { v[3 * k] = r[3]; v[3 * k + 1] = r[4]; v[3 * k + 2] = r[5]; }
        k++;
    }
    if (n_alive) *n_alive = k;
    return OPAL_OK;
}

opal_status opal_energy_momentum(const opal_sim* cs, int32_t sys, double* E, double L[3], double P[3],
                                 double* E_merged_lost) {
    opal_sim* s = const_cast<opal_sim*>(cs);
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    if (sys < 0 || sys >= s->d.nsys) return set_err(s->err, "no system %d", sys), OPAL_EINVAL;
    launch_energy(s->d, s->d_tiles, (int64_t)s->tiles.size(), s->d_tile_off, s->d_en_pair, s->d_en_body,
                  s->d_en_out, s->energy_grid, s->stream);
    CK(cudaGetLastError());
    double o[8];
    CK(cudaMemcpyAsync(o, s->d_en_out + 8 * sys, sizeof(o), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (E) *E = o[0];
    if (L) { L[0] = o[1]; L[1] = o[2]; L[2] = o[3]; }
    if (P) { P[0] = o[4]; P[1] = o[5]; P[2] = o[6]; }
    if (E_merged_lost) *E_merged_lost = o[7];
    return OPAL_OK;
}

opal_status opal_last_step_stats(const opal_sim* cs, int64_t out[8]) {
    opal_sim* s = const_cast<opal_sim*>(cs);
    if (!s || !out) return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    Ctl c{};
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(&c, s->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    out[0] = c.nflag;
    out[1] = c.ngroups;
    out[2] = c.nmerge;
    out[3] = (int64_t)c.nsub;
    out[4] = c.ncand;
    out[5] = c.kepler_max;
    out[6] = c.nacc;
    out[7] = c.nej;
    return OPAL_OK;
}

opal_status opal_central_mass(const opal_sim* cs, int32_t sys, double* M0) {
    opal_sim* s = const_cast<opal_sim*>(cs);
    if (!s || !M0) return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    if (sys < 0 || sys >= s->d.nsys) return set_err(s->err, "no system %d", sys), OPAL_EINVAL;
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(M0, s->d.M0s + sys, sizeof(double), cudaMemcpyDeviceToHost));
    return OPAL_OK;
}

void* opal_stream(const opal_sim* s) { return s ? (void*)s->stream : nullptr; }

opal_status opal_profile_steps(opal_sim* s, int64_t nsteps, int32_t cap, int32_t* nk, double* ms,
                               const char** names) {
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    TRY(choose_mode(s));
    ProfRec rec{};
    rec.stream = s->stream;
    rec.cap = 64;
    for (int k = 0; k < rec.cap; k++) CK(cudaEventCreate(&rec.ev[k]));
    cudaEvent_t start;
    CK(cudaEventCreate(&start));
    std::vector<const char*> order;
    std::vector<double> acc;
    for (int64_t t = 0; t < nsteps; t++) {
        rec.n = 0;
        g_prof = &rec;
        CK(cudaEventRecord(start, s->stream));
        int stages[kNumKernels];
        const int ns = stage_order(s, stages);
        for (int q = 0; q < ns; q++) launch_stage(s, stages[q]);
        g_prof = nullptr;
        CK(cudaEventSynchronize(rec.ev[rec.n - 1]));
        for (int k = 0; k < rec.n; k++) {
            float f = 0;
            CK(cudaEventElapsedTime(&f, k == 0 ? start : rec.ev[k - 1], rec.ev[k]));
            size_t q = 0;
            while (q < order.size() && std::strcmp(order[q], rec.names[k]) != 0) q++;
            if (q == order.size()) {
                order.push_back(rec.names[k]);
                acc.push_back(0.0);
            }
            acc[q] += f;
        }
    }
    for (int k = 0; k < rec.cap; k++) cudaEventDestroy(rec.ev[k]);
    cudaEventDestroy(start);
    if (nk) *nk = (int32_t)order.size();
    for (size_t k = 0; k < order.size() && (int32_t)k < cap; k++) {
        if (ms) ms[k] = nsteps > 0 ? acc[k] / (double)nsteps : 0.0;
        if (names) names[k] = order[k];
    }
    return finish_steps(s, 0);
}

const char* opal_last_error(const opal_sim* s) { return s ? s->err : g_err; }

const char* opal_kick_config(const opal_sim* s) { return s ? s->kick_desc : ""; }

int32_t opal_graph_kernels(const opal_sim* s) {
    if (!s || !s->graph) return -1;
    size_t n = 0;
    if (cudaGraphGetNodes(s->graph, nullptr, &n) != cudaSuccess) return -1;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(s->graph, nodes.data(), &n) != cudaSuccess) return -1;
    int32_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

int32_t opal_step_overlap(const opal_sim* s) { return s ? s->d.overlap : -1; }

opal_status opal_time_kick(opal_sim* s, int32_t enable) {
    if (!s) return set_err(g_err, "sim is NULL"), OPAL_EINVAL;
    if (enable && !s->kick_ev[0]) {
        CK(cudaEventCreate(&s->kick_ev[0]));
        CK(cudaEventCreate(&s->kick_ev[1]));
    }
    CK(cudaStreamSynchronize(s->stream));
    s->time_kick = enable ? 1 : 0;
    return capture_graph(s);
}

double opal_last_kick_ms(const opal_sim* cs) {
    opal_sim* s = const_cast<opal_sim*>(cs);
    if (!s || !s->time_kick) return -1.0;
    if (cudaEventSynchronize(s->kick_ev[1]) != cudaSuccess) return -1.0;
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, s->kick_ev[0], s->kick_ev[1]) != cudaSuccess) return -1.0;
    return ms;
}

opal_status opal_time_kick_alone(opal_sim* s, int32_t reps, double* ms) {
    if (!s || !ms) return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    if (reps < 1) return set_err(s->err, "reps < 1"), OPAL_EINVAL;
    const Dev& d = s->d;
    CK(cudaStreamSynchronize(s->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int64_t ni = (int64_t)s->items.size();
    launch_kick(d, s->d_items, ni, s->kick_grid, d.p.precision, s->kick_variant, s->stream);
    cudaEventRecord(e0, s->stream);
    for (int32_t r = 0; r < reps; r++)
        launch_kick(d, s->d_items, ni, s->kick_grid, d.p.precision, s->kick_variant, s->stream);
    cudaEventRecord(e1, s->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_err(s->err, "kick timing failed: %s", cudaGetErrorString(e)), OPAL_ECUDA;
    *ms = (double)t / reps;
    return OPAL_OK;
}

void opal_destroy(opal_sim* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->side) cudaStreamSynchronize(s->side);
    if (s->side2) cudaStreamSynchronize(s->side2);
    if (s->side3) cudaStreamSynchronize(s->side3);
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    for (auto e : s->kick_ev)
        if (e) cudaEventDestroy(e);
    for (void* p : s->allocs) cudaFree(p);
    if (s->h_rec) cudaFreeHost(s->h_rec);
    if (s->h_ralive) cudaFreeHost(s->h_ralive);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->side) cudaStreamDestroy(s->side);
    if (s->fork_ev) cudaEventDestroy(s->fork_ev);
    if (s->join_ev) cudaEventDestroy(s->join_ev);
    if (s->side2) cudaStreamDestroy(s->side2);
    if (s->side3) cudaStreamDestroy(s->side3);
    if (s->fork2_ev) cudaEventDestroy(s->fork2_ev);
    if (s->join2_ev) cudaEventDestroy(s->join2_ev);
    delete s;
}

// ---------------------------------------------------------------------------
// test hooks (include/opal_testing.h)

opal_status opal_debug_accel(opal_sim* s, const double* rc, double* a) {
    if (!s || !a) return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    Dev& d = s->d;
    const int64_t N = d.ntot;
    if (rc) {
        std::vector<double> h(N, 0.0);
        int64_t src = 0;
        for (auto& si : s->sys)
            for (int64_t t = 0; t < si.n; t++) h[si.off + t] = rc[src++];
        CK(cudaMemcpyAsync(d.rc, h.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    // float copies of the current positions with these rc, then the kick
    CK(cudaMemsetAsync(d.rcmax, 0, d.nsys * 4, s->stream));
    reset_scan_order(s);
    launch_debug_scan_prep(d, s->stream);
    launch_sort_bodies(d, s->stream);
    launch_kick_stage(d, d.p.precision, s->stream);
    launch_kick(d, s->d_items, (int64_t)s->items.size(), s->kick_grid, d.p.precision, s->kick_variant, s->stream);
    launch_kick_rows(d, s->stream);
    launch_first_accel_finish(d, s->stream);
    CK(cudaGetLastError());
    std::vector<double> ax(N), ay(N), az(N);
    CK(cudaMemcpyAsync(ax.data(), d.ax, N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(ay.data(), d.ay, N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(az.data(), d.az, N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    int64_t dst = 0;
    for (auto& si : s->sys)
        for (int64_t t = 0; t < si.n; t++, dst++) {
            a[3 * dst] = ax[si.off + t];
            a[3 * dst + 1] = ay[si.off + t];
            a[3 * dst + 2] = az[si.off + t];
        }
    return OPAL_OK;
}

opal_status opal_debug_drift(int64_t n, double mu, double dt, int32_t max_iter, double* x, double* v,
                             int32_t* iters) {
    if (n <= 0 || !x || !v || !iters) return set_err(g_err, "bad argument"), OPAL_EINVAL;
    double *dx = nullptr, *dv = nullptr;
    int* di = nullptr;
    cudaError_t e = cudaMalloc(&dx, n * 24);
    if (e == cudaSuccess) e = cudaMalloc(&dv, n * 24);
    if (e == cudaSuccess) e = cudaMalloc(&di, n * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, n * 24, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dv, v, n * 24, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_debug_drift((int)n, mu, dt, max_iter > 0 ? max_iter : 50, dx, dv, di, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(x, dx, n * 24, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(v, dv, n * 24, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(iters, di, n * 4, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dv);
    cudaFree(di);
    if (e != cudaSuccess) return set_err(g_err, "drift test hook: %s", cudaGetErrorString(e)), OPAL_ECUDA;
    return OPAL_OK;
}

static opal_status upload_soa(opal_sim* s, const double* src, double* dx, double* dy, double* dz) {
    const int64_t N = s->d.ntot;
    std::vector<double> a(N, 0.0), b(N, 0.0), c(N, 0.0);
    int64_t k = 0;
    for (auto& si : s->sys)
        for (int64_t t = 0; t < si.n; t++, k++) {
            a[si.off + t] = src[3 * k];
            b[si.off + t] = src[3 * k + 1];
            c[si.off + t] = src[3 * k + 2];
        }
    CK(cudaMemcpyAsync(dx, a.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(dy, b.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(dz, c.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return OPAL_OK;
}

opal_status opal_debug_scan(opal_sim* s, const double* x0, const double* V0, const double* x1, const double* V1,
                            const double* rc, int64_t cap, int32_t* pi, int32_t* pj, int64_t* count,
                            int64_t* ncand) {
    if (!s || !x0 || !V0 || !x1 || !V1 || !rc || !count) return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    Dev& d = s->d;
    TRY(upload_soa(s, x0, d.x0, d.y0, d.z0));
    TRY(upload_soa(s, V0, d.vx0, d.vy0, d.vz0));
    TRY(upload_soa(s, x1, d.x, d.y, d.z));
    TRY(upload_soa(s, V1, d.vx, d.vy, d.vz));
    {
        const int64_t N = d.ntot;
        std::vector<double> h(N, 0.0);
        int64_t k = 0;
        for (auto& si : s->sys)
            for (int64_t t = 0; t < si.n; t++) h[si.off + t] = rc[k++];
        CK(cudaMemcpyAsync(d.rc, h.data(), N * 8, cudaMemcpyHostToDevice, s->stream));
    }
    CK(cudaMemsetAsync(reinterpret_cast<char*>(d.ctl) + offsetof(Ctl, ncand), 0,
                       offsetof(Ctl, steps_done) - offsetof(Ctl, ncand), s->stream));
    reset_scan_order(s);
    launch_debug_scan_prep(d, s->stream);
    launch_scan(d, s->d_tiles, (int64_t)s->tiles.size(), s->scan_grid, s->stream);
    launch_confirm(d, s->confirm_grid, s->stream);
    CK(cudaMemsetAsync(d.label, 0xff, d.ntot * sizeof(int32_t), s->stream));   // no groups formed here
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    Ctl c{};
    CK(cudaMemcpy(&c, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (ncand) *ncand = c.ncand;
    if (c.status) {
        int zero[2] = {0, 0};
        cudaMemcpy(d.ctl, zero, sizeof(zero), cudaMemcpyHostToDevice);
        set_err(s->err, "scan: %s", status_name(c.status));
        return (opal_status)c.status;
    }
    std::vector<int2> fl(std::min<int64_t>(c.nflag, d.flag_cap));
    if (!fl.empty()) CK(cudaMemcpy(fl.data(), d.flag, fl.size() * sizeof(int2), cudaMemcpyDeviceToHost));
    // report in body order of the input (system-local indices are global input order)
    std::vector<int64_t> map(d.ntot, -1);
    int64_t k = 0;
    for (auto& si : s->sys)
        for (int64_t t = 0; t < si.n; t++) map[si.off + t] = k++;
    std::vector<std::pair<int64_t, int64_t>> pr;
    for (auto& f : fl) pr.push_back({map[f.x], map[f.y]});
    std::sort(pr.begin(), pr.end());
    *count = (int64_t)pr.size();
    for (int64_t q = 0; q < (int64_t)pr.size() && q < cap; q++) {
        pi[q] = (int32_t)pr[q].first;
        pj[q] = (int32_t)pr[q].second;
    }
    return OPAL_OK;
}

opal_status opal_debug_barrier(opal_sim* s, int64_t wait_ns, int32_t hold) {
    if (!s) return set_err(g_err, "NULL simulation"), OPAL_EINVAL;
    if (wait_ns < 0 || (hold != 0 && hold != 1))
        return set_err(s->err, "wait_ns must be >= 0 and hold 0 or 1"), OPAL_EINVAL;
    s->d.huge_wait_ns = wait_ns > 0 ? wait_ns : kHugeWaitNs;
    s->d.huge_hold = hold;
    return capture_graph(s);
}

opal_status opal_debug_bs_group(opal_sim* s, const double* x0, const double* V0, const double* rc, double* x,
                                double* V, double* m, double* radius, int32_t* alive, double* E_lost,
                                int64_t* substeps) {
    if (!s || !x0 || !V0 || !rc || !x || !V || !m || !radius || !alive)
        return set_err(g_err, "NULL argument"), OPAL_EINVAL;
    if (s->d.nsys != 1) return set_err(s->err, "one system only"), OPAL_EINVAL;
    Dev& d = s->d;
    const SysInfo si = s->sys[0];
    const int64_t n = si.n;
    if (n > kBsMaxMembers) return set_err(s->err, "group larger than %d", kBsMaxMembers), OPAL_EINVAL;
    TRY(upload_soa(s, x0, d.x0, d.y0, d.z0));
    TRY(upload_soa(s, V0, d.vx0, d.vy0, d.vz0));
    std::vector<double> h(d.ntot, 0.0), hm(d.ntot, 0.0), hR(d.ntot, 0.0);
    std::vector<int32_t> ha(d.ntot, 0), mem(n), goff = {0, (int32_t)n};
    for (int64_t t = 0; t < n; t++) {
        h[t] = rc[t];
        hm[t] = m[t];
        hR[t] = radius[t];
        ha[t] = alive[t];
        mem[t] = (int32_t)t;
    }
    CK(cudaMemcpy(d.rc, h.data(), d.ntot * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.m, hm.data(), d.ntot * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.R, hR.data(), d.ntot * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.alive, ha.data(), d.ntot * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.members, mem.data(), n * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.goff, goff.data(), 8, cudaMemcpyHostToDevice));
    Ctl c{};
    c.ngroups = 1;
    c.ninvolved = (int)n;
    if (n > 4) {
        int zero = 0;
        c.nlarge = 1;
        CK(cudaMemcpy(d.glarge, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(d.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice));
    CK(cudaMemsetAsync(d.mlo, 0x7f, d.nsys * sizeof(int), s->stream));
    CK(cudaMemsetAsync(d.mhi, 0, d.nsys * sizeof(int), s->stream));
    launch_bs_packed(d, s->nsm, s->stream);
    CK(launch_bs_lockstep(d, s->nsm, s->stream, s->stream, nullptr, nullptr, false));
    launch_bs_apply(d, s->nsm, s->stream);   // puts the result into the state
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(&c, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    int zero[2] = {0, 0};
    CK(cudaMemcpy(d.ctl, zero, sizeof(zero), cudaMemcpyHostToDevice));
    if (substeps) *substeps = (int64_t)c.nsub;
    if (c.status) {
        set_err(s->err, "bs: %s", status_name(c.status));
        return (opal_status)c.status;
    }
    std::vector<double> a(n), b(n), cc(n), va(n), vb(n), vc(n), gl(1);
    CK(cudaMemcpy(a.data(), d.x, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(b.data(), d.y, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cc.data(), d.z, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(va.data(), d.vx, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vb.data(), d.vy, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vc.data(), d.vz, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(m, d.m, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(radius, d.R, n * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(alive, d.alive, n * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(gl.data(), d.glost, 8, cudaMemcpyDeviceToHost));
    for (int64_t t = 0; t < n; t++) {
        x[3 * t] = a[t]; x[3 * t + 1] = b[t]; x[3 * t + 2] = cc[t];
        V[3 * t] = va[t]; V[3 * t + 1] = vb[t]; V[3 * t + 2] = vc[t];
    }
    if (E_lost) *E_lost = gl[0];
    return OPAL_OK;
}

// Device timeline (timeline builds; the normal build reports none)
int32_t opal_timeline_kernels(void) {
#ifdef OPAL_TIMELINE
    return kTlCount;
#else
    return 0;
#endif
}

const char* opal_timeline_name(int32_t id) {
    static const char* names[kTlCount] = {
        "k_step_reset", "k_open", "k_sort_count", "k_sort_prefix", "k_sort_scatter", "k_sort_order",
        "k_tile_box", "k_tile_cull", "k_scan_tiles", "k_chord", "k_confirm", "k_group_link", "k_group_count",
        "k_group_offsets", "k_group_place", "k_group_order", "k_bs_packed", "k_bs_ws", "k_bs<256>", "k_bs<512>",
        "k_bs_huge", "k_kick_stage", "k_kick", "k_kick_rows", "k_kick_apply", "k_kick_fix", "k_close",
        "k_finish"};
    return id >= 0 && id < kTlCount ? names[id] : nullptr;
}

opal_status opal_timeline(opal_sim* s, int32_t reset, uint64_t* out) {
    if (!s) return OPAL_EINVAL;
#ifdef OPAL_TIMELINE
    CK(cudaStreamSynchronize(s->stream));
    if (reset) {
        unsigned long long h[2 * kTlCount];
        for (int i = 0; i < kTlCount; i++) {
            h[2 * i] = ~0ull;   // the earliest start comes down from here
            h[2 * i + 1] = 0ull;
        }
        CK(cudaMemcpy(s->d.timeline, h, sizeof(h), cudaMemcpyHostToDevice));
        return OPAL_OK;
    }
    if (!out) return set_err(s->err, "opal_timeline: out is NULL"), OPAL_EINVAL;
    CK(cudaMemcpy(out, s->d.timeline, 2 * kTlCount * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return OPAL_OK;
#else
    (void)reset;
    (void)out;
    set_err(s->err, "opal_timeline: the library was built without OPAL_TIMELINE");
    return OPAL_EINVAL;
#endif
}

}  // extern "C"
