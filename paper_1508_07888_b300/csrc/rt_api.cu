// rt_api.cu -- host side of the C ABI declared in include/rt_m1.h.
//
// Every call validates its arguments, returns an rt_status and never lets a
// C++ exception out.  All device work is ordered on a private non-blocking
// stream that is joined to the caller's stream with events at the start and
// end of each call, so the caller may pass the legacy default stream.  The
// per-step kernel sequence (transport, then chemistry with the diagnostics
// fused into it) is captured once into a CUDA graph of RT_GRAPH_STEPS steps
// and replayed.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rt_m1.h"
#include "launch.h"
#include "rt_device.h"

#define RT_GRAPH_STEPS 16

// supercomoving runs advance in chunks of at most this many steps (the a of
// each step of a chunk is computed on the host and read by the chemistry)
static constexpr int kCosmoChunk = 4096;

// a after dt (s) from a: one classical Runge-Kutta step of the Friedmann
// equation da/dt = a H0 sqrt(omega_m / a^3 + omega_l)
static double friedmann_step(double a, double dt, const rt_params &p)
{
    auto rate = [&](double x) { return x * p.H0 * std::sqrt(p.omega_m / (x * x * x) + p.omega_l); };
    const double k1 = rate(a), k2 = rate(a + 0.5 * dt * k1), k3 = rate(a + 0.5 * dt * k2),
                 k4 = rate(a + dt * k3);
    return a + dt * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
}

struct rt_handle {
    rt_params p;
    rtd::Phys ph;
    int nboxes = 0;
    bool fp64 = false, strict = false;
    size_t esize = 4;                        // bytes of one state scalar
    std::vector<rt_box> box;
    std::vector<rtd::BoxDev> bdev;           // host mirror
    rtd::BoxDev *d_boxes = nullptr;
    std::vector<void *> d_us;                // post-transport scratch per box
    std::vector<int64_t *> d_src_cell;
    std::vector<std::vector<int>> src_uidx;  // per box: unique-table index of each given source
    std::vector<double *> d_src_S;
    rtd::DiagPart *d_partials = nullptr;
    double *d_lanes = nullptr;               // per-item lane values of the FP64 diagnostics
    unsigned *d_done = nullptr;              // per-box group counters of the fused reduction
    rtd::DiagPart *d_gpart = nullptr;        // per-group partials
    unsigned *d_gdone = nullptr;             // per-group item counters
    rtd::RateCoef *d_rtab = nullptr;         // rate table (null: fits evaluated directly)
    rtd::CellConst *d_cc = nullptr;          // fast forms: per-cell chemistry constants (k_cconst)
    double *d_hll_d = nullptr;               // HLL wave speeds (FP64, FP32 copies)
    float *d_hll_f = nullptr;
    float4 *d_hll_f4 = nullptr;
    double *d_lastdiag = nullptr;
    rtd::Ctl *d_ctl = nullptr;
    rtd::Ctl *h_ctl = nullptr;               // pinned mirror
    double *h_lastdiag = nullptr;            // pinned
    int64_t ntitems = 0, ncitems = 0;
    int zc = 32;
    int tgrid = 1, cgrid = 1;
    int cgrab = 1;                           // chemistry: work items per draw
    int tvariant = 0;                        // tile shape of the FP32 transport (rtl::kTileX/Y)
    int tzlen = 0;                           // its z-chunk length (0: whole columns)
    void *d_tmaps = nullptr;                 // FP32 GLF transport: 3 TMA tensor maps per box
    bool tma = false;                        // every box has its maps (the TMA kernel runs)
    int tlock = 0;                           // lockstep-rows order: tile columns per row (0: off)
    int tgpb = 1;                            // FP32 GLF transport: photon groups per block
    int nsm = 1, chem_occ = 1;               // SMs, resident chemistry blocks per SM
    std::vector<rtd::FineDev> fdev;          // CRTA fine level per box (host mirror)
    rtd::FineDev *d_fines = nullptr;
    std::vector<int64_t *> d_fparent;        // library copies of the parent indices
    int64_t nfitems = 0;
    int fgrid = 1;
    double a_now = 1.0;                      // cosmo: expansion factor
    double *d_acos = nullptr, *h_acos = nullptr;   // cosmo: a per step of one chunk
    cudaStream_t user = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr;
    int64_t steps_done = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;        // 4 per profiled step
    double kernel_ms[3] = {0, 0, 0};
    int64_t kernel_launches[3] = {0, 0, 0};
    unsigned long long nclamp = 0;
    int error_bits = 0;
    std::string err;
};

static thread_local std::string g_create_err;

void rtl::set_thread_error(const char *msg) { g_create_err = msg ? msg : ""; }

static int fail(rt_handle *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_err = buf;
    return code;
}

#define CU(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((h), RT_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

static void release(rt_handle *h)
{
    if (!h) return;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (void *p : h->d_us) cudaFree(p);
    for (auto *p : h->d_src_cell) cudaFree(p);
    for (auto *p : h->d_src_S) cudaFree(p);
    cudaFree(h->d_boxes);
    cudaFree(h->d_tmaps);
    cudaFree(h->d_partials);
    cudaFree(h->d_lanes);
    cudaFree(h->d_done);
    cudaFree(h->d_gpart);
    cudaFree(h->d_gdone);
    cudaFree(h->d_hll_d);
    cudaFree(h->d_hll_f);
    cudaFree(h->d_hll_f4);
    cudaFree(h->d_acos);
    cudaFreeHost(h->h_acos);
    cudaFree(h->d_fines);
    for (auto q : h->d_fparent) cudaFree(q);
    cudaFree(h->d_rtab);
    cudaFree(h->d_cc);
    cudaFree(h->d_lastdiag);
    cudaFree(h->d_ctl);
    cudaFreeHost(h->h_ctl);
    cudaFreeHost(h->h_lastdiag);
    for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->s) cudaStreamDestroy(h->s);
    delete h;
}

// chemistry launch shapes: k = 3 (b - 1) + j, b = 1, 2 resident blocks per
// SM (capped by what fits), j: 1, 2, 4 work items per draw
static constexpr int kChemCandidates = 6;
static constexpr int kChemGrab[3] = {1, 2, 4};

static int check_params(const rt_params *p)
{
    if (!p) return fail(nullptr, RT_ERR_ARG, "params is NULL");
    if (p->ngroups < 1 || p->ngroups > RT_MAX_GROUPS)
        return fail(nullptr, RT_ERR_ARG, "ngroups=%d outside [1,%d]", p->ngroups, RT_MAX_GROUPS);
    for (int i = 0; i < p->ngroups; i++) {
        if (!(p->sigN[i] >= 0) || !(p->sigE[i] >= 0) || !(p->Eavg[i] >= 0) || !(p->frac[i] >= 0) ||
            !std::isfinite(p->sigN[i]) || !std::isfinite(p->sigE[i]) ||
            !std::isfinite(p->Eavg[i]) || !std::isfinite(p->frac[i]))
            return fail(nullptr, RT_ERR_ARG, "group %d table entries must be finite and >= 0", i);
    }
    if (!(p->c_red > 0) || !std::isfinite(p->c_red))
        return fail(nullptr, RT_ERR_ARG, "c_red must be > 0");
    if (!(p->cfl > 0 && p->cfl <= 1))
        return fail(nullptr, RT_ERR_ARG, "cfl=%g outside (0, 1]", p->cfl);
    if (p->nsub < 0) return fail(nullptr, RT_ERR_ARG, "nsub must be >= 0");
    if (p->max_halvings < 0 || p->max_halvings > 60)
        return fail(nullptr, RT_ERR_ARG, "max_halvings outside [0, 60]");
    if (p->precision < RT_PREC_SPLIT || p->precision > RT_PREC_FP64_STRICT)
        return fail(nullptr, RT_ERR_ARG, "unknown precision %d", p->precision);
    if (p->tune < 0) return fail(nullptr, RT_ERR_ARG, "tune must be >= 0");
    if (p->chem_tune < 0 || p->chem_tune >= 2 + kChemCandidates)
        return fail(nullptr, RT_ERR_ARG, "chem_tune %d outside [0, %d]", p->chem_tune, 1 + kChemCandidates);
    if (p->flux != RT_FLUX_GLF && p->flux != RT_FLUX_HLL)
        return fail(nullptr, RT_ERR_ARG, "unknown flux %d", p->flux);
    if (p->cosmo != 0 && p->cosmo != 1) return fail(nullptr, RT_ERR_ARG, "cosmo must be 0 or 1");
    if (p->cosmo && (!(p->a0 > 0.0) || !(p->H0 >= 0.0) || !(p->omega_m >= 0.0) ||
                     !(p->omega_l >= 0.0) || !(p->omega_m + p->omega_l > 0.0) ||
                     !std::isfinite(p->a0 + p->H0 + p->omega_m + p->omega_l)))
        return fail(nullptr, RT_ERR_ARG, "cosmo needs a0 > 0, H0 >= 0, omega_m, omega_l >= 0");
    for (int f = 0; f < 6; f++) {
        if (p->bc[f] < RT_BC_PERIODIC || p->bc[f] > RT_BC_INFLOW)
            return fail(nullptr, RT_ERR_ARG, "bc[%d]=%d unknown", f, p->bc[f]);
        if (p->bc[f] == RT_BC_INFLOW && f >= 2)
            return fail(nullptr, RT_ERR_ARG, "inflow boundaries on the x faces only");
        if (p->bc[f] == RT_BC_INFLOW && !(p->inflow[f] >= 0.0 && std::isfinite(p->inflow[f])))
            return fail(nullptr, RT_ERR_ARG, "inflow[%d] must be finite and >= 0", f);
    }
    for (int d = 0; d < 3; d++)
        if ((p->bc[2 * d] == RT_BC_PERIODIC) != (p->bc[2 * d + 1] == RT_BC_PERIODIC))
            return fail(nullptr, RT_ERR_ARG, "axis %d: periodic on one face only", d);
    if (p->rates_const && !p->isothermal)
        return fail(nullptr, RT_ERR_ARG, "rates_const requires isothermal (no cooling fits)");
    if (p->rates_const && (!(p->alphaA >= 0) || !(p->alphaB >= 0) || !(p->beta >= 0)))
        return fail(nullptr, RT_ERR_ARG, "constant rates must be >= 0");
    return RT_OK;
}

extern "C" double rt_timestep(const rt_params *p, double dx)
{
    if (!p || !(p->c_red > 0) || !(p->cfl > 0) || !(dx > 0)) return -1.0;
    // radiative Courant condition c <= dx/dt (Sec. 2.2.3) for the unsplit
    // 3-D update: dt = C dx / (3 c)
    return p->cfl * dx / (3.0 * p->c_red);
}

// ------------------------------------------------------------------ tuner
// Launch shape of the FP32 transport: tile (rtl::kTileX/Y) and grid.  Every
// candidate computes each cell with the same arithmetic, so the choice
// changes the time only.  Candidate k:
//   k = 3 t + (b - 1), k < 9: tile t at b = 1..3 resident blocks per SM
//     (capped by what fits), the grid b x SMs;
//   k = 9 + 2 t + (j - 1): tile t with j = 1, 2 blocks per tile column, so
//     the runs of neighbouring columns start at the same planes and each
//     reads its x/y halo while the neighbour's plane is still in L2.
//   k = 24 + 2 t + s: tile t in lockstep rows (groups of as many blocks as a
//     row has tiles, all of a group on the same planes of one row, so a
//     tile's x-halo lines are read by its neighbour at the same time), by
//     per-thread copies (s = 0) or TMA (s = 1); GLF only, and only when every
//     box has the same number of tile columns (else the default order);
//   k = 30 + t: tile t at the most resident blocks, planes loaded by TMA;
//   k = 15 + 3 t + c: tile t at the most resident blocks, the plane units in
//     z-chunks of 16, 32 or 64 planes (c = 0, 1, 2): a block's consecutive
//     runs are neighbouring tiles over the same planes, so a run's x-halo
//     lines were read as interior by the run before, still in L2 (whole
//     columns are far apart in time on large boxes and their halos come
//     from DRAM again).
// tune = 1 times every candidate on the handle's boxes (on a synthetic
// realizable state in scratch, so the caller's state is not touched) and
// keeps the fastest; the choice is cached per device, flux, group count and
// box set for later handles.  tune = 2 + k selects candidate k without timing.
struct TuneChoice {
    int variant, grid;
    int zlen;                 // z-chunk length of the unit order (0: whole columns)
    int lockx;                // lockstep rows: tile columns per row (0: off)
    bool tma;                 // GLF planes loaded by TMA
    int gpb = 1;              // GLF photon groups per block
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;
constexpr int kTuneCandidates = 13 * rtl::kTileVariants;
constexpr int kTuneChunk[3] = {16, 32, 64};

static void apply_layout(rt_handle *h, std::vector<rtd::BoxDev> &bd, int variant, int zlen = 0, int gpb = 1)
{
    int64_t titem = 0;
    for (auto &D : bd) {
        rtl::transport_layout(D, h->p.ngroups, variant, zlen, gpb);
        D.titem0 = titem;
        titem += D.ntitems;
    }
}

static int tgrid_of(int64_t ntitems, int blocks_per_sm, int nsm)
{
    // at least 4 planes per block (each run re-reads 2)
    return (int)std::max<int64_t>(1, std::min<int64_t>((ntitems + 3) / 4, (int64_t)blocks_per_sm * nsm));
}

static TuneChoice tune_candidate(rt_handle *h, int k, int nsm)
{
    constexpr int V = rtl::kTileVariants;
    const int v = k < 3 * V ? k / 3
                : k < 5 * V ? (k - 3 * V) / 2
                : k < 8 * V ? (k - 5 * V) / 3
                : k < 10 * V ? (k - 8 * V) / 2
                : k < 11 * V ? k - 10 * V
                : (k - 11 * V) / 2;
    const int occ = rtl::transport_occupancy(false, false, v, h->p.flux);
    const int occ_tma = rtl::transport_occupancy(false, false, v, h->p.flux, true);
    std::vector<rtd::BoxDev> bd = h->bdev;
    apply_layout(h, bd, v);
    int64_t nt = 0, ncol = 0;
    for (const auto &D : bd) {
        nt += D.ntitems;
        ncol += D.ntitems / D.nz;
    }
    const bool glf = h->p.flux == RT_FLUX_GLF;
    if (k >= 11 * V) {
        // two photon groups per block (GLF with G >= 2), column order or lockstep rows
        if (!glf || h->p.ngroups < 2) return {v, tgrid_of(nt, occ, nsm), 0, 0, false};
        std::vector<rtd::BoxDev> b2 = h->bdev;
        apply_layout(h, b2, v, 0, 2);
        int64_t nt2 = 0;
        for (const auto &D : b2) nt2 += D.ntitems;
        const int occ2 = rtl::transport_occupancy(false, false, v, h->p.flux, false, 2);
        TuneChoice c{v, tgrid_of(nt2, occ2, nsm), 0, 0, false};
        c.gpb = 2;
        if ((k - 11 * V) % 2 == 1) {
            const int tx = b2[0].tiles_x;
            bool same = true;
            for (const auto &D : b2) same = same && D.tiles_x == tx;
            const int m = (occ2 * nsm) / tx;
            if (same && m >= 1) {
                c.grid = m * tx;
                c.lockx = tx;
            }
        }
        return c;
    }
    if (k < 3 * V) return {v, tgrid_of(nt, std::min(k % 3 + 1, occ), nsm), 0, 0, false};
    if (k >= 10 * V) return {v, tgrid_of(nt, glf ? occ_tma : occ, nsm), 0, 0, glf};
    if (k >= 8 * V) {
        const int tx = bd[0].tiles_x;
        bool same = glf;
        for (const auto &D : bd) same = same && D.tiles_x == tx;
        const bool tma = glf && (k - 8 * V) % 2 == 1;
        const int m = ((tma ? occ_tma : occ) * nsm) / tx;
        if (!same || m < 1) return {v, tgrid_of(nt, occ, nsm), 0, 0, false};
        return {v, m * tx, 0, tx, tma};
    }
    if (k >= 5 * V) return {v, tgrid_of(nt, occ, nsm), kTuneChunk[(k - 5 * V) % 3], 0, false};
    const int64_t j = (k - 3 * V) % 2 + 1;
    const int64_t g = std::min<int64_t>(j * ncol, (int64_t)occ * nsm);
    return {v, (int)std::max<int64_t>(1, std::min<int64_t>(g, (nt + 3) / 4)), 0, 0, false};
}

// TMA tensor maps of descriptors bd (tile shape `variant`) written to the
// device buffer dmaps (3 x 128 bytes per box); true when every box has them
static bool build_tmaps(rt_handle *h, std::vector<rtd::BoxDev> &bd, int variant, void *dmaps)
{
    for (auto &D : bd) D.tmap = nullptr;
    if (h->fp64 || h->p.flux != RT_FLUX_GLF || !dmaps) return false;
    struct alignas(64) Maps { unsigned char b[384]; };                // a box's three maps
    std::vector<Maps> buf(bd.size());
    for (size_t b = 0; b < bd.size(); b++)
        if (!rtl::transport_tensor_maps(bd[b], h->p.ngroups, variant, buf[b].b)) return false;
    if (cudaMemcpy(dmaps, buf.data(), buf.size() * sizeof(Maps), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (size_t b = 0; b < bd.size(); b++) bd[b].tmap = static_cast<char *>(dmaps) + 384 * b;
    return true;
}

// the handle's maps for its current layout when `want` (allocated once per
// handle); without them the transport copies per thread
static int setup_tma(rt_handle *h, bool want)
{
    h->tma = false;
    for (auto &D : h->bdev) D.tmap = nullptr;
    if (!want || h->fp64 || h->p.flux != RT_FLUX_GLF) return RT_OK;
    if (!h->d_tmaps) CU(h, cudaMalloc(&h->d_tmaps, (size_t)384 * h->nboxes));
    h->tma = build_tmaps(h, h->bdev, h->tvariant, h->d_tmaps);
    return RT_OK;
}

static int tune_transport(rt_handle *h, int tune, int dev, int nsm)
{
    std::vector<TuneChoice> cand;
    for (int k = 0; k < kTuneCandidates; k++) {
        const TuneChoice c = tune_candidate(h, k, nsm);
        bool dup = false;
        for (const auto &o : cand)
            dup |= o.variant == c.variant && o.grid == c.grid && o.zlen == c.zlen && o.lockx == c.lockx &&
                   o.tma == c.tma && o.gpb == c.gpb;
        if (!dup) cand.push_back(c);
    }
    std::string key = std::to_string(dev) + "/" + std::to_string(h->p.flux) + "/" + std::to_string(h->p.ngroups);
    for (const auto &D : h->bdev)
        key += "/" + std::to_string(D.nx) + "x" + std::to_string(D.ny) + "x" + std::to_string(D.nz);
    TuneChoice best{0, 1, 0, 0, false};
    bool have = false;
    if (tune >= 2) {
        if (tune - 2 >= kTuneCandidates)
            return fail(h, RT_ERR_ARG, "tune %d: only %d launch shapes", tune, kTuneCandidates);
        best = tune_candidate(h, tune - 2, nsm);
        have = true;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { best = it->second; have = true; }
    }
    if (!have) {
        // scratch copy of the descriptors whose U is a synthetic state
        int64_t nU = 0;
        for (const auto &D : h->bdev) nU += (int64_t)h->p.ngroups * D.ncell;
        void *tU = nullptr, *tmaps = nullptr;
        rtd::BoxDev *tbox = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        auto cleanup = [&]() {
            cudaFree(tU);
            cudaFree(tmaps);
            cudaFree(tbox);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        };
        int rc = [&]() -> int {
            CU(h, cudaMalloc(&tU, (size_t)nU * 16));
            CU(h, cudaMalloc(&tbox, sizeof(rtd::BoxDev) * h->nboxes));
            if (h->p.flux == RT_FLUX_GLF) CU(h, cudaMalloc(&tmaps, (size_t)384 * h->nboxes));
            CU(h, cudaEventCreate(&e0));
            CU(h, cudaEventCreate(&e1));
            CU(h, rtl::fill_tune_state(tU, nU, h->s));
            std::vector<rtd::BoxDev> bd = h->bdev;
            int64_t off = 0;
            for (auto &D : bd) {
                D.U = (char *)tU + off * 16;
                off += (int64_t)h->p.ngroups * D.ncell;
            }
            float best_ms = 0.f;
            for (const auto &c : cand) {
                apply_layout(h, bd, c.variant, c.zlen, c.gpb);
                int64_t nt = 0;
                for (const auto &D : bd) nt += D.ntitems;
                CU(h, cudaStreamSynchronize(h->s));               // the maps' buffer is rewritten
                const bool tma = c.tma && build_tmaps(h, bd, c.variant, tmaps);
                if (!tma)
                    for (auto &D : bd) D.tmap = nullptr;
                CU(h, cudaMemcpyAsync(tbox, bd.data(), sizeof(rtd::BoxDev) * h->nboxes,
                                      cudaMemcpyHostToDevice, h->s));
                rtl::Launch L{tbox, h->nboxes, nt, c.grid, h->s, c.variant};
                L.tma = tma;
                L.lockstep = c.lockx;
                L.gpb = c.gpb;
                CU(h, rtl::transport_fast(false, L, h->zc, h->ph, h->d_ctl));      // warm-up
                CU(h, cudaEventRecord(e0, h->s));
                for (int r = 0; r < 5; r++) CU(h, rtl::transport_fast(false, L, h->zc, h->ph, h->d_ctl));
                CU(h, cudaEventRecord(e1, h->s));
                CU(h, cudaEventSynchronize(e1));
                float ms = 0.f;
                CU(h, cudaEventElapsedTime(&ms, e0, e1));
                if (!have || ms < best_ms) { best = c; best_ms = ms; have = true; }
            }
            return RT_OK;
        }();
        cleanup();
        if (rc) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    apply_layout(h, h->bdev, best.variant, best.zlen, best.gpb);
    h->ntitems = 0;
    for (const auto &D : h->bdev) h->ntitems += D.ntitems;
    h->tvariant = best.variant;
    h->tgrid = best.grid;
    h->tzlen = best.zlen;
    h->tlock = best.lockx;
    h->tgpb = best.gpb;
    if (int rc2 = setup_tma(h, best.tma)) return rc2;
    CU(h, cudaMemcpy(h->d_boxes, h->bdev.data(), sizeof(rtd::BoxDev) * h->nboxes, cudaMemcpyHostToDevice));
    return RT_OK;
}

// chemistry launch shape k (grid and work items per draw)
static void chem_candidate(const rt_handle *h, int k, int &grid, int &grab)
{
    const int b = std::min(k / 3 + 1, std::max(h->chem_occ, 1));
    grab = kChemGrab[k % 3];
    const int64_t wpb = RTD_CHEM_BLOCK / 32;             // warps (work items) per block
    grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->ncitems + wpb - 1) / wpb, (int64_t)b * h->nsm));
}

static std::map<std::string, int> g_chem_cache;

// chem_tune = 2 + k fixes shape k; chem_tune = 1 times every shape on scratch
// copies of the boxes' state (x_HI, T, and U as the post-transport field; the
// outputs go to scratch, so the caller's state is not touched): one warm-up,
// then three launches each, CUDA events.  The shape does not enter any result
// (every cell's arithmetic and every sum's order are fixed), so the fastest is
// kept.  Supercomoving runs take the default (their a(t) table is filled per call).
static int tune_chem(rt_handle *h, int tune, int dev)
{
    int best = 0;
    if (tune >= 2) {
        best = tune - 2;
    } else if (!h->p.cosmo) {
        std::string key = std::to_string(dev) + "/" + std::to_string(h->fp64) + "/" +
                          std::to_string(h->p.ngroups) + "/" + std::to_string(h->p.ots);
        for (const auto &D : h->bdev)
            key += "/" + std::to_string(D.nx) + "x" + std::to_string(D.ny) + "x" + std::to_string(D.nz);
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_chem_cache.find(key);
            if (it != g_chem_cache.end()) { best = it->second; have = true; }
        }
        if (!have) {
            const size_t es = h->fp64 ? 8 : 4;
            const int G = h->p.ngroups;
            std::vector<void *> bufs;
            rtd::BoxDev *tbox = nullptr;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            auto cleanup = [&]() {
                for (void *q : bufs) cudaFree(q);
                cudaFree(tbox);
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
            };
            int rc = [&]() -> int {
                std::vector<rtd::BoxDev> bd = h->bdev;
                std::vector<double *> x0(h->nboxes), T0(h->nboxes);
                for (int b = 0; b < h->nboxes; b++) {
                    rtd::BoxDev &D = bd[b];
                    const size_t nU = (size_t)G * D.ncell * 4 * es;
                    void *uo = nullptr, *xs = nullptr, *ts = nullptr;
                    CU(h, cudaMalloc(&uo, nU));
                    bufs.push_back(uo);
                    CU(h, cudaMalloc(&xs, (size_t)D.ncell * 8));
                    bufs.push_back(xs);
                    CU(h, cudaMalloc(&ts, (size_t)D.ncell * 8));
                    bufs.push_back(ts);
                    // the library's post-transport scratch holds the caller's field
                    CU(h, cudaMemcpyAsync(D.Us, D.U, nU, cudaMemcpyDeviceToDevice, h->s));
                    x0[b] = D.xHI;
                    T0[b] = D.T;
                    D.U = uo;
                    D.xHI = static_cast<double *>(xs);
                    D.T = static_cast<double *>(ts);
                }
                auto restore = [&]() -> int {
                    for (int b = 0; b < h->nboxes; b++) {
                        CU(h, cudaMemcpyAsync(bd[b].xHI, x0[b], (size_t)bd[b].ncell * 8, cudaMemcpyDeviceToDevice, h->s));
                        CU(h, cudaMemcpyAsync(bd[b].T, T0[b], (size_t)bd[b].ncell * 8, cudaMemcpyDeviceToDevice, h->s));
                    }
                    return RT_OK;
                };
                CU(h, cudaMalloc(&tbox, sizeof(rtd::BoxDev) * h->nboxes));
                CU(h, cudaMemcpyAsync(tbox, bd.data(), sizeof(rtd::BoxDev) * h->nboxes, cudaMemcpyHostToDevice, h->s));
                CU(h, cudaEventCreate(&e0));
                CU(h, cudaEventCreate(&e1));
                const rtd::DiagBuf db{h->d_partials, h->d_lanes, h->d_gpart, h->d_gdone, h->d_done, h->d_lastdiag};
                {
                    rtl::Launch Lk{tbox, h->nboxes, h->ncitems, 1, h->s};
                    CU(h, rtl::cconst_fast(h->fp64, Lk, h->ph, h->d_cc));
                }
                float best_ms = 0.f;
                for (int k = 0; k < kChemCandidates; k++) {
                    int grid, grab;
                    chem_candidate(h, k, grid, grab);
                    rtl::Launch L{tbox, h->nboxes, h->ncitems, grid, h->s};
                    L.grab = grab;
                    if (int r2 = restore()) return r2;
                    CU(h, rtl::chem_fast(h->fp64, G, L, h->ph, h->d_ctl, db));          // warm-up
                    if (int r2 = restore()) return r2;
                    CU(h, cudaEventRecord(e0, h->s));
                    for (int r = 0; r < 3; r++) CU(h, rtl::chem_fast(h->fp64, G, L, h->ph, h->d_ctl, db));
                    CU(h, cudaEventRecord(e1, h->s));
                    CU(h, cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CU(h, cudaEventElapsedTime(&ms, e0, e1));
                    if (k == 0 || ms < best_ms) { best = k; best_ms = ms; }
                }
                // the timing launches' counters and diagnostics are not the run's
                CU(h, cudaMemsetAsync(h->d_ctl, 0, sizeof(rtd::Ctl), h->s));
                CU(h, cudaMemsetAsync(h->d_lastdiag, 0, sizeof(double) * RTD_NDIAG * h->nboxes, h->s));
                CU(h, cudaStreamSynchronize(h->s));
                return RT_OK;
            }();
            cleanup();
            if (rc) return rc;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_chem_cache[key] = best;
        }
    }
    chem_candidate(h, best, h->cgrid, h->cgrab);
    return RT_OK;
}

extern "C" int rt_create(rt_handle **hout, const rt_params *p, const rt_box *boxes, int nboxes,
                         void *stream)
{
    try {
        if (!hout) return fail(nullptr, RT_ERR_ARG, "handle pointer is NULL");
        int rc = check_params(p);
        if (rc) return rc;
        if (nboxes < 1 || !boxes) return fail(nullptr, RT_ERR_ARG, "need at least one box");
        const bool fp64 = p->precision != RT_PREC_SPLIT;
        const size_t es = fp64 ? 8 : 4;
        for (int b = 0; b < nboxes; b++) {
            const rt_box &B = boxes[b];
            if (B.nx < 1 || B.ny < 1 || B.nz < 1)
                return fail(nullptr, RT_ERR_ARG, "box %d: sizes must be >= 1", b);
            if ((int64_t)B.nx * B.ny * B.nz > ((int64_t)1 << 40))
                return fail(nullptr, RT_ERR_ARG, "box %d too large", b);
            if (!(B.dx > 0) || !std::isfinite(B.dx) || !(B.nunit > 0) || !std::isfinite(B.nunit))
                return fail(nullptr, RT_ERR_ARG, "box %d: dx and nunit must be > 0", b);
            if (!B.U || !B.xHI || !B.T || !B.n0)
                return fail(nullptr, RT_ERR_ARG, "box %d: NULL state pointer", b);
            if (((uintptr_t)B.U % 16) || ((uintptr_t)B.xHI % 8) || ((uintptr_t)B.T % 8) ||
                ((uintptr_t)B.n0 % es))
                return fail(nullptr, RT_ERR_ARG, "box %d: misaligned state pointer", b);
            for (const void *q : {(const void *)B.U, (const void *)B.xHI, (const void *)B.T, B.n0}) {
                cudaPointerAttributes a;
                if (cudaPointerGetAttributes(&a, q) != cudaSuccess ||
                    (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
                    cudaGetLastError();
                    return fail(nullptr, RT_ERR_ARG, "box %d: state pointer is not device memory", b);
                }
            }
        }
        rt_handle *h = new (std::nothrow) rt_handle;
        if (!h) return fail(nullptr, RT_ERR_ARG, "out of host memory");
        h->p = *p;
        h->nboxes = nboxes;
        h->fp64 = fp64;
        h->strict = p->precision == RT_PREC_FP64_STRICT;
        h->esize = es;
        h->box.assign(boxes, boxes + nboxes);
        h->user = (cudaStream_t)stream;
        auto bail = [&](int code) { g_create_err = h->err; release(h); return code; };

        rtd::Phys &ph = h->ph;
        std::memset(&ph, 0, sizeof ph);
        ph.G = p->ngroups;
        ph.ots = p->ots;
        ph.isothermal = p->isothermal;
        ph.nsub = p->nsub;
        ph.rates_const = p->rates_const;
        ph.max_halvings = p->max_halvings;
        ph.c = p->c_red;
        for (int i = 0; i < p->ngroups; i++) {
            ph.csig[i] = p->c_red * p->sigN[i];
            ph.csig_f[i] = (float)ph.csig[i];
            ph.SigE[i] = p->sigE[i] * p->Eavg[i] - p->sigN[i] * (13.6 * rtd::EV);
            ph.hK[i] = (float)std::fabs(p->c_red * ph.SigE[i] / (1.5 * rtd::KB));
        }
        ph.alphaA = p->alphaA;
        ph.alphaB = p->alphaB;
        ph.beta = p->beta;
        const double fit_scale[5] = {0.522, 2.740, 0.354, 0.541, 2.250};
        for (int k = 0; k < 5; k++) ph.lnfit[k] = std::log(fit_scale[k]);
        ph.ln2THI = std::log(2.0 * rtd::T_HI);
        for (int f = 0; f < 6; f++) ph.bc[f] = p->bc[f];
        for (int f = 0; f < 2; f++)                      // inflow: c N per group, per unit nunit
            for (int i = 0; i < p->ngroups; i++)
                ph.inflow_c[f][i] = p->bc[f] == RT_BC_INFLOW ? p->inflow[f] * p->frac[i] / p->c_red : 0.0;

        if ((rc = [&]() -> int {
                CU(h, cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
                CU(h, cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
                CU(h, cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
                const int G = p->ngroups;
                int64_t titem = 0, citem = 0, cgroup = 0;
                h->bdev.resize(nboxes);
                h->d_us.assign(nboxes, nullptr);
                h->d_src_cell.assign(nboxes, nullptr);
                h->d_src_S.assign(nboxes, nullptr);
                h->src_uidx.assign(nboxes, std::vector<int>());
                for (int b = 0; b < nboxes; b++) {
                    const rt_box &B = boxes[b];
                    rtd::BoxDev &D = h->bdev[b];
                    std::memset(&D, 0, sizeof D);
                    D.nx = B.nx; D.ny = B.ny; D.nz = B.nz;
                    D.ncell = (int64_t)B.nx * B.ny * B.nz;
                    D.dx = B.dx;
                    D.nunit = B.nunit;
                    D.inv_nunit = 1.0 / B.nunit;
                    D.nunit_f = (float)B.nunit;
                    for (int i = 0; i < RTD_MAXG; i++) {
                        D.gN[i] = i < G ? h->ph.csig[i] * B.nunit : 0.0;
                        D.hN[i] = i < G ? h->ph.c * B.nunit * h->ph.SigE[i] : 0.0;
                    }
                    D.dt = p->cfl * B.dx / (3.0 * p->c_red);
                    D.lam = p->c_red * D.dt / B.dx;
                    D.U = B.U;
                    D.xHI = B.xHI;
                    D.T = B.T;
                    D.n0 = B.n0;
                    CU(h, cudaMalloc(&h->d_us[b], (size_t)G * D.ncell * 4 * es));
                    D.Us = h->d_us[b];
                    rtl::transport_layout(D, G);
                    D.titem0 = titem;
                    titem += D.ntitems;
                    D.citem0 = citem;
                    D.ncitems = (D.ncell + RTD_CHEM_ITEM * RTD_CHEM_LANE_CELLS - 1) /
                                (RTD_CHEM_ITEM * RTD_CHEM_LANE_CELLS);
                    citem += D.ncitems;
                    D.cgroup0 = cgroup;
                    D.ncgroups = (D.ncitems + RTD_CHEM_GROUP - 1) / RTD_CHEM_GROUP;
                    cgroup += D.ncgroups;
                }
                h->ntitems = titem;
                h->ncitems = citem;
                if (int rc2 = setup_tma(h, false)) return rc2;
                CU(h, cudaMalloc(&h->d_boxes, sizeof(rtd::BoxDev) * nboxes));
                CU(h, cudaMemcpy(h->d_boxes, h->bdev.data(), sizeof(rtd::BoxDev) * nboxes,
                                 cudaMemcpyHostToDevice));
                if (!h->strict) {
                    CU(h, cudaMalloc(&h->d_cc, sizeof(rtd::CellConst) * citem * RTD_CHEM_LANE_CELLS *
                                                   RTD_CHEM_ITEM));
                    h->ph.cc = h->d_cc;
                }
                CU(h, cudaMalloc(&h->d_partials, sizeof(rtd::DiagPart) * citem));
                CU(h, cudaMalloc(&h->d_lanes, sizeof(double) * 2 * RTD_CHEM_ITEM * citem));
                CU(h, cudaMalloc(&h->d_gpart, sizeof(rtd::DiagPart) * cgroup));
                CU(h, cudaMalloc(&h->d_gdone, sizeof(unsigned) * cgroup));
                CU(h, cudaMemset(h->d_gdone, 0, sizeof(unsigned) * cgroup));
                CU(h, cudaMalloc(&h->d_done, sizeof(unsigned) * nboxes));
                CU(h, cudaMemset(h->d_done, 0, sizeof(unsigned) * nboxes));
                if (!p->rates_const) {
                    std::vector<rtd::RateCoef> tab(rtl::rate_table_entries());
                    if (rtl::build_rate_table(p->ots != 0, tab.data())) {
                        // the 2^(j/64) table of the fast forms' exp follows the rate table
                        const size_t tb = sizeof(rtd::RateCoef) * tab.size();
                        double2 e2[64];
                        rtl::build_exp2_table(e2);
                        CU(h, cudaMalloc(&h->d_rtab, tb + sizeof(e2)));
                        CU(h, cudaMemcpy(reinterpret_cast<char *>(h->d_rtab) + tb, e2, sizeof(e2),
                                         cudaMemcpyHostToDevice));
                        h->ph.e2t = reinterpret_cast<const double2 *>(reinterpret_cast<char *>(h->d_rtab) + tb);
                        CU(h, cudaMemcpy(h->d_rtab, tab.data(), sizeof(rtd::RateCoef) * tab.size(),
                                         cudaMemcpyHostToDevice));
                        h->ph.rtab = h->d_rtab;
                    }
                }
                h->ph.flux = p->flux;
                if (p->cosmo) {
                    for (int b = 1; b < nboxes; b++)
                        if (boxes[b].dx != boxes[0].dx)
                            return fail(h, RT_ERR_ARG, "cosmo: every box needs the same dx");
                    CU(h, cudaMalloc(&h->d_acos, sizeof(double) * (kCosmoChunk + 1)));
                    CU(h, cudaMallocHost(&h->h_acos, sizeof(double) * (kCosmoChunk + 1)));
                    h->ph.cosmo = 1;
                    h->ph.acos = h->d_acos;
                    h->a_now = p->a0;
                }
                if (p->flux == RT_FLUX_HLL) {           // wave-speed table, FP64 and FP32 copies
                    const int nt = (RTD_HLL_NF + 1) * (RTD_HLL_NM + 1);
                    std::vector<double> td(nt);
                    std::vector<float> tf(nt);
                    if (rt_hll_speeds(RTD_HLL_NF, RTD_HLL_NM, td.data()) != RT_OK)
                        return fail(h, RT_ERR_ARG, "HLL speed table");
                    for (int i = 0; i < nt; i++) tf[i] = (float)td[i];
                    // FP32 pairs (lambda_min, lambda_max) at (i, j) and
                    // (i, j + 1), lambda_min(f, mu_j) = -lambda_max(f, mu_{NM - j})
                    const int n4 = (RTD_HLL_NF + 1) * RTD_HLL_NM;
                    std::vector<float4> tf4(n4);
                    for (int i = 0; i <= RTD_HLL_NF; i++) {
                        const float *row = tf.data() + i * (RTD_HLL_NM + 1);
                        for (int j = 0; j < RTD_HLL_NM; j++)
                            tf4[i * RTD_HLL_NM + j] = make_float4(-row[RTD_HLL_NM - j], row[j],
                                                                  -row[RTD_HLL_NM - j - 1], row[j + 1]);
                    }
                    CU(h, cudaMalloc(&h->d_hll_f4, sizeof(float4) * n4));
                    CU(h, cudaMemcpy(h->d_hll_f4, tf4.data(), sizeof(float4) * n4, cudaMemcpyHostToDevice));
                    h->ph.hll_f4 = h->d_hll_f4;
                    CU(h, cudaMalloc(&h->d_hll_d, sizeof(double) * nt));
                    CU(h, cudaMalloc(&h->d_hll_f, sizeof(float) * nt));
                    CU(h, cudaMemcpy(h->d_hll_d, td.data(), sizeof(double) * nt, cudaMemcpyHostToDevice));
                    CU(h, cudaMemcpy(h->d_hll_f, tf.data(), sizeof(float) * nt, cudaMemcpyHostToDevice));
                    h->ph.hll_d = h->d_hll_d;
                    h->ph.hll_f = h->d_hll_f;
                }
                CU(h, cudaMalloc(&h->d_lastdiag, sizeof(double) * RTD_NDIAG * nboxes));
                CU(h, cudaMemset(h->d_lastdiag, 0, sizeof(double) * RTD_NDIAG * nboxes));
                CU(h, cudaMalloc(&h->d_ctl, sizeof(rtd::Ctl)));
                CU(h, cudaMemset(h->d_ctl, 0, sizeof(rtd::Ctl)));
                CU(h, cudaMallocHost(&h->h_ctl, sizeof(rtd::Ctl)));
                std::memset(h->h_ctl, 0, sizeof(rtd::Ctl));
                CU(h, cudaMallocHost(&h->h_lastdiag, sizeof(double) * RTD_NDIAG * nboxes));
                std::memset(h->h_lastdiag, 0, sizeof(double) * RTD_NDIAG * nboxes);
                int dev = 0, nsm = 1;
                CU(h, cudaGetDevice(&dev));
                CU(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
                const int to = rtl::transport_occupancy(fp64, h->strict, 0, p->flux);
                const int co = rtl::chem_occupancy(fp64, h->strict, G);
                // transport: at least 4 planes per block (each run re-reads 2)
                h->tgrid = (int)std::max<int64_t>(1, std::min<int64_t>((titem + 3) / 4, (int64_t)to * nsm));
                const int64_t wpb = RTD_CHEM_BLOCK / 32;         // warps (work items) per block
                h->cgrid = (int)std::min<int64_t>((citem + wpb - 1) / wpb, (int64_t)co * nsm);
                h->nsm = nsm;
                h->chem_occ = co;
                h->fdev.assign(nboxes, rtd::FineDev{});
                h->d_fparent.assign(nboxes, nullptr);
                CU(h, cudaMalloc(&h->d_fines, sizeof(rtd::FineDev) * nboxes));
                CU(h, cudaMemcpy(h->d_fines, h->fdev.data(), sizeof(rtd::FineDev) * nboxes,
                                 cudaMemcpyHostToDevice));
                if (!fp64 && p->tune > 0)
                    if (int rc2 = tune_transport(h, p->tune, dev, nsm)) return rc2;
                if (!h->strict && p->chem_tune > 0) return tune_chem(h, p->chem_tune, dev);
                return RT_OK;
            }()))
            return bail(rc);
        *hout = h;
        return RT_OK;
    } catch (...) {
        return fail(nullptr, RT_ERR_ARG, "unexpected host exception in rt_create");
    }
}

extern "C" int rt_set_sources(rt_handle *h, int box, int nsrc, const int64_t *cell, const double *Q)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    try {
        if (box < 0 || box >= h->nboxes) return fail(h, RT_ERR_ARG, "box %d out of range", box);
        if (nsrc < 0 || (nsrc > 0 && (!cell || !Q))) return fail(h, RT_ERR_ARG, "bad source arrays");
        rtd::BoxDev &D = h->bdev[box];
        const int G = h->p.ngroups;
        for (int k = 0; k < nsrc; k++) {
            if (cell[k] < 0 || cell[k] >= D.ncell)
                return fail(h, RT_ERR_ARG, "source %d: cell %lld outside [0, %lld)", k,
                            (long long)cell[k], (long long)D.ncell);
            if (!(Q[k] >= 0) || !std::isfinite(Q[k]))
                return fail(h, RT_ERR_ARG, "source %d: luminosity must be finite and >= 0", k);
        }
        // merge duplicates in list order: S_i = (sum_k Q_k frac_i) / (dx^3 nunit)
        std::vector<int> order(nsrc);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return cell[a] < cell[b]; });
        std::vector<int64_t> ucell;
        std::vector<double> sums;
        std::vector<int> uidx(nsrc);
        for (int j = 0; j < nsrc; j++) {
            const int k = order[j];
            if (ucell.empty() || ucell.back() != cell[k]) {
                ucell.push_back(cell[k]);
                sums.insert(sums.end(), G, 0.0);
            }
            uidx[k] = (int)ucell.size() - 1;
            double *s = &sums[(ucell.size() - 1) * G];
            for (int i = 0; i < G; i++) s[i] += Q[k] * h->p.frac[i];
        }
        const double vol = D.dx * D.dx * D.dx;
        for (double &v : sums) v = v / (vol * D.nunit);
        CU(h, cudaStreamSynchronize(h->s));
        cudaFree(h->d_src_cell[box]);
        cudaFree(h->d_src_S[box]);
        h->d_src_cell[box] = nullptr;
        h->d_src_S[box] = nullptr;
        const int nu = (int)ucell.size();
        if (nu > 0) {
            CU(h, cudaMalloc(&h->d_src_cell[box], sizeof(int64_t) * nu));
            CU(h, cudaMalloc(&h->d_src_S[box], sizeof(double) * nu * G));
            CU(h, cudaMemcpy(h->d_src_cell[box], ucell.data(), sizeof(int64_t) * nu,
                             cudaMemcpyHostToDevice));
            CU(h, cudaMemcpy(h->d_src_S[box], sums.data(), sizeof(double) * nu * G,
                             cudaMemcpyHostToDevice));
        }
        D.src_cell = h->d_src_cell[box];
        D.src_S = h->d_src_S[box];
        D.nsrc = nu;
        h->src_uidx[box] = uidx;
        CU(h, cudaMemcpy(h->d_boxes + box, &D, sizeof D, cudaMemcpyHostToDevice));
        return RT_OK;
    } catch (...) {
        return fail(h, RT_ERR_ARG, "unexpected host exception in rt_set_sources");
    }
}

// one step of the hot path on stream s: transport, then chemistry with the
// per-box diagnostics fused into it; ev (profiling) = 4 events recorded
// before, between and after the kernels (the third interval stays empty)
static cudaError_t enqueue_step(rt_handle *h, cudaStream_t s, cudaEvent_t *ev = nullptr,
                                bool fine = true)
{
    rtl::Launch Lt{h->d_boxes, h->nboxes, h->ntitems, h->tgrid, s, h->tvariant};
    Lt.tma = h->tma;
    Lt.lockstep = h->tlock;
    Lt.gpb = h->tgpb;
    rtl::Launch Lc{h->d_boxes, h->nboxes, h->ncitems, h->cgrid, s};
    Lc.grab = h->cgrab;
    const rtd::DiagBuf db{h->d_partials, h->d_lanes, h->d_gpart, h->d_gdone, h->d_done, h->d_lastdiag};
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    e = h->strict ? rtl::transport_strict(Lt, h->zc, h->ph, h->d_ctl)
                  : rtl::transport_fast(h->fp64, Lt, h->zc, h->ph, h->d_ctl);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    e = h->strict ? rtl::chem_strict(h->p.ngroups, Lc, h->ph, h->d_ctl, db)
                  : rtl::chem_fast(h->fp64, h->p.ngroups, Lc, h->ph, h->d_ctl, db);
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    if (fine && h->nfitems > 0) {           // CRTA fine level: reads U* of this step
        rtl::Launch Lf{h->d_boxes, h->nboxes, h->nfitems, h->fgrid, s};
        e = h->strict ? rtl::chem_fine_strict(h->p.ngroups, Lf, h->d_fines, h->ph, h->d_ctl)
                      : rtl::chem_fine_fast(h->fp64, h->p.ngroups, Lf, h->d_fines, h->ph, h->d_ctl);
        if (e != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[3], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

static int build_graph(rt_handle *h)
{
    cudaGraph_t g = nullptr;
    CU(h, cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < RT_GRAPH_STEPS && e == cudaSuccess; k++) e = enqueue_step(h, h->s);
    cudaError_t e2 = cudaStreamEndCapture(h->s, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(h, RT_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, RT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    return RT_OK;
}

extern "C" int rt_set_fine(rt_handle *h, int box, int64_t nfine, const int64_t *parent,
                           const void *n0, double *xHI, double *T)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    if (box < 0 || box >= h->nboxes) return fail(h, RT_ERR_ARG, "box %d out of range", box);
    if (nfine < 0) return fail(h, RT_ERR_ARG, "nfine < 0");
    if (nfine > 0 && (!parent || !n0 || !xHI || !T))
        return fail(h, RT_ERR_ARG, "NULL fine-level array");
    try {
        const int64_t ncell = h->bdev[box].ncell;
        std::vector<int64_t> hp((size_t)nfine);
        if (nfine > 0) {
            const void *ptrs[4] = {parent, n0, xHI, T};
            for (const void *q : ptrs) {
                cudaPointerAttributes a;
                if (cudaPointerGetAttributes(&a, q) != cudaSuccess ||
                    (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
                    cudaGetLastError();
                    return fail(h, RT_ERR_ARG, "fine-level arrays must be device memory");
                }
            }
            CU(h, cudaMemcpy(hp.data(), parent, sizeof(int64_t) * nfine, cudaMemcpyDeviceToHost));
            for (int64_t f = 0; f < nfine; f++)
                if (hp[f] < 0 || hp[f] >= ncell)
                    return fail(h, RT_ERR_ARG, "parent[%lld] = %lld outside [0, %lld)", (long long)f,
                                (long long)hp[f], (long long)ncell);
        }
        CU(h, cudaStreamSynchronize(h->s));             // no step in flight uses the old level
        cudaFree(h->d_fparent[box]);
        h->d_fparent[box] = nullptr;
        if (nfine > 0) {
            CU(h, cudaMalloc(&h->d_fparent[box], sizeof(int64_t) * nfine));
            CU(h, cudaMemcpy(h->d_fparent[box], hp.data(), sizeof(int64_t) * nfine,
                             cudaMemcpyHostToDevice));
        }
        rtd::FineDev &F = h->fdev[box];
        F.parent = h->d_fparent[box];
        F.n0 = nfine > 0 ? n0 : nullptr;
        F.xHI = nfine > 0 ? xHI : nullptr;
        F.T = nfine > 0 ? T : nullptr;
        F.nfine = nfine;
        int64_t item = 0;
        for (auto &D : h->fdev) {
            D.fitem0 = item;
            D.nfitems = (D.nfine + RTD_CHEM_ITEM - 1) / RTD_CHEM_ITEM;
            item += D.nfitems;
        }
        h->nfitems = item;
        const int64_t wpb = RTD_CHEM_BLOCK / 32;
        h->fgrid = (int)std::max<int64_t>(1, std::min<int64_t>((item + wpb - 1) / wpb,
                                                               (int64_t)h->chem_occ * h->nsm));
        CU(h, cudaMemcpy(h->d_fines, h->fdev.data(), sizeof(rtd::FineDev) * h->nboxes,
                         cudaMemcpyHostToDevice));
        if (h->graph) {                                 // re-captured with the new level
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        return RT_OK;
    } catch (...) {
        return fail(h, RT_ERR_ARG, "unexpected host exception in rt_set_fine");
    }
}

static int step_chunk(rt_handle *h, int nsteps, double *hist);

extern "C" int rt_step(rt_handle *h, int nsteps, double *hist)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    if (nsteps < 0) return fail(h, RT_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return RT_OK;
    if (hist) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hist) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(h, RT_ERR_ARG, "hist must be device memory or NULL");
        }
    }
    if (!h->p.cosmo) return step_chunk(h, nsteps, hist);
    int worst = RT_OK;
    for (int done = 0; done < nsteps; done += kCosmoChunk) {
        const int n = std::min(kCosmoChunk, nsteps - done);
        const int rc = step_chunk(h, n, hist ? hist + (size_t)done * h->nboxes * RTD_NDIAG : nullptr);
        if (rc == RT_ERR_ARG || rc == RT_ERR_CUDA || rc == RT_ERR_STATE) return rc;
        if (rc != RT_OK && worst == RT_OK) worst = rc;
    }
    return worst;
}

// nsteps (<= kCosmoChunk when cosmo) steps in one go
static int step_chunk(rt_handle *h, int nsteps, double *hist)
{
    rtd::Ctl *c = h->h_ctl;
    c->hist = hist;
    c->step = -1;
    c->nboxes = h->nboxes;
    c->err = 0;
    c->nclamp = 0;
    c->chem_next = 0;
    c->chem_fin = 0;
    CU(h, cudaEventRecord(h->ev_in, h->user));
    CU(h, cudaStreamWaitEvent(h->s, h->ev_in, 0));
    CU(h, cudaMemcpyAsync(h->d_ctl, c, sizeof(rtd::Ctl), cudaMemcpyHostToDevice, h->s));
    if (!h->strict) {                    // the chemistry's per-cell constants from n0, once per call
        rtl::Launch Lk{h->d_boxes, h->nboxes, h->ncitems, 1, h->s};
        CU(h, rtl::cconst_fast(h->fp64, Lk, h->ph, h->d_cc));
    }
    if (h->p.cosmo) {                    // a at the start of every step of this chunk
        const double dt_com = h->bdev[0].dt;
        h->h_acos[0] = h->a_now;
        for (int k = 0; k < nsteps; k++)
            h->h_acos[k + 1] = friedmann_step(h->h_acos[k], h->h_acos[k] * dt_com, h->p);
        CU(h, cudaMemcpyAsync(h->d_acos, h->h_acos, sizeof(double) * (nsteps + 1),
                              cudaMemcpyHostToDevice, h->s));
    }
    if (!h->graph && nsteps >= RT_GRAPH_STEPS) {
        int rc = build_graph(h);
        if (rc) return rc;
    }
    int done = 0;
    if (h->profiling) {
        while (h->prof_ev.size() < (size_t)4 * nsteps) {
            cudaEvent_t e;
            CU(h, cudaEventCreate(&e));
            h->prof_ev.push_back(e);
        }
        for (; done < nsteps; done++) CU(h, enqueue_step(h, h->s, &h->prof_ev[4 * (size_t)done]));
    } else {
        if (h->graph)
            for (; done + RT_GRAPH_STEPS <= nsteps; done += RT_GRAPH_STEPS)
                CU(h, cudaGraphLaunch(h->graph, h->s));
        for (; done < nsteps; done++) CU(h, enqueue_step(h, h->s));
    }
    CU(h, cudaMemcpyAsync(c, h->d_ctl, sizeof(rtd::Ctl), cudaMemcpyDeviceToHost, h->s));
    CU(h, cudaMemcpyAsync(h->h_lastdiag, h->d_lastdiag, sizeof(double) * RTD_NDIAG * h->nboxes,
                          cudaMemcpyDeviceToHost, h->s));
    CU(h, cudaEventRecord(h->ev_out, h->s));
    CU(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
    CU(h, cudaStreamSynchronize(h->s));
    if (h->profiling) {
        for (int k = 0; k < nsteps; k++) {
            for (int j = 0; j < 3; j++) {          // transport, chemistry (+ diagnostics), fine level
                if (j == 2 && h->nfitems == 0) continue;
                float ms = 0.f;
                CU(h, cudaEventElapsedTime(&ms, h->prof_ev[4 * (size_t)k + j],
                                           h->prof_ev[4 * (size_t)k + j + 1]));
                h->kernel_ms[j] += ms;
                h->kernel_launches[j] += 1;
            }
        }
    }
    h->steps_done += nsteps;
    if (h->p.cosmo) h->a_now = h->h_acos[nsteps];
    h->nclamp += c->nclamp;
    h->error_bits |= (int)c->err;
    if (c->err & RTD_ERR_SUBCYCLE)
        return fail(h, RT_ERR_SUBCYCLE, "chemistry sub-cycle cap reached (10%% rule)");
    if (c->err & RTD_ERR_NONFINITE) return fail(h, RT_ERR_NONFINITE, "non-finite xHI or T");
    if (c->err & RTD_ERR_REALIZ) return fail(h, RT_ERR_REALIZABILITY, "|F| > 1.01 cN after transport");
    return RT_OK;
}

// device buffers of rt_adjoint, freed on every exit path
struct AdjBufs {
    std::vector<void *> p;
    ~AdjBufs()
    {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    cudaError_t get(T **out, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T));
        if (e == cudaSuccess) p.push_back(q);
        *out = static_cast<T *>(q);
        return e;
    }
};

static bool is_device(const void *q)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" int rt_adjoint(rt_handle *h, const void *U0, const double *xHI0, const double *T0,
                          int nsteps, int ckpt_every, const double *dL_dX, double *dL_dQ,
                          double *dL_dn0)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    try {
        if (h->nboxes != 1) return fail(h, RT_ERR_ARG, "rt_adjoint needs a single-box handle");
        if (!h->fp64) return fail(h, RT_ERR_ARG, "rt_adjoint needs an FP64 precision form");
        if (h->p.flux != RT_FLUX_GLF) return fail(h, RT_ERR_ARG, "rt_adjoint needs the GLF flux");
        if (h->p.cosmo) return fail(h, RT_ERR_ARG, "rt_adjoint: no supercomoving units");
        for (int f = 0; f < 6; f++)
            if (h->p.bc[f] != RT_BC_PERIODIC)
                return fail(h, RT_ERR_ARG, "rt_adjoint needs periodic boundaries");
        if (nsteps < 1 || ckpt_every < 1) return fail(h, RT_ERR_ARG, "nsteps and ckpt_every must be >= 1");
        if (!U0 || !xHI0 || !T0 || !dL_dX || !dL_dn0 || !is_device(U0) || !is_device(xHI0) ||
            !is_device(T0) || !is_device(dL_dX) || !is_device(dL_dn0))
            return fail(h, RT_ERR_ARG, "U0, xHI0, T0, dL_dX and dL_dn0 must be device pointers");
        const rtd::BoxDev &D = h->bdev[0];
        const int G = h->p.ngroups;
        const int64_t ncell = D.ncell;
        const size_t nU = (size_t)G * ncell * 4;
        const int nsrc_given = (int)h->src_uidx[0].size();
        if (nsrc_given > 0 && !dL_dQ) return fail(h, RT_ERR_ARG, "dL_dQ is NULL but the box has sources");
        const int ck = std::min(ckpt_every, nsteps);
        const int nck = (nsteps + ck - 1) / ck;
        cudaStream_t s = h->s;
        AdjBufs B;
        double *ckU, *ckx, *ckT, *segU, *segUs, *segx, *segT, *lamU, *lamS, *lamx, *lamT, *dS = nullptr;
        double *endU, *endx, *endT;
        unsigned *derr;
        CU(h, B.get(&ckU, nU * nck));
        CU(h, B.get(&ckx, (size_t)ncell * nck));
        CU(h, B.get(&ckT, (size_t)ncell * nck));
        CU(h, B.get(&segU, nU * ck));
        CU(h, B.get(&segUs, nU * ck));
        CU(h, B.get(&segx, (size_t)ncell * ck));
        CU(h, B.get(&segT, (size_t)ncell * ck));
        CU(h, B.get(&lamU, nU));
        CU(h, B.get(&lamS, nU));
        CU(h, B.get(&lamx, (size_t)ncell));
        CU(h, B.get(&lamT, (size_t)ncell));
        CU(h, B.get(&endU, nU));
        CU(h, B.get(&endx, (size_t)ncell));
        CU(h, B.get(&endT, (size_t)ncell));
        CU(h, B.get(&derr, 1));
        if (D.nsrc > 0) CU(h, B.get(&dS, (size_t)D.nsrc * G));
        std::vector<double> dLdX(nsteps);
        const size_t bU = nU * sizeof(double), bS = (size_t)ncell * sizeof(double);

        CU(h, cudaEventRecord(h->ev_in, h->user));
        CU(h, cudaStreamWaitEvent(s, h->ev_in, 0));
        CU(h, cudaMemcpyAsync(dLdX.data(), dL_dX, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, s));
        rtd::Ctl *c = h->h_ctl;
        c->hist = nullptr;
        c->step = -1;
        c->nboxes = 1;
        c->err = 0;
        c->nclamp = 0;
        c->chem_next = 0;
        c->chem_fin = 0;
        CU(h, cudaMemcpyAsync(h->d_ctl, c, sizeof(rtd::Ctl), cudaMemcpyHostToDevice, s));
        if (!h->strict) {                // the chemistry's per-cell constants from n0
            rtl::Launch Lk{h->d_boxes, h->nboxes, h->ncitems, 1, s};
            CU(h, rtl::cconst_fast(h->fp64, Lk, h->ph, h->d_cc));
        }
        // forward from (U0, xHI0, T0) with a checkpoint every ck steps
        CU(h, cudaMemcpyAsync(D.U, U0, bU, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(D.xHI, xHI0, bS, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(D.T, T0, bS, cudaMemcpyDeviceToDevice, s));
        for (int k = 0; k < nsteps; k++) {
            if (k % ck == 0) {
                const int q = k / ck;
                CU(h, cudaMemcpyAsync(ckU + nU * q, D.U, bU, cudaMemcpyDeviceToDevice, s));
                CU(h, cudaMemcpyAsync(ckx + ncell * q, D.xHI, bS, cudaMemcpyDeviceToDevice, s));
                CU(h, cudaMemcpyAsync(ckT + ncell * q, D.T, bS, cudaMemcpyDeviceToDevice, s));
            }
            CU(h, enqueue_step(h, s, nullptr, false));
        }
        CU(h, cudaMemcpyAsync(endU, D.U, bU, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(endx, D.xHI, bS, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(endT, D.T, bS, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaStreamSynchronize(s));          // dLdX is on the host from here
        // reverse, one checkpoint segment at a time
        CU(h, cudaMemsetAsync(lamU, 0, bU, s));
        CU(h, cudaMemsetAsync(lamx, 0, bS, s));
        CU(h, cudaMemsetAsync(lamT, 0, bS, s));
        CU(h, cudaMemsetAsync(dL_dn0, 0, bS, s));
        CU(h, cudaMemsetAsync(derr, 0, sizeof(unsigned), s));
        if (dS) CU(h, cudaMemsetAsync(dS, 0, sizeof(double) * D.nsrc * G, s));
        for (int q = nck - 1; q >= 0; q--) {
            const int k0 = q * ck, k1 = std::min(nsteps, k0 + ck);
            CU(h, cudaMemcpyAsync(D.U, ckU + nU * q, bU, cudaMemcpyDeviceToDevice, s));
            CU(h, cudaMemcpyAsync(D.xHI, ckx + ncell * q, bS, cudaMemcpyDeviceToDevice, s));
            CU(h, cudaMemcpyAsync(D.T, ckT + ncell * q, bS, cudaMemcpyDeviceToDevice, s));
            for (int k = k0; k < k1; k++) {       // recompute the segment, keeping every state
                const int j = k - k0;
                CU(h, cudaMemcpyAsync(segU + nU * j, D.U, bU, cudaMemcpyDeviceToDevice, s));
                CU(h, cudaMemcpyAsync(segx + ncell * j, D.xHI, bS, cudaMemcpyDeviceToDevice, s));
                CU(h, cudaMemcpyAsync(segT + ncell * j, D.T, bS, cudaMemcpyDeviceToDevice, s));
                CU(h, enqueue_step(h, s, nullptr, false));
                CU(h, cudaMemcpyAsync(segUs + nU * j, D.Us, bU, cudaMemcpyDeviceToDevice, s));
            }
            for (int k = k1 - 1; k >= k0; k--) {
                const int j = k - k0;
                const double gx = -dLdX[k] / (double)ncell;   // X(k+1) = mean(1 - xHI)
                CU(h, rtl::chem_adj(G, h->d_boxes, h->ph, segUs + nU * j, segx + ncell * j,
                                    segT + ncell * j, lamU, lamx, lamT, gx, dL_dn0, dS, derr, ncell, s));
                CU(h, rtl::transport_adj(G, h->d_boxes, segU + nU * j, lamU, lamS, ncell, s));
                std::swap(lamU, lamS);
            }
        }
        // leave the box at the end of the forward run
        CU(h, cudaMemcpyAsync(D.U, endU, bU, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(D.xHI, endx, bS, cudaMemcpyDeviceToDevice, s));
        CU(h, cudaMemcpyAsync(D.T, endT, bS, cudaMemcpyDeviceToDevice, s));
        std::vector<double> hS((size_t)D.nsrc * G);
        if (dS) CU(h, cudaMemcpyAsync(hS.data(), dS, sizeof(double) * hS.size(), cudaMemcpyDeviceToHost, s));
        unsigned herr = 0;
        CU(h, cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CU(h, cudaMemcpyAsync(c, h->d_ctl, sizeof(rtd::Ctl), cudaMemcpyDeviceToHost, s));
        CU(h, cudaEventRecord(h->ev_out, s));
        CU(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
        CU(h, cudaStreamSynchronize(s));
        // S_i = (sum_k Q_k frac_i) / (dx^3 nunit)  =>  dL/dQ_k = sum_i frac_i dL/dS_i / (dx^3 nunit)
        const double vol = D.dx * D.dx * D.dx;
        for (int k = 0; k < nsrc_given; k++) {
            const int u = h->src_uidx[0][k];
            double g = 0.0;
            for (int i = 0; i < G; i++) g += h->p.frac[i] * hS[(size_t)u * G + i];
            dL_dQ[k] = g / (vol * D.nunit);
        }
        if ((herr | c->err) & RTD_ERR_SUBCYCLE)
            return fail(h, RT_ERR_SUBCYCLE, "adjoint: a cell-step needed more than 2048 sub-cycles "
                                            "or hit the halving cap");
        if (c->err & RTD_ERR_NONFINITE) return fail(h, RT_ERR_NONFINITE, "non-finite xHI or T");
        return RT_OK;
    } catch (...) {
        return fail(h, RT_ERR_ARG, "unexpected host exception in rt_adjoint");
    }
}

static int copy_state(rt_handle *h, int box, bool up, void *U, double *xHI, double *T, void *n0)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    if (box < 0 || box >= h->nboxes) return fail(h, RT_ERR_ARG, "box %d out of range", box);
    const rtd::BoxDev &D = h->bdev[box];
    const size_t nU = (size_t)h->p.ngroups * D.ncell * 4 * h->esize;
    const size_t nS = (size_t)D.ncell * sizeof(double);
    const cudaMemcpyKind k = up ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    CU(h, cudaEventRecord(h->ev_in, h->user));
    CU(h, cudaStreamWaitEvent(h->s, h->ev_in, 0));
    if (U) CU(h, up ? cudaMemcpyAsync(D.U, U, nU, k, h->s) : cudaMemcpyAsync(U, D.U, nU, k, h->s));
    if (xHI) CU(h, up ? cudaMemcpyAsync(D.xHI, xHI, nS, k, h->s) : cudaMemcpyAsync(xHI, D.xHI, nS, k, h->s));
    if (T) CU(h, up ? cudaMemcpyAsync(D.T, T, nS, k, h->s) : cudaMemcpyAsync(T, D.T, nS, k, h->s));
    if (n0 && up)
        CU(h, cudaMemcpyAsync(const_cast<void *>(D.n0), n0, (size_t)D.ncell * h->esize, k, h->s));
    CU(h, cudaEventRecord(h->ev_out, h->s));
    CU(h, cudaStreamWaitEvent(h->user, h->ev_out, 0));
    CU(h, cudaStreamSynchronize(h->s));
    return RT_OK;
}

extern "C" int rt_upload(rt_handle *h, int box, const void *U, const double *xHI, const double *T,
                         const void *n0)
{
    return copy_state(h, box, true, const_cast<void *>(U), const_cast<double *>(xHI),
                      const_cast<double *>(T), const_cast<void *>(n0));
}

extern "C" int rt_download(rt_handle *h, int box, void *U, double *xHI, double *T)
{
    return copy_state(h, box, false, U, xHI, T, nullptr);
}

extern "C" int rt_set_profiling(rt_handle *h, int on)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    h->profiling = on != 0;
    for (int j = 0; j < 3; j++) {
        h->kernel_ms[j] = 0.0;
        h->kernel_launches[j] = 0;
    }
    return RT_OK;
}

extern "C" int rt_query(rt_handle *h, rt_stats *st)
{
    if (!h) return fail(nullptr, RT_ERR_STATE, "NULL handle");
    if (!st) return fail(h, RT_ERR_ARG, "stats pointer is NULL");
    std::memset(st, 0, sizeof *st);
    st->steps = h->steps_done;
    st->realizability_clamps = (int64_t)h->nclamp;
    st->error_bits = h->error_bits;
    st->nboxes = h->nboxes;
    for (const auto &D : h->bdev) st->cells += D.ncell;
    for (int k = 0; k < RT_NDIAG; k++) st->last_diag[k] = h->h_lastdiag[k];
    for (int j = 0; j < 3; j++) {
        st->kernel_ms[j] = h->kernel_ms[j];
        st->kernel_launches[j] = h->kernel_launches[j];
    }
    const int v = h->fp64 ? 0 : h->tvariant;
    st->tile_x = rtl::kTileX[v];
    st->tile_y = rtl::kTileY[v];
    st->transport_grid = h->tgrid;
    st->transport_zchunk = h->fp64 ? 0 : h->tzlen;
    st->transport_tma = h->tma ? 1 : 0;
    st->transport_lockstep = h->fp64 ? 0 : h->tlock;
    st->chem_grid = h->cgrid;
    st->chem_grab = h->cgrab;
    st->transport_gpb = h->tgpb;
    st->a = h->p.cosmo ? h->a_now : 1.0;
    return RT_OK;
}

extern "C" const char *rt_last_error(rt_handle *h)
{
    return h ? h->err.c_str() : g_create_err.c_str();
}

extern "C" void rt_destroy(rt_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->s);
    release(h);
}
