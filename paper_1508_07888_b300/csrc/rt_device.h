// rt_device.h -- descriptors shared by the host side of librt_m1 and its
// kernels (internal; the public ABI is include/rt_m1.h).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#define RTD_MAXG 4
#define RTD_NDIAG 5

// transport tile: TX x TY threads, one (x, y) column each, marching in z
#define RTD_TX 32
#define RTD_TY 8
// chemistry: threads per block (independent warps, one cell per thread at a
// time), lanes of a work item (one warp), cells per lane in a coarse work
// item (the fine level's items have one), work items per diagnostics group
#define RTD_CHEM_BLOCK 256
#define RTD_CHEM_ITEM 32
#define RTD_CHEM_LANE_CELLS 4
#define RTD_CHEM_GROUP 64

// device error bits (OR-ed into Ctl::err)
#define RTD_ERR_NONFINITE 1u
#define RTD_ERR_REALIZ 2u
#define RTD_ERR_SUBCYCLE 4u
#define RTD_ERR_TIMEOUT 8u      // a bounded device wait (TMA arrival) gave up

#define RTD_MAXCYC 1000000   // sub-cycles per cell and step before giving up

// intercell flux (rt_flux) and the HLL wave-speed table size (rt_hll_speeds)
#define RTD_FLUX_GLF 0
#define RTD_FLUX_HLL 1
#define RTD_HLL_NF 64
#define RTD_HLL_NM 64

// rate tables: piecewise polynomials in T.  T in [2^E0, 2^E1) falls in
// interval j = 2^SUB (e - E0) + (top SUB bits of T's mantissa), e = T's binary
// exponent, so the index and the local variable t in [-1, 1) come from T's
// bits (no logarithm); 2^SUB equal intervals per binade (see rate_table.cu).
// Each polynomial p(t) = c0 + t (c1 + t (c2 + t q)) keeps c0 .. c2 in FP64
// and its tail q = c3 + t (c4 + t c5), terms below ~1e-6 of p, in FP32.
#define RTD_TAB_NF 5         // aA, aB, kR, ln(beta) + T_HI/T, ln(cce) + 118348/T
#define RTD_TAB_E0 0         // 1 K
#define RTD_TAB_E1 30        // 2^30 K = 1.07e9 K
#define RTD_TAB_SUB 6        // 64 intervals per binade
#define RTD_TAB_NINT ((RTD_TAB_E1 - RTD_TAB_E0) << RTD_TAB_SUB)
#define RTD_TAB_NC 6         // degree 5 in t
// below this temperature both exp(-T_HI/T) and exp(-118348/T) factors of the
// fits are exactly zero in double precision (checked when the table is built)
#define RTD_TAB_TCUT 155.0
// below this temperature beta < 1e-77 cm^3/s and kC / (1.5 kB T) < 2e-57
// cm^3/s, so in a cell with n0 dtau <= RTD_TAB_NDMAX (cm^-3 s) the
// collisional ionisation and cooling terms are below 2^-60 of the terms
// they enter (1 in the x_HI denominator, the internal energy), below any
// FP64 rounding; the chemistry then treats the cell as cold (both bounds
// checked when the table is built)
#define RTD_TAB_TWARM 1000.0
#define RTD_TAB_NDMAX 1e38f

namespace rtd {

// coefficients of one tabulated polynomial (one function on one interval)
struct RateCoef {
    double c0, c1, c2;
    float c3, c4, c5;
    float b32;      // entries 0, 1, 2 of an interval: c0, c1, c2 of alpha_B's polynomial in
                    // FP32 (with entry 1's c3 .. c5, alpha_B wholly in FP32); entry 3: an
                    // upper bound of kR over the interval in FP32 (the fast forms'
                    // pre-test); 0 in entry 4
};

// physical constants (cgs)
constexpr double KB = 1.380649e-16;         // erg/K
constexpr double EV = 1.602176634e-12;      // erg
constexpr double T_HI = 157807.0;           // K, temperature scale of the rate fits

// Per-cell constants of the fast forms' chemistry (n0 is static within an
// rt_step call): formed once per call by k_cconst, read by k_chem with the
// cell's other inputs.  n0, n0^2, n0^2 / nunit (0 with OTS), (3/2) kB n0 and
// 3 kB n0 in FP64, n0^2 / nunit in FP32.  Indexed by work item x 128 + the
// cell's place in the item.
struct CellConst {
    double n0, n02, K, cvn, cvn2;
    float K32, pad;
};

// Parameters shared by every box (kernel argument, by value).
struct Phys {
    int G;
    int ots, isothermal, nsub, rates_const, max_halvings;
    double c;                     // reduced speed of light, cm/s
    double csig[RTD_MAXG];        // c * sigma_N,i
    float csig_f[RTD_MAXG];       // the same rounded to FP32 (the split form's photon update)
    float hK[RTD_MAXG];           // |c Sigma_E,i| / (1.5 kB) in FP32 (the chemistry's FP32 pre-test)
    double SigE[RTD_MAXG];        // Sigma_E,i = sigma_E,i <E>_i - sigma_N,i E_13.6 (Sec. 2.2.4)
    double alphaA, alphaB, beta;  // rates_const values
    double lnfit[5];              // ln of the rate-fit scales 0.522, 2.740, 0.354, 0.541, 2.250
    double ln2THI;                // ln(2 T_HI)
    const RateCoef *rtab;         // rate table [RTD_TAB_NINT][RTD_TAB_NF] or null
    const double2 *e2t;           // 2^(j/64) as pairs (hi, lo), j = 0..63 (the fast forms' exp), or null
    const CellConst *cc;          // per-cell chemistry constants of the fast forms (k_cconst)
    int flux;                     // RTD_FLUX_GLF / RTD_FLUX_HLL
    const float *hll_f;           // HLL wave speeds [RTD_HLL_NF + 1][RTD_HLL_NM + 1], FP32 copy
    const double *hll_d;          // the same in FP64
    const float4 *hll_f4;         // FP32 (lambda_min, lambda_max) at (i, j) and (i, j+1), [NF + 1][NM] (k_transport_hll)
    int bc[6];                    // -x,+x,-y,+y,-z,+z
    double inflow_c[2][RTD_MAXG]; // inflow faces -x, +x: beam density N per group times nunit
    int cosmo;                    // supercomoving units: state comoving, chemistry at a(t)
    const double *acos;           // a at the start of each step of the current call, [nsteps + 1]
};

// One box (array in device memory, indexed by work items).
struct BoxDev {
    int nx, ny, nz;
    int tiles_x, tiles_y;             // transport tiling
    int zlen;                         // plane units ordered (group, y-tile, z-chunk of zlen
                                      // planes, x-tile, z); zlen = nz: whole columns
    int64_t ncell;
    double dx, nunit, dt, lam;        // lam = c dt / dx (Courant number)
    double inv_nunit;                 // 1 / nunit
    double gN[RTD_MAXG];              // c sigma_N,i nunit
    double hN[RTD_MAXG];              // c nunit Sigma_E,i
    void *U;                          // caller's state, [G][nz][ny][nx][4]
    void *Us;                         // post-transport state (library scratch)
    const void *tmap;                 // FP32 transport: three TMA tensor maps of U (the tile
                                      // with halo, a halo column, a halo row), 64-byte aligned
                                      // in device memory; null: per-thread copies
    double *xHI, *T;
    const void *n0;
    const int64_t *src_cell;          // sorted unique source cells (nsrc)
    const double *src_S;              // [nsrc][G] source term, stored units per second
    int nsrc;
    float nunit_f;                    // nunit in FP32 (the chemistry's FP32 pre-test)
    int64_t titem0, ntitems;          // transport plane units of this box (prefix, count)
    int64_t citem0, ncitems;          // chemistry work items (32 cells) of this box
    int64_t cgroup0, ncgroups;        // diagnostics groups (64 items) of this box
};

// Per-item diagnostic partials of the chemistry kernel and the per-box
// reduction state (the last item of a box to finish reduces the box).
struct DiagPart {
    double X, ph;                     // sum of (1 - xHI), sum of N over groups
    unsigned long long fbits;         // max |F|/N (bits of a non-negative double)
    unsigned long long count, ncyc;   // cells with xHI < 0.5, chemistry sub-cycles
};
struct DiagBuf {
    DiagPart *part;                   // one per chemistry work item (X, ph unused)
    double *lane;                     // per work item: its 32 lanes' (1 - xHI), then their photons
    DiagPart *gpart;                  // one per group of RTD_CHEM_GROUP items
    unsigned *gdone;                  // per group: items finished in this step
    unsigned *done;                   // per box: groups finished in this step
    double *last;                     // per box: RTD_NDIAG values of the last step
};

// Per-call control block in device memory.
struct Ctl {
    double *hist;                     // caller's [step][box][RTD_NDIAG] or nullptr
    int step;                         // step index within the current rt_step call
    int nboxes;
    unsigned int err;                 // RTD_ERR_* bits
    unsigned long long nclamp;        // post-transport flux-limit clamps
    unsigned long long chem_next;     // chemistry: next work item to hand out
    unsigned long long chem_fin;      // chemistry: warps that found no more work
    unsigned long long fine_next;     // CRTA fine level: next work item
    unsigned long long fine_fin;      // CRTA fine level: warps that found no more work
};

// CRTA fine level of one box: refined cells that run the chemistry with the
// post-transport radiation and the source of their coarse parent cell.
struct FineDev {
    const int64_t *parent;            // [nfine] parent's linear cell index (library copy)
    const void *n0;                   // [nfine] caller's densities (float SPLIT, double FP64)
    double *xHI, *T;                  // [nfine] caller's state, read/write
    int64_t nfine;
    int64_t fitem0, nfitems;          // work items (32 refined cells) of this box
};

}  // namespace rtd
