/*
 * rt_m1.h -- C ABI of the B300 M1 radiative-transfer library (librt_m1.so).
 *
 * One call of rt_step advances every box of a handle by explicit M1
 * radiative-transfer steps as described by Aubert, Deparis & Ocvirk,
 * "EMMA: an AMR cosmological simulation code with radiative transfer"
 * (arXiv:1508.07888):
 *   1. dt from the radiative Courant condition (Sec. 2.2.3, Sec. 2.3),
 *      read in 3-D as dt = cfl dx / (3 c);
 *   2. per photon group: Levermore M1 closure, GLF intercell fluxes and the
 *      unsplit conservative update (Sec. 2.2.3, Eqs. e:pdert1i, e:pdert2i,
 *      e:uprt, e:glf) with the boundary ghosts of Sec. 4.2;
 *   3. per cell: sub-cycled hydrogen thermochemistry -- sources and implicit
 *      absorption, ionisation and energy updates in the paper's order, with
 *      the 10% energy rule (Sec. 2.2.4, Eqs. e:therm1-e:therm4, e:therm1g,
 *      e:therm2g, e:g2, e:g3);
 *   4. per box: diagnostics (volume-weighted ionised fraction, photon
 *      total, max |F|/(cN), count of cells with xHI < 0.5 -- the front
 *      definition of Sec. 6.4 -- and mean chemistry sub-cycles per cell).
 *
 * Conventions
 *   - All functions return RT_OK (0) or a negative rt_status; no C++
 *     exception crosses this boundary.  rt_last_error() gives a message.
 *   - Device memory of the state belongs to the caller; the library never
 *     frees it.  The library allocates only its own scratch (the
 *     post-transport radiation state, source tables, reduction partials,
 *     the error word) and frees it in rt_destroy.
 *   - Work is ordered on the CUDA stream given to rt_create.  rt_step
 *     returns after the stream has drained (it reads the device error word).
 *   - Radiation state in the stored variables Nhat = N/nunit and
 *     Fhat = F/(c_red nunit) (photons/cm^3 scaled by the box's nunit), so
 *     the flux limit reads |Fhat| <= Nhat.
 *   - Layouts are C order: U[g][z][y][x][4] = (Nhat, Fhat_x, Fhat_y, Fhat_z),
 *     scalars [z][y][x]; linear cell index = (z*ny + y)*nx + x.
 */
#ifndef RT_M1_H
#define RT_M1_H

#include <stdint.h>

#if defined(__GNUC__)
#define RT_API __attribute__((visibility("default")))
#else
#define RT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define RT_MAX_GROUPS 4
#define RT_NDIAG 5          /* ionised fraction, photons, max f, n(xHI<0.5), mean sub-cycles */

typedef enum rt_status {
    RT_OK = 0,
    RT_ERR_ARG = -1,            /* invalid argument (message in rt_last_error) */
    RT_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    RT_ERR_NONFINITE = -3,      /* a cell's xHI or T became NaN/Inf */
    RT_ERR_REALIZABILITY = -4,  /* |F| > 1.01 cN after transport */
    RT_ERR_SUBCYCLE = -5,       /* 10% rule needed more than max_halvings halvings,
                                   or a cell exceeded 1e6 sub-cycles in one step */
    RT_ERR_TIMEOUT = -6,        /* reserved: a bounded device wait gave up */
    RT_ERR_STATE = -7,          /* call out of order (e.g. on a destroyed handle) */
    RT_ERR_TOO_LARGE = -8       /* rt_transport_static: the box does not fit its static scratch */
} rt_status;

typedef enum rt_precision {
    RT_PREC_SPLIT = 0,       /* FP32 transport (float U, float n0), FP64 chemistry */
    RT_PREC_FP64 = 1,        /* FP64 everywhere (double U, double n0) */
    RT_PREC_FP64_STRICT = 2  /* FP64, no fused multiply-add, the operation order of a
                                plain IEEE evaluation of the equations (bit-reproducible
                                against such an evaluation when rates_const is set) */
} rt_precision;

typedef enum rt_bc {
    RT_BC_PERIODIC = 0,      /* Sec. 4.2 default */
    RT_BC_TRANSMISSIVE = 1,  /* ghost = copy of the boundary cell */
    RT_BC_REFLECTIVE = 2,    /* ghost = copy with the normal flux component inverted */
    RT_BC_INFLOW = 3         /* ghost = a beam entering the box along the normal, F = c N,
                                carrying rt_params.inflow[face] photons/cm^2/s split over the
                                groups by frac (the clump test of Sec. 6.5); x faces only */
} rt_bc;

typedef enum rt_flux {
    RT_FLUX_GLF = 0,         /* global Lax-Friedrichs (Eq. e:glf), the paper's flux */
    RT_FLUX_HLL = 1          /* Harten-Lax-van Leer with the M1 signal speeds (the less
                                diffusive flux the paper plans, Sec. 2.2.3); see rt_hll_speeds */
} rt_flux;

typedef struct rt_params {
    int    ngroups;                      /* 1..RT_MAX_GROUPS */
    double sigN[RT_MAX_GROUPS];          /* cm^2, number-weighted group cross-section (Eq. e:siggroup) */
    double sigE[RT_MAX_GROUPS];          /* cm^2, energy-weighted group cross-section (Sec. 2.2.4) */
    double Eavg[RT_MAX_GROUPS];          /* erg, mean photon energy of the group */
    double frac[RT_MAX_GROUPS];          /* share of each source's photons in the group (Eq. e:sgroup) */
    double c_red;                        /* cm/s, reduced speed of light (Sec. 2.2.3) */
    double cfl;                          /* Courant factor C in dt = C dx/(3 c_red); (0, 1] */
    int    ots;                          /* on-the-spot: alpha_A -> alpha_B, no recombination photons */
    int    isothermal;                   /* T held fixed (one chemistry sub-cycle per step) */
    int    nsub;                         /* 0: adaptive dtau = min(rest, |e/(H-Lambda)|);
                                            >0: dt split in nsub equal intervals */
    int    rates_const;                  /* 1: alpha_A, alpha_B, beta below, no cooling
                                            (requires isothermal); 0: temperature fits */
    double alphaA, alphaB, beta;         /* cm^3/s, used when rates_const */
    int    bc[6];                        /* faces -x,+x,-y,+y,-z,+z, rt_bc values */
    int    max_halvings;                 /* cap of the 10% rule (e.g. 30) */
    int    precision;                    /* rt_precision */
    int    tune;                         /* launch shape of the SPLIT form's transport, GLF or
                                            HLL (tile and grid; the results do not depend on
                                            it): 0 = default, 1 = time every shape at rt_create
                                            on a synthetic state in scratch and keep the
                                            fastest (cached per device, flux and box set for
                                            the process), 2 + k = shape k: k = 3 t + (b - 1)
                                            for tile t (32x8, 16x16, 64x4) at b = 1..3 resident
                                            blocks per SM (capped by what fits), k = 9 + 2 t +
                                            (j - 1) for tile t at j = 1, 2 blocks per tile
                                            column, k = 15 + 3 t + c for tile t at the most
                                            resident blocks with the plane units in z-chunks
                                            of 16, 32, 64 planes (c = 0, 1, 2), k = 24 + 2 t +
                                            s for tile t in lockstep rows by per-thread copies
                                            (s = 0) or TMA (s = 1), k = 30 + t for tile t with
                                            TMA, k = 33 + 2 t + s for tile t with two photon
                                            groups per block in column order (s = 0) or
                                            lockstep rows (s = 1) (GLF; TMA, lockstep rows and
                                            groups per block fall back to the default where
                                            they do not apply); k >= 39 is RT_ERR_ARG.  Ignored
                                            by the FP64 forms */
    int    flux;                         /* rt_flux; rt_adjoint and rt_transport_static need GLF */
    double inflow[6];                    /* photons/cm^2/s entering through each RT_BC_INFLOW face */
    int    cosmo;                        /* 1: supercomoving units (Sec. 3).  U holds the comoving
                                            N^ = a^3 N / nunit and F^ = a^3 F / (c_red nunit), T holds
                                            T~ = a^2 T, n0 and dx are comoving (their a = 1 values);
                                            each step runs the chemistry in physical units at its a
                                            and advances a over dt = a dt_com by the Friedmann
                                            equation.  Every box must have the same dx. */
    double H0, omega_m, omega_l;         /* cosmo: Hubble constant (1/s), matter and vacuum densities */
    double a0;                           /* cosmo: expansion factor at rt_create (> 0) */
    int    chem_tune;                    /* launch shape of the chemistry of the SPLIT and FP64
                                            forms (the results do not depend on it): 0 = default
                                            (the most resident blocks per SM, one work item per
                                            draw), 1 = time every shape at rt_create on scratch
                                            copies of the boxes' state and keep the fastest
                                            (cached per device, form and box set for the
                                            process; cosmo runs take the default), 2 + k = shape
                                            k = 3 (b - 1) + j: b = 1, 2 resident blocks per SM
                                            (capped by what fits), j = 0, 1, 2 for 1, 2, 4 work
                                            items (128 cells each) per draw from the counter;
                                            k >= 6 is RT_ERR_ARG.  Ignored by the strict form */
} rt_params;

typedef struct rt_box {
    int     nx, ny, nz;                  /* cells per axis, each >= 1 */
    double  dx;                          /* cm, cell size */
    double  nunit;                       /* photons/cm^3 per stored unit of N (> 0) */
    void   *U;                           /* device, G*ncell*4 float (SPLIT) or double, read/write */
    double *xHI;                         /* device, ncell, neutral fraction, read/write */
    double *T;                           /* device, ncell, K, read/write */
    const void *n0;                      /* device, ncell, cm^-3, float (SPLIT) or double, read only */
} rt_box;

typedef struct rt_stats {
    int64_t steps;                       /* steps run since rt_create */
    int64_t realizability_clamps;        /* post-transport cells with |F| > cN (1 + tol),
                                            tol 1e-12 (FP64) or 1e-5 (FP32), summed over steps;
                                            cells with N <= 1e-290 (FP64) / 1e-30 (FP32) stored
                                            units are not checked (|F|/N has no digits there) */
    int     error_bits;                  /* OR of device error bits seen (1 nonfinite, 2 realizability,
                                            4 sub-cycle cap) */
    int     nboxes;
    int64_t cells;                       /* cells over all boxes */
    double  last_diag[RT_NDIAG];         /* diagnostics of box 0 after the last step */
    double  kernel_ms[3];                /* with profiling on: summed CUDA-event time of the
                                            transport, chemistry (with the fused per-box
                                            diagnostics) and CRTA fine-level kernels */
    int64_t kernel_launches[3];          /* launches timed into kernel_ms */
    int     tile_x, tile_y;              /* transport tile (columns x rows per block) */
    int     transport_grid, chem_grid;   /* blocks of the persistent transport / chemistry grids */
    double  a;                           /* cosmo: current expansion factor (1 otherwise) */
    int     transport_zchunk;            /* z-chunk length of the transport's work order
                                            (0: whole tile columns) */
    int     transport_tma;               /* 1: the SPLIT form's GLF transport loads its planes
                                            by TMA (tensor maps of every box encoded);
                                            0: per-thread copies */
    int     transport_lockstep;          /* tile columns per row of the lockstep-rows work
                                            order (0: off) */
    int     chem_grab;                   /* chemistry work items a warp takes per draw */
    int     transport_gpb;               /* photon groups per block of the FP32 GLF transport */
} rt_stats;

typedef struct rt_handle rt_handle;

/* Create a solver over nboxes independent boxes that share p.  Validates
 * every argument, copies p and the box descriptors, allocates scratch on the
 * current device and orders all later work on `stream` (a cudaStream_t, NULL =
 * legacy default stream).  *h is set only on success. */
RT_API int rt_create(rt_handle **h, const rt_params *p, const rt_box *boxes, int nboxes, void *stream);

/* Point sources of box `box` (Sec. 2.2.4, source term S of Eq. e:therm1g):
 * nsrc host arrays, cell = linear cell index in [0, ncell), Q = photons/s of
 * the whole spectrum, split over groups by p->frac.  The per-cell source term
 * is S_i = (sum_k Q_k frac_i) / (dx^3 nunit), duplicates summed in list order.
 * Replaces the box's previous sources; nsrc = 0 removes them. */
RT_API int rt_set_sources(rt_handle *h, int box, int nsrc, const int64_t *cell, const double *Q);

/* CRTA fine level of `box` (Sec. 5, coarse radiative transport
 * approximation: radiation is transported on the coarse grid only, while
 * the thermochemistry also runs on refined cells, which see the coarse
 * radiation field injected unchanged).  After the coarse chemistry of every
 * later step, each of the nfine refined cells runs the same sub-cycled
 * chemistry over the box's dt, starting from the post-transport N, F of its
 * parent coarse cell and with the parent's source term per unit volume; its
 * radiation result is not kept.
 *   parent  device, nfine int64: linear index of the parent cell in the box
 *           (validated and copied by the library)
 *   n0      device, nfine densities (cm^-3), float (SPLIT) or double
 *   xHI, T  device, nfine doubles: the refined cells' state, updated in place
 * The caller owns n0, xHI and T, which must stay valid while registered.
 * nfine = 0 removes the box's fine level.  Synchronises the handle's stream.
 * rt_adjoint differentiates the coarse run only and leaves the fine level
 * untouched. */
RT_API int rt_set_fine(rt_handle *h, int box, int64_t nfine, const int64_t *parent, const void *n0,
                       double *xHI, double *T);

/* Advance all boxes by nsteps (>= 0) steps, in place.  hist: device pointer to
 * nsteps*nboxes*RT_NDIAG doubles ([step][box][diag]) or NULL.  Returns the
 * most severe device error of the call (RT_ERR_SUBCYCLE, RT_ERR_NONFINITE,
 * RT_ERR_REALIZABILITY) after completing all steps. */
RT_API int rt_step(rt_handle *h, int nsteps, double *hist);

/* Gradient of a loss of the ionised-fraction history (the paper has no
 * adjoint: this is the reverse mode of its step).
 * Runs the handle's step nsteps times from the device state (U0, xHI0, T0)
 * with the handle's current sources and density, X(t) = volume-weighted
 * ionised fraction mean(1 - xHI) after step t (the first diagnostic of
 * rt_step), then the hand-written reverse pass of every step with the
 * forward's branch decisions frozen (10% halvings, dtau sequence, flux
 * clamp), recomputing each segment of ckpt_every steps from a checkpoint.
 *   dL_dX   device, nsteps doubles: dL/dX(t), t = 1..nsteps
 *   dL_dQ   host, one double per source of the last rt_set_sources call, in
 *           its order: dL/dQ (per photons/s of the whole spectrum)
 *   dL_dn0  device, ncell doubles: dL/dn0 per cell (per cm^-3)
 * Needs one box, an FP64 form and periodic faces (RT_ERR_ARG otherwise).
 * Allocates its checkpoints and segment states for the call.  On return the
 * box holds the state after the nsteps forward steps.  RT_ERR_SUBCYCLE if a
 * cell-step of the recomputation needs more than 2048 accepted sub-cycles. */
RT_API int rt_adjoint(rt_handle *h, const void *U0, const double *xHI0, const double *T0,
                      int nsteps, int ckpt_every, const double *dL_dX, double *dL_dQ,
                      double *dL_dn0);

/* Copy host arrays into the device state of `box` (any argument may be NULL
 * to skip it; U in the precision's element type; n0 overwrites the caller's
 * density buffer).  Ordered on the handle's stream; returns after the copy. */
RT_API int rt_upload(rt_handle *h, int box, const void *U, const double *xHI, const double *T,
              const void *n0);

/* Copy the device state of `box` into host arrays (NULL skips an array). */
RT_API int rt_download(rt_handle *h, int box, void *U, double *xHI, double *T);

/* Profiling switch.  on != 0: later rt_step calls launch each kernel directly
 * (no graph replay) between CUDA events recorded on the library's stream and
 * add the elapsed times to rt_stats.kernel_ms; the counters restart at zero.
 * on == 0: back to graph replay. */
RT_API int rt_set_profiling(rt_handle *h, int on);

/* Counters and the last diagnostics; never launches work. */
RT_API int rt_query(rt_handle *h, rt_stats *st);

/* Message of the last failing call on h; when h is NULL, of the last failing
 * rt_create or rt_transport_static on the calling thread.  Never NULL. */
RT_API const char *rt_last_error(rt_handle *h);

/* Free the scratch and the handle (h may be NULL). */
RT_API void rt_destroy(rt_handle *h);

/* Host helper: dt of the radiative Courant condition (Sec. 2.2.3, 3-D
 * reading dt = cfl dx / (3 c_red)); returns a negative value on bad input. */
RT_API double rt_timestep(const rt_params *p, double dx);

/* Host helper: wave-speed table of the HLL flux (rt_params.flux = RT_FLUX_HLL).
 * lmax[i][j], (nf + 1) x (nm + 1) doubles, row-major: the largest eigenvalue
 * (units of c) of the Jacobian of the M1 flux (Levermore closure) along an
 * axis, at f = |F|/(cN) = 1 - (i/nf)^2 and mu = F_axis/|F| = -1 + 2j/nm; the
 * kernels use the 64 x 64 table, interpolated bilinearly in (sqrt(1 - f), mu),
 * and lambda_min(f, mu) = -lambda_max(f, -mu).  Returns RT_ERR_ARG on bad
 * sizes or a NULL pointer. */
RT_API int rt_hll_speeds(int nf, int nm, double *lmax);

/* Host helper: group averages of the hydrogen photo-ionisation cross-section
 * over a black-body photon spectrum of temperature T_bb (Eq. e:siggroup and
 * the sigma_E, <E> definitions of Sec. 2.2.4; Eq. e:sgroup for frac).
 * edges_eV: ngroups+1 increasing energies (eV, first >= 13.6).  Outputs
 * ngroups values each: sigN, sigE (cm^2), Eavg (erg), frac (sums to 1). */
RT_API int rt_group_table(int ngroups, const double *edges_eV, double T_bb,
                   double *sigN, double *sigE, double *Eavg, double *frac);

/* Bytes of the file-scope device array that rt_transport_static uses as its
 * only scratch (32 MiB).  Every GPU that loads this library holds it until
 * the process exits. */
#define RT_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* Transport without allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc while they run -- a
 * framework whose caching allocator owns all device memory, or a code that
 * must not grow its device footprint or let an allocation synchronise the
 * device in the middle of a run.  rt_create allocates scratch; this call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * It advances the radiation state box->U of one box, in place, by nsteps
 * homogeneous GLF transport steps -- the first stage of rt_step, without
 * sources, absorption or chemistry -- using p->ngroups, c_red, cfl, bc and
 * precision (SPLIT: float U; FP64 / FP64_STRICT: double U); the chemistry
 * fields of p and box->xHI, box->T, box->n0 are not used and may be NULL.
 * The post-transport state lives in a static device array of
 * RT_STATIC_SCRATCH_BYTES bytes, so the box must satisfy
 *     ngroups * nx * ny * nz * 4 * element size <= RT_STATIC_SCRATCH_BYTES - 768
 * (2,097,104 cells for one FP32 group); a larger box is rejected with
 * RT_ERR_TOO_LARGE before any work is queued.  Unlike rt_step, no flux-limit
 * check (|F| <= cN, the realizability count of rt_stats) is applied to the
 * result.
 *
 * Work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and the call returns after that stream has drained, so it may not be called
 * while the stream is being captured into a CUDA graph.  The first call made
 * while a given device is current looks up the array's device address on
 * that device (cudaGetSymbolAddress) and caches it.  Every call shares the one
 * array and it keeps the last call's contents (each call rewrites what it
 * reads before reading it), so calls that overlap on the GPU -- from several
 * threads or streams at once -- race and must be serialised by the caller.
 * Returns RT_OK, RT_ERR_ARG (bad argument), RT_ERR_TOO_LARGE or RT_ERR_CUDA,
 * with the message in rt_last_error(NULL).  After RT_ERR_CUDA the stream has
 * drained, but box->U holds an undefined number of the requested steps. */
RT_API int rt_transport_static(const rt_params *p, const rt_box *box, int nsteps, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_M1_H */
