/*
 * m1_oracle.c -- plain, single-threaded FP64 CPU oracle of one explicit M1
 * radiative-transfer step on a uniform Cartesian grid, as described in
 * Aubert, Deparis & Ocvirk, "EMMA: an AMR cosmological simulation code with
 * radiative transfer" (arXiv:1508.07888):
 *
 *   1. time step from the radiative Courant condition   (Sec. 2.2.3, Sec. 2.3)
 *   2. M1 closure, GLF intercell fluxes, unsplit update (Sec. 2.2.3, Eqs.
 *      e:pdert1i, e:pdert2i, e:uprt, e:glf), boundary ghosts (Sec. 4.2)
 *   3. per-cell sub-cycled thermochemistry: sources/absorption, ionisation,
 *      energy, with the 10% energy rule (Sec. 2.2.4, Eqs. e:therm1-e:therm4,
 *      e:therm1g, e:therm2g, e:g2, e:g3 and the semi-implicit update that
 *      follows them)
 *   4. per-step diagnostics (front = ionised fraction 0.5, Sec. 6.4)
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  The GPU library shares no
 * code, header or constant generator with it.
 *
 * Arithmetic: FP64, compiled with -ffp-contract=off (no fused multiply-add),
 * every sum in the fixed order written below (x, then y, then z; groups in
 * increasing order; cells in increasing linear index).
 *
 * State variables.  The paper evolves N (photons/cm^3) and F (photons/cm^2/s).
 * The oracle evolves the same quantities rescaled by constants:
 *     Nhat = N / nunit,     Fhat = F / (c nunit)
 * so that Fhat has the units of N and |Fhat| <= Nhat is the flux limit.  The
 * transport equations e:pdert1i/e:pdert2i then read
 *     dNhat/dt + c div Fhat = 0,   dFhat/dt + c div (D Nhat) = 0,
 * and the GLF flux e:glf divides through by c nunit (first component) and by
 * c^2 nunit (the three flux components).
 *
 * Readings of the paper where it is silent, garbled or at odds with itself
 * (each one is marked READING below):
 *   R1 closure: D = (1-chi)/2 I + (3chi-1)/2 n n (the printed coefficients are
 *      swapped: the printed form gives D = n n/3 in the diffusive limit);
 *      chi = (3+4f^2)/(5+2 sqrt(4-3f^2)) (Levermore 1984), f = |F|/(cN)
 *      clamped to 1; evaluated as (3chi-1)/2 = f^2 g with
 *      g = (6 + 3/(2+s))/(5+2s), s = sqrt(4-3f^2), so D is smooth at F = 0.
 *   R2 3-D Courant condition: dt = C dx / (3 c), C = cfl (0.9).
 *   R3 the chemistry denominators carry the missing dtau:
 *      1 + c sigma_N (1-x) n0 dtau.
 *   R4 dtau = min(remaining, |e/(H - Lambda)|); redo with dtau/2 while
 *      |e^{p+1} - e^p| > 0.1 e^p (cap: max_halvings, then an error flag);
 *      isothermal cells take dtau = dt; fixed-nsub mode splits dt into nsub
 *      equal intervals, each advanced with the same 10% rule.
 *   R5 the neutral fraction xHI = 1 - x is the stored variable; the x update
 *      of the paper is rewritten for xHI (same expression).
 *   R6 e = (3/2)(1+x) n0 kB T (pure hydrogen, gamma = 5/3).
 *   R7 the (reduced) speed of light c appears in transport and chemistry.
 *   R8 rates: the paper cites, but does not print, its rate compilations.
 *      The fits used are those of Hui & Gnedin (1997) for case-A/B
 *      recombination, collisional ionisation and recombination cooling;
 *      collisional-excitation cooling exp(-118348/T) form of Cen (1992);
 *      bremsstrahlung 1.42e-27 g_ff sqrt(T) with g_ff = 1.3; no Compton term.
 *      Pinned, independently of the fits: alpha_A/alpha_B against the
 *      textbook values at 5e3-2e4 K; the case A - B split of the rate and
 *      of the cooling against recombination to 1s (Milne relation with the
 *      exact 1s cross-section); case B against Kramers sums over n >= 2;
 *      beta against Lotz's cross-section and Voronov's fit; the thresholds
 *      of beta and of the excitation cooling; the ionisation energy of the
 *      collisional-ionisation cooling; the classical free-free emissivity.
 *   R9 photo-ionisation cross-section: the exact hydrogenic form
 *      sigma = A0 (E1/E)^4 exp(4 - 4 atan(eps)/eps)/(1 - exp(-2 pi/eps)),
 *      eps = sqrt(E/E1 - 1), A0 = 6.30e-18 cm^2, E1 = 13.6 eV.
 *   R10 group averages (Eq. e:siggroup and the sigma_E, <E> definitions) over
 *      a black-body photon spectrum; source photons split by the group
 *      fraction of that spectrum (Eq. e:sgroup).
 *   R11 HLL flux (the paper plans it, Sec. 2.2.3, without formulas): the
 *      Harten-Lax-van Leer flux with the extreme eigenvalues of the M1 flux
 *      Jacobian as wave speeds, tabulated in (f, mu) and interpolated
 *      bilinearly (see face_flux), and |F| <= cN enforced after each HLL
 *      transport step (see hll_limit).
 *   R12 inflow boundary (the clump test of Sec. 6.5 feeds a photon flux in
 *      through the x = 0 face): the ghost state is a beam, F = c N along the
 *      inward normal, whose photon number flux c N is the given one.
 *   R13 supercomoving units (Sec. 3) for the radiation path: see section 7.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXG 4

/* physical constants (cgs) */
#define ORC_KB      1.380649e-16      /* erg/K */
#define ORC_EV      1.602176634e-12   /* erg */
#define ORC_E_HI    (13.6 * ORC_EV)   /* the paper's E_13.6 */
#define ORC_T_HI    157807.0          /* K, HI ionisation temperature of the rate fits */
#define ORC_MAXCYC  1000000           /* sub-cycles per cell and step before giving up */

/* error bits (returned OR-ed) */
#define ORC_ERR_NONFINITE 1
#define ORC_ERR_SUBCYCLE  4

/* Thread count for the cell loops (OpenMP).  Every cell update reads only the
 * previous state and writes only its own cell, so the result is bit-identical
 * for any thread count; the diagnostics are summed serially. */
static int orc_threads = 1;
void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return orc_threads; }

typedef struct {
    int    G;                    /* number of photon groups */
    double sigN[ORC_MAXG];       /* cm^2   number-weighted group cross-section */
    double sigE[ORC_MAXG];       /* cm^2   energy-weighted group cross-section */
    double Eavg[ORC_MAXG];       /* erg    mean photon energy of the group */
    double frac[ORC_MAXG];       /* share of the source photons in the group */
    double c;                    /* cm/s   (reduced) speed of light */
    double cfl;                  /* Courant factor C */
    int    ots;                  /* on-the-spot approximation */
    int    isothermal;           /* temperature held fixed */
    int    nsub;                 /* 0: adaptive chemistry steps; >0 fixed intervals */
    int    rates_const;          /* 1: constant alpha_A, alpha_B, beta; no cooling */
    double alphaA, alphaB, beta; /* cm^3/s, used when rates_const */
    int    bc[6];                /* faces -x,+x,-y,+y,-z,+z: 0 periodic, 1 transmissive, 2 reflective */
    int    max_halvings;         /* cap of the 10% rule */
    int    flux;                 /* intercell flux: 0 GLF (Eq. e:glf), 1 HLL (R11) */
    const double *hll;           /* HLL: lambda_max at f_i = 1 - (i/hll_nf)^2, mu_j = -1 + 2j/hll_nm,
                                    [hll_nf + 1][hll_nm + 1], row-major */
    int    hll_nf, hll_nm;
    double inflow[6][ORC_MAXG];  /* bc 3 (inflow, R12): stored photon density N^ of the
                                    incoming beam per face and group */
} orc_params;

/* ------------------------------------------------------------------ */
/* 1. time step (Sec. 2.2.3 Courant condition, Sec. 2.3 dt_rad; R2)    */
/* ------------------------------------------------------------------ */
double orc_timestep(const orc_params *p, double dx)
{
    return p->cfl * dx / (3.0 * p->c);
}

double orc_courant_number(const orc_params *p, double dx)
{
    double dt = orc_timestep(p, dx);
    return p->c * dt / dx;
}

/* ------------------------------------------------------------------ */
/* 2. M1 closure (Sec. 2.2.3, P = D N; R1)                              */
/*    U = (Nhat, Fhat_x, Fhat_y, Fhat_z).  Output P6 = Nhat * D as      */
/*    (xx, xy, xz, yy, yz, zz); returns chi.                            */
/* ------------------------------------------------------------------ */
double orc_closure(const double *U, double *P6, double *a_out, double *g_out)
{
    double N = U[0];
    double a = 1.0 / 3.0, g = 0.75, chi = 1.0 / 3.0;
    if (N > 0.0) {
        double ux = U[1] / N, uy = U[2] / N, uz = U[3] / N;
        double f2 = ux * ux + uy * uy + uz * uz;
        if (f2 > 1.0) {             /* flux limit |F| <= cN (rounding guard) */
            double f = sqrt(f2);
            ux = ux / f; uy = uy / f; uz = uz / f;
            f2 = 1.0;
        }
        double s = sqrt(4.0 - 3.0 * f2);
        a = ((1.0 + s) - 2.0 * f2) / (5.0 + 2.0 * s);    /* (1 - chi)/2        */
        g = (6.0 + 3.0 / (2.0 + s)) / (5.0 + 2.0 * s);   /* (3chi - 1)/(2 f^2) */
        chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * s);
        P6[0] = N * (a + g * (ux * ux));
        P6[1] = N * (g * (ux * uy));
        P6[2] = N * (g * (ux * uz));
        P6[3] = N * (a + g * (uy * uy));
        P6[4] = N * (g * (uy * uz));
        P6[5] = N * (a + g * (uz * uz));
    } else {
        for (int k = 0; k < 6; k++) P6[k] = 0.0;
    }
    if (a_out) *a_out = a;
    if (g_out) *g_out = g;
    return chi;
}

static const int P6IDX[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

/* physical flux of U along axis d, in the rescaled variables:
 * Ftilde_d = (Fhat_d, (Nhat D)_{d x}, (Nhat D)_{d y}, (Nhat D)_{d z})  (Sec. 2.2.3) */
static void phys_flux(int d, const double *U, double *Gd)
{
    double P6[6];
    orc_closure(U, P6, NULL, NULL);
    Gd[0] = U[1 + d];
    Gd[1] = P6[P6IDX[d][0]];
    Gd[2] = P6[P6IDX[d][1]];
    Gd[3] = P6[P6IDX[d][2]];
}

/* GLF intercell flux between left state L and right state R along d
 * (Eq. e:glf, divided by c nunit resp. c^2 nunit). */
void orc_glf_flux(int d, const double *L, const double *R, double *Phi)
{
    double GL[4], GR[4];
    phys_flux(d, L, GL);
    phys_flux(d, R, GR);
    for (int m = 0; m < 4; m++)
        Phi[m] = 0.5 * ((GL[m] + GR[m]) - (R[m] - L[m]));
}

/* ---- HLL intercell flux (R11) ----
 * The paper names the HLL flux as the less diffusive alternative it plans
 * after GLF.  Reading: the Harten-Lax-van Leer flux
 *   Phi = (l+ G_L - l- G_R + l+ l- (U_R - U_L)) / (l+ - l-),
 *   l+ = max(0, lmax_L, lmax_R),  l- = min(0, lmin_L, lmin_R),
 * with the extreme eigenvalues of the Jacobian of the physical flux along the
 * face normal (units of c).  They depend on f = |F|/(cN) and mu = F_d/|F|
 * only; lmax(f, mu) is the bilinear interpolant, in z = sqrt(1 - f) and mu,
 * of its values at the nodes of a table (computed outside this file from
 * the Jacobian below; the eigenvalues split like sqrt(1 - f) from their
 * common value mu at f = 1, so they are smooth in z), and
 * lmin(f, mu) = -lmax(f, -mu) by reflection.  A state with N <= 0 or F = 0
 * takes f = 0 (isotropic speeds).  GLF is the special case l+ = -l- = 1. */
static double hll_lmax(const orc_params *p, double f, double mu)
{
    int nf = p->hll_nf, nm = p->hll_nm;
    double x = sqrt(1.0 - f) * nf, y = (mu + 1.0) * 0.5 * nm;
    int i = (int)x, j = (int)y;
    if (i > nf - 1) i = nf - 1;
    if (i < 0) i = 0;
    if (j > nm - 1) j = nm - 1;
    if (j < 0) j = 0;
    double tx = x - i, ty = y - j;
    const double *T = p->hll;
    double v00 = T[i * (nm + 1) + j], v01 = T[i * (nm + 1) + j + 1];
    double v10 = T[(i + 1) * (nm + 1) + j], v11 = T[(i + 1) * (nm + 1) + j + 1];
    return (v00 * (1.0 - tx) + v10 * tx) * (1.0 - ty) + (v01 * (1.0 - tx) + v11 * tx) * ty;
}

/* wave-speed bounds of state U along axis d */
static void hll_speeds(const orc_params *p, int d, const double *U, double *lmin, double *lmax)
{
    double f = 0.0, mu = 0.0;
    double N = U[0];
    if (N > 0.0) {
        double F = sqrt(U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
        if (F > 0.0) {
            f = F / N;
            if (f > 1.0) f = 1.0;
            mu = U[1 + d] / F;
        }
    }
    *lmax = hll_lmax(p, f, mu);
    *lmin = -hll_lmax(p, f, -mu);
}

/* intercell flux at a face along d from the states and physical fluxes of
 * its left and right cells (GLF or HLL) */
static void face_flux(const orc_params *p, int d, const double *UL, const double *GL,
                      const double *UR, const double *GR, double *Phi)
{
    if (p->flux == 0) {
        for (int m = 0; m < 4; m++) Phi[m] = 0.5 * ((GL[m] + GR[m]) - (UR[m] - UL[m]));
        return;
    }
    double a0, a1, b0, b1;
    hll_speeds(p, d, UL, &a0, &a1);
    hll_speeds(p, d, UR, &b0, &b1);
    double lp = a1 > b1 ? a1 : b1, lm = a0 < b0 ? a0 : b0;
    if (lp < 0.0) lp = 0.0;
    if (lm > 0.0) lm = 0.0;
    if (!(lp - lm > 0.0)) {
        /* no wave crosses the face (two beams along it, f = 1, mu = 0 on
           both sides): their fluxes along d vanish; take the mean */
        for (int m = 0; m < 4; m++) Phi[m] = 0.5 * (GL[m] + GR[m]);
        return;
    }
    for (int m = 0; m < 4; m++)
        Phi[m] = (lp * GL[m] - lm * GR[m] + lp * lm * (UR[m] - UL[m])) / (lp - lm);
}

/* After an HLL transport step the flux is limited to |F| <= cN, F scaled
 * down where it exceeds it (R11).  With the speeds lambda = mu of f = 1 the
 * HLL update amplifies the excess |F| - cN that rounding leaves in beam
 * cells (e' = (1 + lam) e - lam e_left along the beam), so without the
 * limiter beams blow up; GLF's unit speeds damp the same mode. */
static void hll_limit(double *U)
{
    double F = sqrt(U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
    if (F > U[0]) {
        double r = U[0] > 0.0 ? U[0] / F : 0.0;
        U[1] *= r;
        U[2] *= r;
        U[3] *= r;
    }
}

void orc_hll_speeds(const orc_params *p, int d, const double *U, double *lmin, double *lmax)
{
    hll_speeds(p, d, U, lmin, lmax);
}

static void phys_flux(int d, const double *U, double *Gd);

/* the face flux of p->flux between states L and R along d */
void orc_face_flux(const orc_params *p, int d, const double *L, const double *R, double *Phi)
{
    double GL[4], GR[4];
    phys_flux(d, L, GL);
    phys_flux(d, R, GR);
    face_flux(p, d, L, GL, R, GR, Phi);
}

/* Jacobian of the x flux at N = 1, F = f (mu, sqrt(1 - mu^2), 0), on the
 * closure's smooth branch (f <= 1; also at f = 1), for the HLL speed table */
void orc_flux_jacobian_fmu(double f, double mu, double J[4][4]);

/* neighbour state of cell (x,y,z) of group g along axis d, side = -1 or +1,
 * with the global boundary conditions of Sec. 4.2: periodic by default;
 * transmissive copies the cell itself; reflective copies it and inverts the
 * normal flux; inflow (R12) is a beam of the face's given density moving
 * into the box along the normal (F = c N). */
static void neighbour(const orc_params *p, const double *Ug, int nx, int ny, int nz,
                      int x, int y, int z, int d, int side, int g, double *out)
{
    int c[3] = {x, y, z};
    int n[3] = {nx, ny, nz};
    c[d] += side;
    if (c[d] >= 0 && c[d] < n[d]) {
        const double *s = Ug + 4 * (((size_t)c[2] * ny + c[1]) * nx + c[0]);
        memcpy(out, s, 4 * sizeof(double));
        return;
    }
    int face = 2 * d + (side > 0 ? 1 : 0);
    int bc = p->bc[face];
    if (bc == 0) {
        c[d] = (c[d] + n[d]) % n[d];
        const double *s = Ug + 4 * (((size_t)c[2] * ny + c[1]) * nx + c[0]);
        memcpy(out, s, 4 * sizeof(double));
        return;
    }
    if (bc == 3) {
        double N = p->inflow[face][g];
        out[0] = N;
        out[1] = out[2] = out[3] = 0.0;
        out[1 + d] = side < 0 ? N : -N;
        return;
    }
    const double *s = Ug + 4 * (((size_t)z * ny + y) * nx + x);
    memcpy(out, s, 4 * sizeof(double));
    if (bc == 2) out[1 + d] = -out[1 + d];
}

/* physical flux along d from a state and its closure P6 */
static void flux_from(int d, const double *U, const double *P6, double *Gd)
{
    Gd[0] = U[1 + d];
    Gd[1] = P6[P6IDX[d][0]];
    Gd[2] = P6[P6IDX[d][1]];
    Gd[3] = P6[P6IDX[d][2]];
}

/* One homogeneous transport step of every group (Eq. e:uprt, unsplit over
 * x, y, z).  U and Uout: [G][nz][ny][nx][4]; Jacobi style (Uout != U).
 * The closure of every cell is evaluated once (P array); a ghost state's
 * closure is evaluated where the ghost is built.  Each face flux is the same
 * function of (left, right) from either side, so both cells of a face see
 * the same value. */
void orc_transport(const orc_params *p, int nx, int ny, int nz, double lam,
                   const double *U, double *Uout)
{
    size_t ncell = (size_t)nx * ny * nz;
    double *P = (double *)malloc(sizeof(double) * 6 * ncell);
    for (int g = 0; g < p->G; g++) {
        const double *Ug = U + 4 * ncell * g;
        double *Og = Uout + 4 * ncell * g;
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (size_t id = 0; id < ncell; id++) orc_closure(Ug + 4 * id, P + 6 * id, NULL, NULL);
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    size_t id = ((size_t)z * ny + y) * nx + x;
                    const double *Uc = Ug + 4 * id;
                    const double *Pc = P + 6 * id;
                    int cc[3] = {x, y, z}, nn[3] = {nx, ny, nz};
                    size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
                    double diff[3][4];
                    for (int d = 0; d < 3; d++) {
                        double Gs[2][4], Gc[4], Us[2][4], Pg[6];
                        flux_from(d, Uc, Pc, Gc);
                        for (int side = 0; side < 2; side++) {
                            int sgn = side ? +1 : -1;
                            int c2 = cc[d] + sgn;
                            if (c2 >= 0 && c2 < nn[d]) {
                                size_t nid = side ? id + stride[d] : id - stride[d];
                                memcpy(Us[side], Ug + 4 * nid, 4 * sizeof(double));
                                flux_from(d, Us[side], P + 6 * nid, Gs[side]);
                            } else if (p->bc[2 * d + side] == 0) {
                                size_t nid = side ? id - stride[d] * (nn[d] - 1)
                                                  : id + stride[d] * (nn[d] - 1);
                                memcpy(Us[side], Ug + 4 * nid, 4 * sizeof(double));
                                flux_from(d, Us[side], P + 6 * nid, Gs[side]);
                            } else {
                                neighbour(p, Ug, nx, ny, nz, x, y, z, d, sgn, g, Us[side]);
                                orc_closure(Us[side], Pg, NULL, NULL);
                                flux_from(d, Us[side], Pg, Gs[side]);
                            }
                        }
                        /* faces i-1/2 (left neighbour, cell) and i+1/2 (cell, right) */
                        double Fm[4], Fp[4];
                        face_flux(p, d, Us[0], Gs[0], Uc, Gc, Fm);
                        face_flux(p, d, Uc, Gc, Us[1], Gs[1], Fp);
                        for (int m = 0; m < 4; m++) diff[d][m] = Fp[m] - Fm[m];
                    }
                    for (int m = 0; m < 4; m++)
                        Og[4 * id + m] = Uc[m] - lam * ((diff[0][m] + diff[1][m]) + diff[2][m]);
                    if (p->flux == 1) hll_limit(Og + 4 * id);
                }
    }
    free(P);
}

/* Transport of single cells (the same per-cell expression as
 * orc_transport, with every closure evaluated from its state): post-transport
 * state of cells cell[0..ncells) of group g, written to out[ncells][4].
 * Used to check a large grid one sampled cell at a time. */
void orc_transport_cells(const orc_params *p, int nx, int ny, int nz, double lam, const double *U,
                         int g, int ncells, const int64_t *cell, double *out)
{
    size_t ncell = (size_t)nx * ny * nz;
    const double *Ug = U + 4 * ncell * g;
    for (int k = 0; k < ncells; k++) {
        int64_t id = cell[k];
        int x = (int)(id % nx), y = (int)((id / nx) % ny), z = (int)(id / ((int64_t)nx * ny));
        const double *Uc = Ug + 4 * id;
        double Pc[6], diff[3][4];
        orc_closure(Uc, Pc, NULL, NULL);
        for (int d = 0; d < 3; d++) {
            double Gc[4], Us[2][4], Ps[6], Gs[2][4];
            flux_from(d, Uc, Pc, Gc);
            for (int side = 0; side < 2; side++) {
                neighbour(p, Ug, nx, ny, nz, x, y, z, d, side ? +1 : -1, g, Us[side]);
                orc_closure(Us[side], Ps, NULL, NULL);
                flux_from(d, Us[side], Ps, Gs[side]);
            }
            double Fm[4], Fp[4];
            face_flux(p, d, Us[0], Gs[0], Uc, Gc, Fm);
            face_flux(p, d, Uc, Gc, Us[1], Gs[1], Fp);
            for (int m = 0; m < 4; m++) diff[d][m] = Fp[m] - Fm[m];
        }
        for (int m = 0; m < 4; m++)
            out[4 * k + m] = Uc[m] - lam * ((diff[0][m] + diff[1][m]) + diff[2][m]);
        if (p->flux == 1) hll_limit(out + 4 * k);
    }
}

/* ------------------------------------------------------------------ */
/* 3a. atomic rates (R8); T in K, results in cgs                        */
/* ------------------------------------------------------------------ */
double orc_alphaA(double T)
{
    double l = 2.0 * ORC_T_HI / T;
    return 1.269e-13 * pow(l, 1.503) / pow(1.0 + pow(l / 0.522, 0.470), 1.923);
}

double orc_alphaB(double T)
{
    double l = 2.0 * ORC_T_HI / T;
    return 2.753e-14 * pow(l, 1.500) / pow(1.0 + pow(l / 2.740, 0.407), 2.242);
}

double orc_beta(double T)   /* collisional ionisation, cm^3/s */
{
    double l = 2.0 * ORC_T_HI / T;
    return 21.11 * pow(T, -1.5) * exp(-0.5 * l) * pow(l, -1.089)
           / pow(1.0 + pow(l / 0.354, 0.874), 1.101);
}

double orc_cool_recA(double T)   /* erg cm^3/s, multiplies n_e n_HII */
{
    double l = 2.0 * ORC_T_HI / T;
    return 1.778e-29 * T * pow(l, 1.965) / pow(1.0 + pow(l / 0.541, 0.502), 2.697);
}

double orc_cool_recB(double T)
{
    double l = 2.0 * ORC_T_HI / T;
    return 3.435e-30 * T * pow(l, 1.970) / pow(1.0 + pow(l / 2.250, 0.376), 3.720);
}

double orc_cool_colion(double T)   /* multiplies n_e n_HI */
{
    return ORC_KB * ORC_T_HI * orc_beta(T);
}

double orc_cool_colexc(double T)   /* multiplies n_e n_HI */
{
    return 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1.0e5));
}

double orc_cool_brems(double T)    /* multiplies n_e n_HII */
{
    return 1.42e-27 * 1.3 * sqrt(T);
}

/* cooling rate Lambda(n0, x, T) of Eq. e:therm4, erg/cm^3/s */
double orc_cooling(const orc_params *p, double n0, double xHI, double T)
{
    if (p->rates_const) return 0.0;
    double x = 1.0 - xHI;
    double ne = x * n0, nHII = x * n0, nHI = xHI * n0;
    double crec = p->ots ? orc_cool_recB(T) : orc_cool_recA(T);
    return ne * nHII * (crec + orc_cool_brems(T))
         + ne * nHI * (orc_cool_colion(T) + orc_cool_colexc(T));
}

/* internal energy density e = (3/2)(1 + x) n0 kB T (R6) */
static double eint(double xHI, double n0, double T)
{
    return 1.5 * (1.0 + (1.0 - xHI)) * n0 * ORC_KB * T;
}

/* ------------------------------------------------------------------ */
/* 3b. per-cell thermochemistry over one transport step (Sec. 2.2.4)    */
/* ------------------------------------------------------------------ */
typedef struct {
    int G;
    double N[ORC_MAXG], F[ORC_MAXG][3];
    double xHI, T;
} cellstate;

/* one trial update of length dtau from state s into o, in the paper's order
 * N -> F -> x -> e; returns e^p and e^{p+1} through ep/e1 */
static void chem_trial(const orc_params *p, double nunit, double n0, const double *S,
                       double alpha, double alphaA, double alphaB, double beta,
                       const cellstate *s, double dtau, cellstate *o,
                       double *ep, double *e1)
{
    int G = p->G;
    double c = p->c;
    double x = 1.0 - s->xHI;
    o->G = G;
    /* Eqs. e:therm1g / e:therm2g, implicit absorption (R3) */
    for (int i = 0; i < G; i++) {
        double den = 1.0 + c * p->sigN[i] * s->xHI * n0 * dtau;
        double src = S[i];
        if (i == 0 && !p->ots)   /* recombination photons feed group 1 only */
            src = src + (alphaA - alphaB) * x * x * n0 * n0 / nunit;
        o->N[i] = (s->N[i] + src * dtau) / den;
        for (int k = 0; k < 3; k++) o->F[i][k] = s->F[i][k] / den;
    }
    /* ionisation, Eq. e:therm3 with Eq. e:g2, written for xHI (R5) */
    double gam = 0.0;
    for (int i = 0; i < G; i++) gam += c * p->sigN[i] * (nunit * o->N[i]);
    o->xHI = (s->xHI + alpha * x * x * n0 * dtau) / (1.0 + dtau * (beta * x * n0 + gam));
    /* energy, Eq. e:therm4 with Eq. e:g3 */
    double e0 = eint(s->xHI, n0, s->T);
    *ep = e0;
    if (p->isothermal) {
        o->T = s->T;
        *e1 = e0;
        return;
    }
    double heat = 0.0;
    for (int i = 0; i < G; i++) {
        double SigE = p->sigE[i] * p->Eavg[i] - p->sigN[i] * ORC_E_HI;
        heat += c * o->xHI * n0 * (nunit * o->N[i]) * SigE;
    }
    double lam = orc_cooling(p, n0, o->xHI, s->T);   /* Lambda(n0, x^{p+1}, T^p) */
    double e = e0 + dtau * heat - dtau * lam;
    *e1 = e;
    o->T = e / (1.5 * (1.0 + (1.0 - o->xHI)) * n0 * ORC_KB);
}

/* accepted trials of one cell's step, recorded for the adjoint */
typedef struct {
    int n, cap;
    cellstate *s;     /* state before each accepted trial */
    double *dtau;     /* its length */
} chem_trace;

static void trace_push(chem_trace *tr, const cellstate *s, double dtau)
{
    if (!tr) return;
    if (tr->n == tr->cap) {
        tr->cap = tr->cap ? 2 * tr->cap : 16;
        tr->s = (cellstate *)realloc(tr->s, sizeof(cellstate) * tr->cap);
        tr->dtau = (double *)realloc(tr->dtau, sizeof(double) * tr->cap);
    }
    tr->s[tr->n] = *s;
    tr->dtau[tr->n] = dtau;
    tr->n++;
}

/* advance one cell over a span of time with sub-cycles (R4) */
static int chem_span_tr(const orc_params *p, double nunit, double n0, const double *S,
                        cellstate *s, double span, int use_estimate, int *ncyc, chem_trace *tr);

static int chem_span(const orc_params *p, double nunit, double n0, const double *S,
                     cellstate *s, double span, int use_estimate, int *ncyc)
{
    return chem_span_tr(p, nunit, n0, S, s, span, use_estimate, ncyc, NULL);
}

static int chem_span_tr(const orc_params *p, double nunit, double n0, const double *S,
                        cellstate *s, double span, int use_estimate, int *ncyc, chem_trace *tr)
{
    int err = 0;
    double tau = 0.0;
    for (;;) {
        double rem = span - tau;
        double T = s->T;
        double aA, aB, beta;
        if (p->rates_const) { aA = p->alphaA; aB = p->alphaB; beta = p->beta; }
        else { aA = orc_alphaA(T); aB = orc_alphaB(T); beta = orc_beta(T); }
        double alpha = p->ots ? aB : aA;

        double dtau = rem;
        int last = 1;
        if (!p->isothermal && use_estimate) {
            /* dtau from the p state: e^p / (H^p - Lambda^p) */
            double heat = 0.0;
            for (int i = 0; i < p->G; i++) {
                double SigE = p->sigE[i] * p->Eavg[i] - p->sigN[i] * ORC_E_HI;
                heat += p->c * s->xHI * n0 * (nunit * s->N[i]) * SigE;
            }
            double rate = heat - orc_cooling(p, n0, s->xHI, T);
            double e = eint(s->xHI, n0, T);
            if (rate != 0.0) {
                double est = fabs(e / rate);
                if (est < rem) { dtau = est; last = 0; }
            }
        }
        cellstate o;
        double ep, e1;
        for (int h = 0;; h++) {
            chem_trial(p, nunit, n0, S, alpha, aA, aB, beta, s, dtau, &o, &ep, &e1);
            if (p->isothermal) break;
            if (fabs(e1 - ep) <= 0.1 * ep) break;    /* 10% rule */
            if (h >= p->max_halvings) { err |= ORC_ERR_SUBCYCLE; break; }
            dtau = 0.5 * dtau;
            last = 0;
        }
        trace_push(tr, s, dtau);
        *s = o;
        (*ncyc)++;
        if (last) break;
        tau = tau + dtau;
        if (*ncyc >= ORC_MAXCYC) { err |= ORC_ERR_SUBCYCLE; break; }
    }
    return err;
}

/* Thermochemistry of one cell over dt.  U: G x 4 rescaled radiation state
 * (in/out), S: G source terms in nunit per second. */
int orc_chem_cell(const orc_params *p, double dt, double nunit, double n0,
                  const double *S, double *U, double *xHI, double *T, int *ncyc_out)
{
    cellstate s;
    s.G = p->G;
    for (int i = 0; i < p->G; i++) {
        s.N[i] = U[4 * i];
        for (int k = 0; k < 3; k++) s.F[i][k] = U[4 * i + 1 + k];
    }
    s.xHI = *xHI;
    s.T = *T;
    int ncyc = 0, err = 0;
    if (p->nsub > 0) {
        double h = dt / p->nsub;
        for (int k = 0; k < p->nsub; k++) err |= chem_span(p, nunit, n0, S, &s, h, 0, &ncyc);
    } else {
        err |= chem_span(p, nunit, n0, S, &s, dt, 1, &ncyc);
    }
    for (int i = 0; i < p->G; i++) {
        U[4 * i] = s.N[i];
        for (int k = 0; k < 3; k++) U[4 * i + 1 + k] = s.F[i][k];
    }
    *xHI = s.xHI;
    *T = s.T;
    if (!isfinite(s.xHI) || !isfinite(s.T)) err |= ORC_ERR_NONFINITE;
    if (ncyc_out) *ncyc_out = ncyc;
    return err;
}

/* dense source field S[g][cell] in nunit per second from a point-source list:
 * S_i = (sum_k Q_k frac_i) / (dx^3 nunit), duplicates summed in list order. */
void orc_source_field(const orc_params *p, int64_t ncell, int nsrc, const int64_t *cell,
                      const double *Q, double dx, double nunit, double *S)
{
    memset(S, 0, sizeof(double) * (size_t)p->G * ncell);
    for (int k = 0; k < nsrc; k++)
        for (int i = 0; i < p->G; i++)
            S[(size_t)i * ncell + cell[k]] += Q[k] * p->frac[i];
    double vol = dx * dx * dx;
    for (int i = 0; i < p->G; i++)
        for (int64_t c = 0; c < ncell; c++)
            S[(size_t)i * ncell + c] = S[(size_t)i * ncell + c] / (vol * nunit);
}

/* One full step (transport, then chemistry) of the sampled cells only,
 * from the full state U/xHI/T: Uout[ncells][G][4], xout, Tout[ncells].
 * S: dense source field [G][ncell] or NULL.  Returns the error bits. */
int orc_step_cells(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
                   const double *U, const double *xHI, const double *T, const double *n0,
                   const double *S, int ncells, const int64_t *cell,
                   double *Uout, double *xout, double *Tout)
{
    size_t ncell = (size_t)nx * ny * nz;
    int G = p->G;
    double dt = orc_timestep(p, dx);
    double lam = p->c * dt / dx;
    double *tmp = (double *)malloc(sizeof(double) * 4 * (size_t)ncells);
    if (!tmp) return -1;
    for (int i = 0; i < G; i++) {
        orc_transport_cells(p, nx, ny, nz, lam, U, i, ncells, cell, tmp);
        for (int k = 0; k < ncells; k++)
            for (int m = 0; m < 4; m++) Uout[((size_t)k * G + i) * 4 + m] = tmp[4 * k + m];
    }
    free(tmp);
    int err = 0;
    for (int k = 0; k < ncells; k++) {
        double Sc[ORC_MAXG];
        for (int i = 0; i < G; i++) Sc[i] = S ? S[ncell * i + cell[k]] : 0.0;
        xout[k] = xHI[cell[k]];
        Tout[k] = T[cell[k]];
        err |= orc_chem_cell(p, dt, nunit, n0[cell[k]], Sc, Uout + (size_t)k * G * 4, &xout[k],
                             &Tout[k], NULL);
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* 4. full steps: transport, then chemistry, then diagnostics           */
/*    hist[step][5] = {ionised fraction (volume weighted), photon total,*/
/*    max |F|/(cN), count(xHI < 0.5), mean sub-cycles per cell}        */
/* ------------------------------------------------------------------ */
/* nsteps steps with an optional CRTA fine level (Sec. 5, second
 * approximation: transport only on the coarse grid, thermochemistry also on
 * refined cells, which see the coarse radiation field injected unchanged).
 * Reading: each of the nfine refined cells runs the same sub-cycled
 * chemistry as a coarse cell over the coarse dt, starting from the
 * post-transport N, F of its parent coarse cell parent[f] and with the
 * parent's source term per unit volume; the refined cell's own radiation
 * result is not kept, since radiation lives on the coarse grid only. */
int orc_run_crta(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
                 double *U, double *xHI, double *T, const double *n0, const double *S,
                 int nsteps, double *hist, int64_t *nclamp_out, int64_t nfine,
                 const int64_t *parent, const double *n0f, double *xHIf, double *Tf);

int orc_run(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
            double *U, double *xHI, double *T, const double *n0, const double *S,
            int nsteps, double *hist, int64_t *nclamp_out)
{
    return orc_run_crta(p, nx, ny, nz, dx, nunit, U, xHI, T, n0, S, nsteps, hist, nclamp_out,
                        0, NULL, NULL, NULL, NULL);
}

int orc_run_crta(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
                 double *U, double *xHI, double *T, const double *n0, const double *S,
                 int nsteps, double *hist, int64_t *nclamp_out, int64_t nfine,
                 const int64_t *parent, const double *n0f, double *xHIf, double *Tf)
{
    size_t ncell = (size_t)nx * ny * nz;
    int G = p->G;
    double *Us = (double *)malloc(sizeof(double) * 4 * ncell * G);
    if (!Us) return -1;
    double dt = orc_timestep(p, dx);
    double lam = p->c * dt / dx;
    int err = 0;
    int64_t nclamp = 0;
    for (int step = 0; step < nsteps; step++) {
        orc_transport(p, nx, ny, nz, lam, U, Us);
        /* realizability after transport: |F| <= cN (1 + 1e-12); a count, so
         * the order in which threads add it up does not matter */
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(+:nclamp)
        for (size_t k = 0; k < ncell * G; k++) {
            double N = Us[4 * k];
            if (N > 0.0) {
                double ux = Us[4 * k + 1] / N, uy = Us[4 * k + 2] / N, uz = Us[4 * k + 3] / N;
                if (ux * ux + uy * uy + uz * uz > (1.0 + 1e-12) * (1.0 + 1e-12)) nclamp++;
            }
        }
        double cyc_sum = 0.0;
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 256) reduction(|:err) reduction(+:cyc_sum)
        for (size_t id = 0; id < ncell; id++) {
            double Uc[4 * ORC_MAXG], Sc[ORC_MAXG];
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) Uc[4 * i + m] = Us[4 * (ncell * i + id) + m];
                Sc[i] = S ? S[ncell * i + id] : 0.0;
            }
            int ncyc = 0;
            err |= orc_chem_cell(p, dt, nunit, n0[id], Sc, Uc, &xHI[id], &T[id], &ncyc);
            for (int i = 0; i < G; i++)
                for (int m = 0; m < 4; m++) U[4 * (ncell * i + id) + m] = Uc[4 * i + m];
            cyc_sum += ncyc;
        }
        /* refined cells: the parent's post-transport radiation and source */
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 256) reduction(|:err)
        for (int64_t f = 0; f < nfine; f++) {
            size_t id = (size_t)parent[f];
            double Uc[4 * ORC_MAXG], Sc[ORC_MAXG];
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) Uc[4 * i + m] = Us[4 * (ncell * i + id) + m];
                Sc[i] = S ? S[ncell * i + id] : 0.0;
            }
            int ncyc = 0;
            err |= orc_chem_cell(p, dt, nunit, n0f[f], Sc, Uc, &xHIf[f], &Tf[f], &ncyc);
        }
        if (hist) {
            /* the two sums in index order; the count and the maximum are exact
             * in any order, so threads share them */
            double X = 0.0, ph = 0.0, fmax = 0.0;
            int64_t nion = 0;
            for (size_t id = 0; id < ncell; id++) X += 1.0 - xHI[id];
            for (size_t k = 0; k < ncell * G; k++) ph += U[4 * k];
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(+:nion)
            for (size_t id = 0; id < ncell; id++)
                if (xHI[id] < 0.5) nion++;
#pragma omp parallel for num_threads(orc_threads) schedule(static) reduction(max:fmax)
            for (size_t k = 0; k < ncell * G; k++) {
                double N = U[4 * k];
                if (N > 0.0) {
                    double ux = U[4 * k + 1] / N, uy = U[4 * k + 2] / N, uz = U[4 * k + 3] / N;
                    double f = sqrt(ux * ux + uy * uy + uz * uz);
                    if (f > fmax) fmax = f;
                }
            }
            double *h = hist + 5 * (size_t)step;
            h[0] = X / (double)ncell;
            h[1] = ph * nunit * (dx * dx * dx);
            h[2] = fmax;
            h[3] = (double)nion;
            h[4] = cyc_sum / (double)ncell;
        }
    }
    free(Us);
    if (nclamp_out) *nclamp_out = nclamp;
    return err;
}

/* ------------------------------------------------------------------ */
/* 5. group averages over a black-body source spectrum (R9, R10)        */
/* ------------------------------------------------------------------ */
double orc_sigma_HI(double E_eV)
{
    const double E1 = 13.6, A0 = 6.30e-18;
    if (E_eV < E1) return 0.0;
    double r = E_eV / E1;
    double eps = sqrt(r - 1.0);
    if (eps < 1e-6) return A0;                 /* threshold limit */
    double r4 = r * r * r * r;
    return A0 / r4 * exp(4.0 - 4.0 * atan(eps) / eps) / (1.0 - exp(-2.0 * M_PI / eps));
}

/* Photon-number spectrum n(E) dE ~ E^2/(exp(E/kT) - 1) dE.  For each group
 * [edges[i], edges[i+1]] (eV):
 *   sigN = int sigma n dE / int n dE             (Eq. e:siggroup)
 *   Eavg = int E n dE / int n dE                 (mean photon energy)
 *   sigE = int sigma E n dE / (int n dE * Eavg)  (energy-weighted sigma)
 *   frac = int n dE / sum over groups            (Eq. e:sgroup)
 * Composite Simpson rule in u = ln E with 2*20000 intervals per group.
 * weight(E) lets the tests replace sigma by 1 to check the integrator. */
void orc_group_table_w(int G, const double *edges, double Tbb, int use_sigma,
                       double *sigN, double *sigE, double *Eavg, double *frac)
{
    const int M = 40000;
    double kT = ORC_KB * Tbb / ORC_EV;
    double tot = 0.0;
    double I0v[ORC_MAXG];
    for (int i = 0; i < G; i++) {
        double u0 = log(edges[i]), u1 = log(edges[i + 1]);
        double h = (u1 - u0) / M;
        double I0 = 0.0, I1 = 0.0, I2 = 0.0, I3 = 0.0;
        for (int k = 0; k <= M; k++) {
            double w = (k == 0 || k == M) ? 1.0 : ((k % 2) ? 4.0 : 2.0);
            double E = exp(u0 + h * k);
            double nE = E * E * E / expm1(E / kT);    /* n(E) dE/du, dE = E du */
            double sg = use_sigma ? orc_sigma_HI(E) : 1.0;
            I0 += w * nE;
            I1 += w * sg * nE;
            I2 += w * E * nE;
            I3 += w * sg * E * nE;
        }
        I0 *= h / 3.0; I1 *= h / 3.0; I2 *= h / 3.0; I3 *= h / 3.0;
        sigN[i] = I1 / I0;
        Eavg[i] = (I2 / I0) * ORC_EV;
        sigE[i] = I3 / I2;
        I0v[i] = I0;
        tot += I0;
    }
    for (int i = 0; i < G; i++) frac[i] = I0v[i] / tot;
}

void orc_group_table(int G, const double *edges, double Tbb,
                     double *sigN, double *sigE, double *Eavg, double *frac)
{
    orc_group_table_w(G, edges, Tbb, 1, sigN, sigE, Eavg, frac);
}


/* ------------------------------------------------------------------ */
/* 6. adjoint (reverse mode) of the step, branch decisions frozen       */
/*    READING: the halving decisions, the dtau sequence and the flux-   */
/*    limit clamp of the forward pass are held fixed (stop-gradient     */
/*    through the dtau selection); everything else is differentiated.   */
/* ------------------------------------------------------------------ */

/* rates at T and their T-derivatives (cgs, per K) */
typedef struct {
    double aA, aB, beta, kR, kC;
    double daA, daB, dbeta, dkR, dkC;
} rates_d;

static void rates_with_derivs(const orc_params *p, double T, rates_d *r)
{
    memset(r, 0, sizeof *r);
    if (p->rates_const) {
        r->aA = p->alphaA; r->aB = p->alphaB; r->beta = p->beta;
        return;
    }
    double l = 2.0 * ORC_T_HI / T;
    double y;
    r->aA = orc_alphaA(T);
    y = pow(l / 0.522, 0.470);
    r->daA = r->aA * (1.503 - 1.923 * 0.470 * y / (1.0 + y)) * (-1.0 / T);
    r->aB = orc_alphaB(T);
    y = pow(l / 2.740, 0.407);
    r->daB = r->aB * (1.500 - 2.242 * 0.407 * y / (1.0 + y)) * (-1.0 / T);
    r->beta = orc_beta(T);
    y = pow(l / 0.354, 0.874);
    r->dbeta = r->beta * (-1.5 + 0.5 * l + 1.089 + 1.101 * 0.874 * y / (1.0 + y)) / T;
    double crec, dcrec;
    if (p->ots) {
        crec = orc_cool_recB(T);
        y = pow(l / 2.250, 0.376);
        dcrec = crec * (1.0 - 1.970 + 3.720 * 0.376 * y / (1.0 + y)) / T;
    } else {
        crec = orc_cool_recA(T);
        y = pow(l / 0.541, 0.502);
        dcrec = crec * (1.0 - 1.965 + 2.697 * 0.502 * y / (1.0 + y)) / T;
    }
    double cff = orc_cool_brems(T), dcff = 0.5 * cff / T;
    double cci = orc_cool_colion(T), dcci = ORC_KB * ORC_T_HI * r->dbeta;
    double cce = orc_cool_colexc(T);
    double dcce = cce * (118348.0 / (T * T) - (0.5 / sqrt(1.0e5 * T)) / (1.0 + sqrt(T / 1.0e5)));
    r->kR = crec + cff;
    r->dkR = dcrec + dcff;
    r->kC = cci + cce;
    r->dkC = dcci + dcce;
}

/* Reverse of one accepted trial (chem_trial) of length dtau from state s.
 * In: adjoints ob of the trial's output.  Out: adjoints sb of its input
 * (overwritten), and dn0 / dS accumulated. */
static void chem_trial_adj(const orc_params *p, double nunit, double n0, const double *S,
                           const cellstate *s, double dtau, const cellstate *ob, cellstate *sb,
                           double *dn0, double *dS)
{
    int G = p->G;
    double c = p->c;
    rates_d r;
    rates_with_derivs(p, s->T, &r);
    double alpha = p->ots ? r.aB : r.aA;
    double x = 1.0 - s->xHI;
    /* forward again, keeping the intermediates */
    double den[ORC_MAXG], N1[ORC_MAXG], F1[ORC_MAXG][3], csig[ORC_MAXG], SigE[ORC_MAXG];
    double rec = (p->ots ? 0.0 : (r.aA - r.aB) * x * x * n0 * n0 / nunit);
    for (int i = 0; i < G; i++) {
        csig[i] = c * p->sigN[i];
        SigE[i] = p->sigE[i] * p->Eavg[i] - p->sigN[i] * ORC_E_HI;
        den[i] = 1.0 + csig[i] * s->xHI * n0 * dtau;
        double src = S[i] + (i == 0 ? rec : 0.0);
        N1[i] = (s->N[i] + src * dtau) / den[i];
        for (int k = 0; k < 3; k++) F1[i][k] = s->F[i][k] / den[i];
    }
    double gam = 0.0;
    for (int i = 0; i < G; i++) gam += csig[i] * nunit * N1[i];
    double A = s->xHI + alpha * x * x * n0 * dtau;
    double Bd = 1.0 + dtau * (r.beta * x * n0 + gam);
    double xHI1 = A / Bd;

    double bN1[ORC_MAXG], bxHI1 = ob->xHI, bT = 0.0, bxHI = 0.0, bx = 0.0, bn0 = 0.0;
    double baA = 0.0, baB = 0.0, bbeta = 0.0, bkR = 0.0, bkC = 0.0, balpha = 0.0;
    for (int i = 0; i < G; i++) bN1[i] = ob->N[i];
    if (p->isothermal) {
        bT += ob->T;
    } else {
        double x1 = 1.0 - xHI1;
        double heat = 0.0;
        for (int i = 0; i < G; i++) heat += c * xHI1 * n0 * (nunit * N1[i]) * SigE[i];
        double Lam = (x1 * n0) * (x1 * n0) * r.kR + (x1 * n0) * (xHI1 * n0) * r.kC;
        double e0 = 1.5 * (1.0 + (1.0 - s->xHI)) * n0 * ORC_KB * s->T;
        double e1 = e0 + dtau * heat - dtau * Lam;
        double W = 1.5 * (1.0 + x1) * n0 * ORC_KB;
        double T1 = e1 / W;
        double be1 = ob->T / W;
        double bW = -ob->T * T1 / W;
        bxHI1 += bW * (-1.5 * n0 * ORC_KB);
        bn0 += bW * 1.5 * (1.0 + x1) * ORC_KB;
        double be0 = be1, bheat = be1 * dtau, bLam = -be1 * dtau;
        /* Lam = n0^2 (x1^2 kR + x1 xHI1 kC), x1 = 1 - xHI1 */
        bxHI1 += bLam * n0 * n0 * (x1 * r.kC - (2.0 * x1 * r.kR + xHI1 * r.kC));
        bn0 += bLam * 2.0 * n0 * (x1 * x1 * r.kR + x1 * xHI1 * r.kC);
        bkR += bLam * n0 * n0 * x1 * x1;
        bkC += bLam * n0 * n0 * x1 * xHI1;
        /* heat = sum_i c xHI1 n0 nunit N1_i SigE_i */
        double hs = 0.0;
        for (int i = 0; i < G; i++) hs += c * nunit * N1[i] * SigE[i];
        bxHI1 += bheat * n0 * hs;
        bn0 += bheat * xHI1 * hs;
        for (int i = 0; i < G; i++) bN1[i] += bheat * c * xHI1 * n0 * nunit * SigE[i];
        /* e0 = 1.5 (2 - xHI) n0 kB T */
        bxHI += be0 * (-1.5 * n0 * ORC_KB * s->T);
        bn0 += be0 * 1.5 * (1.0 + x) * ORC_KB * s->T;
        bT += be0 * 1.5 * (1.0 + x) * n0 * ORC_KB;
    }
    /* xHI1 = A / Bd */
    double bA = bxHI1 / Bd, bBd = -bxHI1 * xHI1 / Bd;
    bxHI += bA;
    balpha += bA * x * x * n0 * dtau;
    bx += bA * 2.0 * alpha * x * n0 * dtau;
    bn0 += bA * alpha * x * x * dtau;
    bbeta += bBd * dtau * x * n0;
    bx += bBd * dtau * r.beta * n0;
    bn0 += bBd * dtau * r.beta * x;
    double bgam = bBd * dtau;
    for (int i = 0; i < G; i++) bN1[i] += bgam * csig[i] * nunit;
    double brec = 0.0;
    for (int i = 0; i < G; i++) {
        double bnum = bN1[i] / den[i];
        double bden = -bN1[i] * N1[i] / den[i];
        for (int k = 0; k < 3; k++) {
            sb->F[i][k] = ob->F[i][k] / den[i];
            bden += -ob->F[i][k] * F1[i][k] / den[i];
        }
        sb->N[i] = bnum;
        double bsrc = bnum * dtau;
        dS[i] += bsrc;
        if (i == 0 && !p->ots) brec += bsrc;
        bxHI += bden * csig[i] * n0 * dtau;
        bn0 += bden * csig[i] * s->xHI * dtau;
    }
    if (!p->ots) {
        double k2 = x * x * n0 * n0 / nunit;
        baA += brec * k2;
        baB -= brec * k2;
        bx += brec * 2.0 * (r.aA - r.aB) * x * n0 * n0 / nunit;
        bn0 += brec * 2.0 * (r.aA - r.aB) * x * x * n0 / nunit;
    }
    if (p->ots) baB += balpha; else baA += balpha;
    bxHI -= bx;
    bT += baA * r.daA + baB * r.daB + bbeta * r.dbeta + bkR * r.dkR + bkC * r.dkC;
    sb->xHI = bxHI;
    sb->T = bT;
    *dn0 += bn0;
}

/* Adjoint of orc_chem_cell: U, xHI, T are the inputs of the forward call;
 * bU (G x 4), bxHI, bT hold the adjoints of its outputs on entry and of its
 * inputs on return; dn0 and dS (G) are accumulated.  Returns the number of
 * accepted trials. */
int orc_chem_cell_adj(const orc_params *p, double dt, double nunit, double n0, const double *S,
                      const double *U, double xHI, double T, double *bU, double *bxHI, double *bT,
                      double *dn0, double *dS)
{
    cellstate s;
    s.G = p->G;
    for (int i = 0; i < p->G; i++) {
        s.N[i] = U[4 * i];
        for (int k = 0; k < 3; k++) s.F[i][k] = U[4 * i + 1 + k];
    }
    s.xHI = xHI;
    s.T = T;
    chem_trace tr = {0, 0, NULL, NULL};
    int ncyc = 0;
    if (p->nsub > 0) {
        double h = dt / p->nsub;
        for (int k = 0; k < p->nsub; k++) chem_span_tr(p, nunit, n0, S, &s, h, 0, &ncyc, &tr);
    } else {
        chem_span_tr(p, nunit, n0, S, &s, dt, 1, &ncyc, &tr);
    }
    cellstate ob;
    ob.G = p->G;
    for (int i = 0; i < p->G; i++) {
        ob.N[i] = bU[4 * i];
        for (int k = 0; k < 3; k++) ob.F[i][k] = bU[4 * i + 1 + k];
    }
    ob.xHI = *bxHI;
    ob.T = *bT;
    for (int t = tr.n - 1; t >= 0; t--) {
        cellstate sb;
        chem_trial_adj(p, nunit, n0, S, &tr.s[t], tr.dtau[t], &ob, &sb, dn0, dS);
        ob = sb;
    }
    for (int i = 0; i < p->G; i++) {
        bU[4 * i] = ob.N[i];
        for (int k = 0; k < 3; k++) bU[4 * i + 1 + k] = ob.F[i][k];
    }
    *bxHI = ob.xHI;
    *bT = ob.T;
    int n = tr.n;
    free(tr.s);
    free(tr.dtau);
    return n;
}

static void jacobian_smooth(int d, const double *u, double f2, double J[4][4]);

/* Jacobian J[r][m] = d G_d[r] / d U[m] of the physical flux along d (the
 * closure P = N D of orc_closure, with its clamp branch frozen). */
void orc_flux_jacobian(int d, const double *U, double J[4][4])
{
    memset(J, 0, sizeof(double) * 16);
    J[0][1 + d] = 1.0;                      /* G_0 = F_d */
    double N = U[0];
    if (!(N > 0.0)) return;
    double u[3] = {U[1] / N, U[2] / N, U[3] / N};
    double f2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (f2 > 1.0) {
        /* P = N uh uh^T, uh = F/|F|: dP/dN = uh uh^T,
           dP_dj/dF_k = (N/|F|)(d_dk uh_j + uh_d d_jk - 2 uh_d uh_j uh_k) */
        double Fn = sqrt(U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
        double uh[3] = {U[1] / Fn, U[2] / Fn, U[3] / Fn};
        for (int j = 0; j < 3; j++) {
            J[1 + j][0] = uh[d] * uh[j];
            for (int k = 0; k < 3; k++)
                J[1 + j][1 + k] = (N / Fn) * ((d == k ? uh[j] : 0.0) + (j == k ? uh[d] : 0.0)
                                              - 2.0 * uh[d] * uh[j] * uh[k]);
        }
        return;
    }
    jacobian_smooth(d, u, f2, J);
}

/* smooth-branch Jacobian of the flux along d at N = 1 (it is homogeneous of
 * degree 0 in (N, F)), velocity u = F/N, f2 = |u|^2 <= 1 */
static void jacobian_smooth(int d, const double *u, double f2, double J[4][4])
{
    memset(J, 0, sizeof(double) * 16);
    J[0][1 + d] = 1.0;
    double s = sqrt(4.0 - 3.0 * f2);
    double a = ((1.0 + s) - 2.0 * f2) / (5.0 + 2.0 * s);
    double g = (6.0 + 3.0 / (2.0 + s)) / (5.0 + 2.0 * s);
    /* derivatives with respect to f2, ds/df2 = -3/(2s) */
    double ds = -1.5 / s;
    double da = ((ds - 2.0) * (5.0 + 2.0 * s) - ((1.0 + s) - 2.0 * f2) * 2.0 * ds)
                / ((5.0 + 2.0 * s) * (5.0 + 2.0 * s));
    double dg = ((-3.0 * ds / ((2.0 + s) * (2.0 + s))) * (5.0 + 2.0 * s)
                 - (6.0 + 3.0 / (2.0 + s)) * 2.0 * ds) / ((5.0 + 2.0 * s) * (5.0 + 2.0 * s));
    for (int j = 0; j < 3; j++) {
        double djd = (j == d) ? 1.0 : 0.0;
        /* dP_dj/dN = (a - 2 f2 a') d_dj - (g + 2 f2 g') u_d u_j */
        J[1 + j][0] = (a - 2.0 * f2 * da) * djd - (g + 2.0 * f2 * dg) * u[d] * u[j];
        /* dP_dj/dF_k = 2 u_k (a' d_dj + g' u_d u_j) + g (d_dk u_j + d_jk u_d) */
        for (int k = 0; k < 3; k++)
            J[1 + j][1 + k] = 2.0 * u[k] * (da * djd + dg * u[d] * u[j])
                              + g * ((d == k ? u[j] : 0.0) + (j == k ? u[d] : 0.0));
    }
}

void orc_flux_jacobian_fmu(double f, double mu, double J[4][4])
{
    double st = 1.0 - mu * mu;
    double u[3] = {f * mu, f * sqrt(st > 0.0 ? st : 0.0), 0.0};
    jacobian_smooth(0, u, f * f, J);
}

/* Adjoint of orc_transport on a periodic box: lamU = (dUs/dU)^T lamS for
 * every group, with
 *   (Us = U* the post-transport state)
 *   lamU_c = lamS_c + (lam/2) sum_d [ J_d(U_c)^T (lamS_{c+d} - lamS_{c-d})
 *                                     + (lamS_{c+d} - 2 lamS_c + lamS_{c-d}) ]
 * (from U*_c = U_c - lam sum_d (Phi_{d,+} - Phi_{d,-}) and Eq. e:glf). */
int orc_transport_adj(const orc_params *p, int nx, int ny, int nz, double lam, const double *U,
                      const double *lamS, double *lamU)
{
    for (int f = 0; f < 6; f++)
        if (p->bc[f] != 0) return -1;
    if (p->flux != 0) return -1;                 /* the adjoint is of the GLF step */
    size_t ncell = (size_t)nx * ny * nz;
    int n[3] = {nx, ny, nz};
    size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
    for (int g = 0; g < p->G; g++) {
        const double *Ug = U + 4 * ncell * g;
        const double *Lg = lamS + 4 * ncell * g;
        double *Og = lamU + 4 * ncell * g;
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    int c[3] = {x, y, z};
                    size_t id = ((size_t)z * ny + y) * nx + x;
                    double acc[4];
                    for (int m = 0; m < 4; m++) acc[m] = 0.0;
                    for (int d = 0; d < 3; d++) {
                        size_t ip = c[d] + 1 < n[d] ? id + stride[d] : id - stride[d] * (n[d] - 1);
                        size_t im = c[d] > 0 ? id - stride[d] : id + stride[d] * (n[d] - 1);
                        double J[4][4], dl[4];
                        orc_flux_jacobian(d, Ug + 4 * id, J);
                        for (int r = 0; r < 4; r++) dl[r] = Lg[4 * ip + r] - Lg[4 * im + r];
                        for (int m = 0; m < 4; m++) {
                            double jt = 0.0;
                            for (int r = 0; r < 4; r++) jt += J[r][m] * dl[r];
                            acc[m] += jt + ((Lg[4 * ip + m] - 2.0 * Lg[4 * id + m]) + Lg[4 * im + m]);
                        }
                    }
                    for (int m = 0; m < 4; m++) Og[4 * id + m] = Lg[4 * id + m] + 0.5 * lam * acc[m];
                }
    }
    return 0;
}

/* Gradient of a loss L(X(1..nsteps)) of the volume-weighted ionised
 * fraction history X(t) = mean(1 - xHI) after step t, for a run of nsteps
 * steps from (U0, xHI0, T0): in dLdX[t-1] = dL/dX(t); out dS[G][ncell]
 * (dL/dS, S in stored units per second) and dn0[ncell].  Plain: the whole
 * trajectory is stored.  Periodic boxes only.  Returns 0 or -1. */
int orc_adjoint(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
                const double *U0, const double *xHI0, const double *T0, const double *n0,
                const double *S, int nsteps, const double *dLdX, double *dS, double *dn0)
{
    for (int f = 0; f < 6; f++)
        if (p->bc[f] != 0) return -1;
    size_t ncell = (size_t)nx * ny * nz;
    int G = p->G;
    size_t nu = 4 * ncell * G;
    double dt = orc_timestep(p, dx);
    double lam = p->c * dt / dx;
    double *Uk = (double *)malloc(sizeof(double) * nu * (nsteps + 1));
    double *Us = (double *)malloc(sizeof(double) * nu * nsteps);
    double *xk = (double *)malloc(sizeof(double) * ncell * (nsteps + 1));
    double *Tk = (double *)malloc(sizeof(double) * ncell * (nsteps + 1));
    double *lU = (double *)calloc(nu, sizeof(double));
    double *lS = (double *)calloc(nu, sizeof(double));
    double *lx = (double *)calloc(ncell, sizeof(double));
    double *lT = (double *)calloc(ncell, sizeof(double));
    if (!Uk || !Us || !xk || !Tk || !lU || !lS || !lx || !lT) return -1;
    memcpy(Uk, U0, sizeof(double) * nu);
    memcpy(xk, xHI0, sizeof(double) * ncell);
    memcpy(Tk, T0, sizeof(double) * ncell);
    for (int k = 0; k < nsteps; k++) {           /* forward, keeping every state */
        double *Un = Uk + nu * (k + 1), *xn = xk + ncell * (k + 1), *Tn = Tk + ncell * (k + 1);
        orc_transport(p, nx, ny, nz, lam, Uk + nu * k, Us + nu * k);
        memcpy(xn, xk + ncell * k, sizeof(double) * ncell);
        memcpy(Tn, Tk + ncell * k, sizeof(double) * ncell);
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 256)
        for (size_t id = 0; id < ncell; id++) {
            double Uc[4 * ORC_MAXG], Sc[ORC_MAXG];
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) Uc[4 * i + m] = Us[nu * k + 4 * (ncell * i + id) + m];
                Sc[i] = S ? S[ncell * i + id] : 0.0;
            }
            orc_chem_cell(p, dt, nunit, n0[id], Sc, Uc, &xn[id], &Tn[id], NULL);
            for (int i = 0; i < G; i++)
                for (int m = 0; m < 4; m++) Un[4 * (ncell * i + id) + m] = Uc[4 * i + m];
        }
    }
    memset(dS, 0, sizeof(double) * G * ncell);
    memset(dn0, 0, sizeof(double) * ncell);
    for (int k = nsteps - 1; k >= 0; k--) {      /* reverse */
        double gx = -dLdX[k] / (double)ncell;    /* X(k+1) = mean(1 - xHI) */
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 256)
        for (size_t id = 0; id < ncell; id++) {
            double Uc[4 * ORC_MAXG], Sc[ORC_MAXG], bU[4 * ORC_MAXG], dSc[ORC_MAXG];
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) {
                    Uc[4 * i + m] = Us[nu * k + 4 * (ncell * i + id) + m];
                    bU[4 * i + m] = lU[4 * (ncell * i + id) + m];
                }
                Sc[i] = S ? S[ncell * i + id] : 0.0;
                dSc[i] = 0.0;
            }
            double bx = lx[id] + gx, bT = lT[id], bn = 0.0;
            orc_chem_cell_adj(p, dt, nunit, n0[id], Sc, Uc, xk[ncell * k + id], Tk[ncell * k + id],
                              bU, &bx, &bT, &bn, dSc);
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) lS[4 * (ncell * i + id) + m] = bU[4 * i + m];
                dS[ncell * i + id] += dSc[i];
            }
            lx[id] = bx;
            lT[id] = bT;
            dn0[id] += bn;
        }
        orc_transport_adj(p, nx, ny, nz, lam, Uk + nu * k, lS, lU);
    }
    free(Uk); free(Us); free(xk); free(Tk); free(lU); free(lS); free(lx); free(lT);
    return 0;
}

/* ------------------------------------------------------------------ */
/* 7. supercomoving units (Sec. 3; R13)                                 */
/* ------------------------------------------------------------------ */
/* R13 The paper transforms to supercomoving variables, N~ = a^3 N r_s^3,
 * F~ = a^4 r_s^2 t_s F, x~ = x/(a r_s), dt~ = dt/(a^2 t_s) (r_s, t_s the
 * length and time units), in which the equations keep their standard form.
 * For the radiation path this makes the transport the usual M1 step with
 * the light speed c~ = a c t_s / r_s, so at the fixed Courant number the
 * transport is unchanged; the thermochemistry acts on physical quantities.
 * The state is stored as
 *   N^ = a^3 N / nunit,  F^ = a^3 F / (c nunit)  (comoving, units of nunit),
 *   T~ = a^2 T           (constant under adiabatic expansion of a
 *                         gamma = 5/3 gas at rest in comoving coordinates),
 * n0 is the comoving hydrogen density (the physical one at a = 1) and dx
 * the comoving cell size.  Step k at a_k:
 *   (1) transport with lam = c dt_com / dx, dt_com = cfl dx / (3 c);
 *   (2) chemistry of every cell over dt_k = a_k dt_com with N, F, S, n0
 *       scaled by 1/a_k^3 and T = T~ / a_k^2;
 *   (3) back to the stored units with a_k^3 and T~ = a_k^2 T; F^ also by
 *       a_k / a_(k+1), since F^ follows F~ / c~ and c~ grows like a;
 *   (4) a_(k+1) from a_k over dt_k by the Friedmann equation
 *       da/dt = a H0 sqrt(Om / a^3 + OL), one classical Runge-Kutta step. */
static double dadt_cosmo(double a, double H0, double Om, double OL)
{
    return a * H0 * sqrt(Om / (a * a * a) + OL);
}

double orc_advance_a(double a, double dt, double H0, double Om, double OL)
{
    double k1 = dadt_cosmo(a, H0, Om, OL);
    double k2 = dadt_cosmo(a + 0.5 * dt * k1, H0, Om, OL);
    double k3 = dadt_cosmo(a + 0.5 * dt * k2, H0, Om, OL);
    double k4 = dadt_cosmo(a + dt * k3, H0, Om, OL);
    return a + dt * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
}

int orc_run_cosmo(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
                  double *U, double *xHI, double *T, const double *n0, const double *S,
                  int nsteps, double *hist, double H0, double Om, double OL, double *a_io)
{
    size_t ncell = (size_t)nx * ny * nz;
    int G = p->G;
    double *Us = (double *)malloc(sizeof(double) * 4 * ncell * G);
    if (!Us) return -1;
    double dt_com = orc_timestep(p, dx);
    double lam = p->c * dt_com / dx;
    double a = *a_io;
    int err = 0;
    for (int step = 0; step < nsteps; step++) {
        double dtk = a * dt_com;
        double a1 = orc_advance_a(a, dtk, H0, Om, OL);
        double ia3 = 1.0 / (a * a * a), a3 = a * a * a, a2 = a * a, fr = a / a1;
        orc_transport(p, nx, ny, nz, lam, U, Us);
        double cyc_sum = 0.0;
#pragma omp parallel for num_threads(orc_threads) schedule(dynamic, 256) reduction(|:err) reduction(+:cyc_sum)
        for (size_t id = 0; id < ncell; id++) {
            double Uc[4 * ORC_MAXG], Sc[ORC_MAXG];
            for (int i = 0; i < G; i++) {
                for (int m = 0; m < 4; m++) Uc[4 * i + m] = Us[4 * (ncell * i + id) + m] * ia3;
                Sc[i] = S ? S[ncell * i + id] * ia3 : 0.0;
            }
            double Tp = T[id] / a2;
            int ncyc = 0;
            err |= orc_chem_cell(p, dtk, nunit, n0[id] * ia3, Sc, Uc, &xHI[id], &Tp, &ncyc);
            for (int i = 0; i < G; i++) {
                U[4 * (ncell * i + id)] = Uc[4 * i] * a3;
                for (int m = 1; m < 4; m++) U[4 * (ncell * i + id) + m] = Uc[4 * i + m] * a3 * fr;
            }
            T[id] = Tp * a2;
            cyc_sum += ncyc;
        }
        if (hist) {
            double X = 0.0, ph = 0.0, nion = 0.0;
            for (size_t id = 0; id < ncell; id++) {
                X += 1.0 - xHI[id];
                if (xHI[id] < 0.5) nion += 1.0;
            }
            for (size_t k = 0; k < ncell * G; k++) ph += U[4 * k];
            double *h = hist + 5 * (size_t)step;
            h[0] = X / (double)ncell;
            h[1] = ph * nunit * (dx * dx * dx);
            h[2] = 0.0;
            h[3] = nion;
            h[4] = cyc_sum / (double)ncell;
        }
        a = a1;
    }
    free(Us);
    *a_io = a;
    return err;
}
