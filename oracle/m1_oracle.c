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
 *      parity unpinned beyond alpha_A/alpha_B at 5e3, 1e4, 2e4 K (textbook).
 *   R9 photo-ionisation cross-section: the exact hydrogenic form
 *      sigma = A0 (E1/E)^4 exp(4 - 4 atan(eps)/eps)/(1 - exp(-2 pi/eps)),
 *      eps = sqrt(E/E1 - 1), A0 = 6.30e-18 cm^2, E1 = 13.6 eV.
 *   R10 group averages (Eq. e:siggroup and the sigma_E, <E> definitions) over
 *      a black-body photon spectrum; source photons split by the group
 *      fraction of that spectrum (Eq. e:sgroup).
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

/* neighbour state of cell (x,y,z) along axis d, side = -1 or +1, with the
 * global boundary conditions of Sec. 4.2: periodic by default; transmissive
 * copies the cell itself; reflective copies it and inverts the normal flux. */
static void neighbour(const orc_params *p, const double *Ug, int nx, int ny, int nz,
                      int x, int y, int z, int d, int side, double *out)
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
                                neighbour(p, Ug, nx, ny, nz, x, y, z, d, sgn, Us[side]);
                                orc_closure(Us[side], Pg, NULL, NULL);
                                flux_from(d, Us[side], Pg, Gs[side]);
                            }
                        }
                        for (int m = 0; m < 4; m++) {
                            /* Eq. e:glf at faces i-1/2 (left neighbour, cell) and i+1/2 */
                            double Fm = 0.5 * ((Gs[0][m] + Gc[m]) - (Uc[m] - Us[0][m]));
                            double Fp = 0.5 * ((Gc[m] + Gs[1][m]) - (Us[1][m] - Uc[m]));
                            diff[d][m] = Fp - Fm;
                        }
                    }
                    for (int m = 0; m < 4; m++)
                        Og[4 * id + m] = Uc[m] - lam * ((diff[0][m] + diff[1][m]) + diff[2][m]);
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
                neighbour(p, Ug, nx, ny, nz, x, y, z, d, side ? +1 : -1, Us[side]);
                orc_closure(Us[side], Ps, NULL, NULL);
                flux_from(d, Us[side], Ps, Gs[side]);
            }
            for (int m = 0; m < 4; m++) {
                double Fm = 0.5 * ((Gs[0][m] + Gc[m]) - (Uc[m] - Us[0][m]));
                double Fp = 0.5 * ((Gc[m] + Gs[1][m]) - (Us[1][m] - Uc[m]));
                diff[d][m] = Fp - Fm;
            }
        }
        for (int m = 0; m < 4; m++)
            out[4 * k + m] = Uc[m] - lam * ((diff[0][m] + diff[1][m]) + diff[2][m]);
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

/* advance one cell over a span of time with sub-cycles (R4) */
static int chem_span(const orc_params *p, double nunit, double n0, const double *S,
                     cellstate *s, double span, int use_estimate, int *ncyc)
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
int orc_run(const orc_params *p, int nx, int ny, int nz, double dx, double nunit,
            double *U, double *xHI, double *T, const double *n0, const double *S,
            int nsteps, double *hist, int64_t *nclamp_out)
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
        /* realizability after transport: |F| <= cN (1 + 1e-12) */
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
        if (hist) {
            double X = 0.0, ph = 0.0, fmax = 0.0, nion = 0.0;
            for (size_t id = 0; id < ncell; id++) {
                X += 1.0 - xHI[id];
                if (xHI[id] < 0.5) nion += 1.0;
            }
            for (size_t k = 0; k < ncell * G; k++) {
                double N = U[4 * k];
                ph += N;
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
            h[3] = nion;
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
