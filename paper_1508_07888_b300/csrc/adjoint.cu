// adjoint.cu -- reverse-mode kernels of one radiative step (FP64), used by
// rt_adjoint.
//
// The forward step is  U* = Transport(U),  (U', xHI', T') = Chem(U*, xHI, T;
// n0, S).  Its adjoint, with the branch decisions of the forward pass frozen
// (the halvings of the 10% rule, the dtau sequence, the flux-limit clamp),
// runs the chemistry adjoint and then the transport adjoint:
//   * k_chem_adj: per cell, recompute the accepted sub-cycles of the forward
//     chemistry from (U*, xHI, T), keep their input states, and walk them
//     backwards through the hand-written reverse of one trial; accumulate
//     dL/dn0 of the cell and dL/dS of its source;
//   * k_transport_adj: lamU_c = lamS_c + (lam/2) sum_d [ J_d(U_c)^T
//     (lamS_{c+d} - lamS_{c-d}) + (lamS_{c+d} - 2 lamS_c + lamS_{c-d}) ],
//     the transpose of the unsplit GLF update (Eq. e:uprt with Eq. e:glf) on
//     a periodic box, J_d the Jacobian of the physical flux along d.
#define RTK_SKIP_SINGLE_KERNELS 1
#include <algorithm>

#include "launch.h"
#include "rt_kernels.cuh"

namespace rta {

using namespace rtk;

constexpr int MAXTR = 32;   // accepted trials kept per cell and step

struct RatesD {
    double aA, aB, beta, kR, kC;
    double daA, daB, dbeta, dkR, dkC;   // d/dT
};

// the fits evaluated directly, with their T derivatives
__device__ RatesD rates_d_exact(const Phys &ph, double T)
{
    RatesD r;
    const Rates v = rates_at(ph, T);
    r.aA = v.aA; r.aB = v.aB; r.beta = v.beta; r.kR = v.kR; r.kC = v.kC;
    if (ph.rates_const) {
        r.daA = r.daB = r.dbeta = r.dkR = r.dkC = 0.0;
        return r;
    }
    const double l = 2.0 * rtd::T_HI / T, iT = 1.0 / T;
    double y;
    y = exp(0.407 * (log(l) - ph.lnfit[1]));
    r.daB = -r.aB * (1.500 - 2.242 * 0.407 * y / (1.0 + y)) * iT;
    if (ph.ots) {
        r.daA = r.daB;
    } else {
        y = exp(0.470 * (log(l) - ph.lnfit[0]));
        r.daA = -r.aA * (1.503 - 1.923 * 0.470 * y / (1.0 + y)) * iT;
    }
    y = exp(0.874 * (log(l) - ph.lnfit[2]));
    r.dbeta = r.beta * (-1.5 + 0.5 * l + 1.089 + 1.101 * 0.874 * y / (1.0 + y)) * iT;
    const double sT = sqrt(T);
    const double cff = 1.42e-27 * 1.3 * sT;
    const double crec = r.kR - cff;
    double dcrec;
    if (ph.ots) {
        y = exp(0.376 * (log(l) - ph.lnfit[4]));
        dcrec = crec * (1.0 - 1.970 + 3.720 * 0.376 * y / (1.0 + y)) * iT;
    } else {
        y = exp(0.502 * (log(l) - ph.lnfit[3]));
        dcrec = crec * (1.0 - 1.965 + 2.697 * 0.502 * y / (1.0 + y)) * iT;
    }
    const double cce = r.kC - rtd::KB * rtd::T_HI * r.beta;
    const double dcce = cce * (118348.0 * iT * iT - (0.5 / sqrt(1.0e5 * T)) / (1.0 + sqrt(T * 1e-5)));
    r.dkR = dcrec + 0.5 * cff * iT;
    r.dkC = rtd::KB * rtd::T_HI * r.dbeta + dcce;
    return r;
}

// the tabulated rates of the forward pass (rates_tab), differentiated
// through the interpolating polynomials in their variable t (t = -1 at the
// interval's start, 1 at its end): d/dT = (dt/dT) d/dt, with
// dt/dT = 2 / (interval width) = 2^(SUB + 1 - e)
__device__ RatesD rates_d(const Phys &ph, const RateCoef *tab, double T)
{
    if (!tab || ph.rates_const) return rates_d_exact(ph, T);
    int j;
    double t;
    float t32;
    if (!tab_pos(T, j, t, t32)) return rates_d_exact(ph, T);
    const int e = (int)(__double_as_longlong(T) >> 52) - 1023;
    const double dtdT = ldexp(1.0, RTD_TAB_SUB + 1 - e);
    const RateCoef *a = tab + (size_t)j * RTD_TAB_NF;
    double g[RTD_TAB_NF], dg[RTD_TAB_NF];
    for (int f = 0; f < RTD_TAB_NF; f++) {
        const RateCoef &c = a[f];
        g[f] = tab_eval(&c, t, t32);
        const double dp = fma(fma(fma(fma(5.0 * (double)c.c5, t, 4.0 * (double)c.c4), t,
                                      3.0 * (double)c.c3), t, 2.0 * c.c2), t, c.c1);
        dg[f] = dp * dtdT;
    }
    RatesD r;
    r.aB = g[1];
    r.daB = dg[1];
    r.aA = ph.ots ? g[1] : g[0];
    r.daA = ph.ots ? dg[1] : dg[0];
    r.kR = g[2];
    r.dkR = dg[2];
    if (T >= RTD_TAB_TCUT) {
        const double invT = 1.0 / T;
        r.beta = exp(g[3] - rtd::T_HI * invT);
        r.dbeta = r.beta * (dg[3] + rtd::T_HI * invT * invT);
        const double cce = exp(g[4] - 118348.0 * invT);
        const double dcce = cce * (dg[4] + 118348.0 * invT * invT);
        r.kC = rtd::KB * rtd::T_HI * r.beta + cce;
        r.dkC = rtd::KB * rtd::T_HI * r.dbeta + dcce;
    } else {                       // both factors are exactly zero here
        r.beta = r.dbeta = 0.0;
        r.kC = r.dkC = 0.0;
    }
    return r;
}

// Reverse of one accepted trial (chem_trial) of length dtau from state s:
// ob = adjoint of its output, returns the adjoint of its input; adds to
// bn0 and bS.
template <int G>
__device__ Cell<G> trial_adj(const Phys &ph, const RateCoef *tab, double nunit, double n0,
                             const double *S, const Cell<G> &s, double dtau, const Cell<G> &ob,
                             double &bn0, double *bS)
{
    const RatesD r = rates_d(ph, tab, s.T);
    const double c = ph.c;
    const double alpha = ph.ots ? r.aB : r.aA;
    const double x = 1.0 - s.xHI;
    const double rec = ph.ots ? 0.0 : (r.aA - r.aB) * x * x * n0 * n0 / nunit;
    double den[G], N1[G], F1[G][3];
    double gam = 0.0;
#pragma unroll
    for (int i = 0; i < G; i++) {
        den[i] = 1.0 + ph.csig[i] * s.xHI * n0 * dtau;
        const double src = S[i] + (i == 0 ? rec : 0.0);
        N1[i] = (s.N[i] + src * dtau) / den[i];
#pragma unroll
        for (int k = 0; k < 3; k++) F1[i][k] = s.F[i][k] / den[i];
        gam += ph.csig[i] * nunit * N1[i];
    }
    const double A = s.xHI + alpha * x * x * n0 * dtau;
    const double Bd = 1.0 + dtau * (r.beta * x * n0 + gam);
    const double xHI1 = A / Bd;

    Cell<G> sb;
    double bN1[G];
#pragma unroll
    for (int i = 0; i < G; i++) bN1[i] = ob.N[i];
    double bxHI1 = ob.xHI, bT = 0.0, bxHI = 0.0, bx = 0.0;
    double balpha = 0.0, baA = 0.0, baB = 0.0, bbeta = 0.0, bkR = 0.0, bkC = 0.0;
    if (ph.isothermal) {
        bT += ob.T;
    } else {
        const double x1 = 1.0 - xHI1;
        double hs = 0.0;                                    // sum c nunit N1 SigE
#pragma unroll
        for (int i = 0; i < G; i++) hs += c * nunit * N1[i] * ph.SigE[i];
        const double heat = xHI1 * n0 * hs;
        const double Lam = (x1 * n0) * (x1 * n0) * r.kR + (x1 * n0) * (xHI1 * n0) * r.kC;
        const double e0 = 1.5 * (1.0 + x) * n0 * rtd::KB * s.T;
        const double e1 = e0 + dtau * heat - dtau * Lam;
        const double W = 1.5 * (1.0 + x1) * n0 * rtd::KB;
        const double T1 = e1 / W;
        const double be1 = ob.T / W;
        const double bW = -ob.T * T1 / W;
        bxHI1 += bW * (-1.5 * n0 * rtd::KB);
        bn0 += bW * 1.5 * (1.0 + x1) * rtd::KB;
        const double bheat = be1 * dtau, bLam = -be1 * dtau;
        bxHI1 += bLam * n0 * n0 * (x1 * r.kC - (2.0 * x1 * r.kR + xHI1 * r.kC));
        bn0 += bLam * 2.0 * n0 * (x1 * x1 * r.kR + x1 * xHI1 * r.kC);
        bkR += bLam * n0 * n0 * x1 * x1;
        bkC += bLam * n0 * n0 * x1 * xHI1;
        bxHI1 += bheat * n0 * hs;
        bn0 += bheat * xHI1 * hs;
#pragma unroll
        for (int i = 0; i < G; i++) bN1[i] += bheat * c * xHI1 * n0 * nunit * ph.SigE[i];
        bxHI += be1 * (-1.5 * n0 * rtd::KB * s.T);
        bn0 += be1 * 1.5 * (1.0 + x) * rtd::KB * s.T;
        bT += be1 * 1.5 * (1.0 + x) * n0 * rtd::KB;
    }
    const double bA = bxHI1 / Bd, bBd = -bxHI1 * xHI1 / Bd;
    bxHI += bA;
    balpha += bA * x * x * n0 * dtau;
    bx += bA * 2.0 * alpha * x * n0 * dtau;
    bn0 += bA * alpha * x * x * dtau;
    bbeta += bBd * dtau * x * n0;
    bx += bBd * dtau * r.beta * n0;
    bn0 += bBd * dtau * r.beta * x;
    const double bgam = bBd * dtau;
    double brec = 0.0;
#pragma unroll
    for (int i = 0; i < G; i++) {
        bN1[i] += bgam * ph.csig[i] * nunit;
        const double bnum = bN1[i] / den[i];
        double bden = -bN1[i] * N1[i] / den[i];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            sb.F[i][k] = ob.F[i][k] / den[i];
            bden -= ob.F[i][k] * F1[i][k] / den[i];
        }
        sb.N[i] = bnum;
        const double bsrc = bnum * dtau;
        bS[i] += bsrc;
        if (i == 0) brec += bsrc;
        bxHI += bden * ph.csig[i] * n0 * dtau;
        bn0 += bden * ph.csig[i] * s.xHI * dtau;
    }
    if (!ph.ots) {
        const double k2 = x * x * n0 * n0 / nunit;
        baA += brec * k2;
        baB -= brec * k2;
        bx += brec * 2.0 * (r.aA - r.aB) * x * n0 * n0 / nunit;
        bn0 += brec * 2.0 * (r.aA - r.aB) * x * x * n0 / nunit;
    }
    if (ph.ots) baB += balpha; else baA += balpha;
    bxHI -= bx;
    bT += baA * r.daA + baB * r.daB + bbeta * r.dbeta + bkR * r.dkR + bkC * r.dkC;
    sb.xHI = bxHI;
    sb.T = bT;
    return sb;
}

// accepted trials with index in [lo, lo + MAXTR) of one forward replay
template <int G>
struct TraceBuf {
    Cell<G> s[MAXTR];
    double dt[MAXTR];
    int lo = 0, idx = 0;
    __device__ __forceinline__ void push(const Cell<G> &c, double d)
    {
        const int j = idx - lo;
        if (j >= 0 && j < MAXTR) { s[j] = c; dt[j] = d; }
        idx++;
    }
};

// One thread per cell: adjoint of the chemistry of step k.  Us, xk, Tk: the
// step's post-transport radiation state and its (xHI, T) before chemistry.
// lamU in: adjoint of U after the step; out: adjoint of U*.  lamx/lamT: in
// after, out before.  gx = dL/dX(k+1) * (-1/ncell) is added to lamx first.
template <int G>
__global__ void __launch_bounds__(128)
k_chem_adj(const BoxDev *__restrict__ boxes, Phys ph, const double *__restrict__ Us,
           const double *__restrict__ xk, const double *__restrict__ Tk, double *lamU,
           double *lamx, double *lamT, double gx, double *dn0, double *dS, unsigned *err)
{
    const BoxDev &B = boxes[0];
    const RateCoef *tab = ph.rates_const ? nullptr : ph.rtab;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < B.ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        Cell<G> s;
        for (int i = 0; i < G; i++) {
            const double *u = Us + 4 * ((int64_t)i * B.ncell + c);
            s.N[i] = u[0];
            s.F[i][0] = u[1]; s.F[i][1] = u[2]; s.F[i][2] = u[3];
        }
        s.xHI = xk[c];
        s.T = Tk[c];
        const double n0 = reinterpret_cast<const double *>(B.n0)[c];
        double S[G];
        int src = -1;
        for (int i = 0; i < G; i++) S[i] = 0.0;
        if (B.nsrc > 0) {
            int lo = 0, hi = B.nsrc - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (B.src_cell[mid] < c) lo = mid + 1; else hi = mid;
            }
            if (B.src_cell[lo] == c) {
                src = lo;
                for (int i = 0; i < G; i++) S[i] = B.src_S[(int64_t)lo * G + i];
            }
        }
        // forward replay of the cell's chemistry, recording the window of
        // accepted trials [lo, lo + MAXTR)
        TraceBuf<G> tr;
        auto replay = [&](int lo) {
            Cell<G> w = s;
            tr.lo = lo;
            tr.idx = 0;
            int ncyc = 0;
            if (ph.nsub > 0) {
                const double h = B.dt / ph.nsub;
                for (int k = 0; k < ph.nsub; k++)
                    chem_span<G, false, TraceBuf<G>, double>(ph, tab, B, n0, S, w, h, false, ncyc, &tr, nullptr, false,
                                                   nullptr, d2f(h));
            } else {
                chem_span<G, false, TraceBuf<G>, double>(ph, tab, B, n0, S, w, B.dt, true, ncyc, &tr, nullptr, false,
                                               nullptr, d2f(B.dt));
            }
        };
        replay(0);
        const int ntr = tr.idx;
        const int nwin = (ntr + MAXTR - 1) / MAXTR;
        if (nwin > 64) atomicOr(err, RTD_ERR_SUBCYCLE);    // > 2048 trials: give up on the cell
        Cell<G> ob;
        for (int i = 0; i < G; i++) {
            const double *l = lamU + 4 * ((int64_t)i * B.ncell + c);
            ob.N[i] = l[0];
            ob.F[i][0] = l[1]; ob.F[i][1] = l[2]; ob.F[i][2] = l[3];
        }
        ob.xHI = lamx[c] + gx;
        ob.T = lamT[c];
        double bn0 = 0.0, bS[G];
        for (int i = 0; i < G; i++) bS[i] = 0.0;
        for (int wdx = (nwin > 64 ? 0 : nwin - 1); wdx >= 0; wdx--) {
            if (wdx != 0 || nwin > 1) replay(wdx * MAXTR);
            const int hi = min(MAXTR, ntr - wdx * MAXTR);
            for (int t = hi - 1; t >= 0; t--)
                ob = trial_adj<G>(ph, tab, B.nunit, n0, S, tr.s[t], tr.dt[t], ob, bn0, bS);
        }
        for (int i = 0; i < G; i++) {
            double *l = lamU + 4 * ((int64_t)i * B.ncell + c);
            l[0] = ob.N[i];
            l[1] = ob.F[i][0]; l[2] = ob.F[i][1]; l[3] = ob.F[i][2];
        }
        lamx[c] = ob.xHI;
        lamT[c] = ob.T;
        dn0[c] += bn0;
        if (src >= 0)
            for (int i = 0; i < G; i++) dS[(int64_t)src * G + i] += bS[i];
    }
}

// Jacobian J[r][m] = dG_d[r]/dU[m] of the physical flux (F_d, P_d.) along d
__device__ void flux_jacobian(int d, const double U[4], double J[4][4])
{
    for (int r = 0; r < 4; r++)
        for (int m = 0; m < 4; m++) J[r][m] = 0.0;
    J[0][1 + d] = 1.0;
    const double N = U[0];
    if (!(N > 0.0)) return;
    const double u[3] = {U[1] / N, U[2] / N, U[3] / N};
    const double f2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (f2 > 1.0) {                 // clamped: P = N uh uh^T, uh = F/|F|
        const double Fn = sqrt(U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
        const double uh[3] = {U[1] / Fn, U[2] / Fn, U[3] / Fn};
        for (int j = 0; j < 3; j++) {
            J[1 + j][0] = uh[d] * uh[j];
            for (int k = 0; k < 3; k++)
                J[1 + j][1 + k] = (N / Fn) * ((d == k ? uh[j] : 0.0) + (j == k ? uh[d] : 0.0) -
                                              2.0 * uh[d] * uh[j] * uh[k]);
        }
        return;
    }
    const double s = sqrt(4.0 - 3.0 * f2);
    const double q = 5.0 + 2.0 * s;
    const double a = ((1.0 + s) - 2.0 * f2) / q;
    const double gn = 6.0 + 3.0 / (2.0 + s);
    const double g = gn / q;
    const double ds = -1.5 / s;                                   // ds/df2
    const double da = ((ds - 2.0) * q - ((1.0 + s) - 2.0 * f2) * 2.0 * ds) / (q * q);
    const double dg = ((-3.0 * ds / ((2.0 + s) * (2.0 + s))) * q - gn * 2.0 * ds) / (q * q);
    for (int j = 0; j < 3; j++) {
        const double djd = (j == d) ? 1.0 : 0.0;
        J[1 + j][0] = (a - 2.0 * f2 * da) * djd - (g + 2.0 * f2 * dg) * u[d] * u[j];
        for (int k = 0; k < 3; k++)
            J[1 + j][1 + k] = 2.0 * u[k] * (da * djd + dg * u[d] * u[j]) +
                              g * ((d == k ? u[j] : 0.0) + (j == k ? u[d] : 0.0));
    }
}

// transpose of the periodic unsplit GLF update, one thread per (group, cell)
__global__ void __launch_bounds__(256)
k_transport_adj(const BoxDev *__restrict__ boxes, int G, const double *__restrict__ U,
                const double *__restrict__ lamS, double *__restrict__ lamU)
{
    const BoxDev &B = boxes[0];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int64_t ncell = B.ncell;
    const double lam = B.lam;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < G * ncell;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / ncell);
        const int64_t c = t - (int64_t)g * ncell;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
        const double *Ug = U + 4 * (int64_t)g * ncell;
        const double *Lg = lamS + 4 * (int64_t)g * ncell;
        double u[4], lc[4], acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int m = 0; m < 4; m++) { u[m] = Ug[4 * c + m]; lc[m] = Lg[4 * c + m]; }
        const int co[3] = {x, y, z}, n[3] = {nx, ny, nz};
        const int64_t st[3] = {1, nx, (int64_t)nx * ny};
        for (int d = 0; d < 3; d++) {
            const int64_t ip = co[d] + 1 < n[d] ? c + st[d] : c - st[d] * (n[d] - 1);
            const int64_t im = co[d] > 0 ? c - st[d] : c + st[d] * (n[d] - 1);
            double J[4][4];
            flux_jacobian(d, u, J);
            double lp[4], lm[4];
            for (int m = 0; m < 4; m++) { lp[m] = Lg[4 * ip + m]; lm[m] = Lg[4 * im + m]; }
            for (int m = 0; m < 4; m++) {
                double jt = 0.0;
                for (int r = 0; r < 4; r++) jt += J[r][m] * (lp[r] - lm[r]);
                acc[m] += jt + ((lp[m] - 2.0 * lc[m]) + lm[m]);
            }
        }
        for (int m = 0; m < 4; m++) lamU[4 * (int64_t)g * ncell + 4 * c + m] = lc[m] + 0.5 * lam * acc[m];
    }
}

}  // namespace rta

namespace rtl {

cudaError_t chem_adj(int G, const rtd::BoxDev *boxes, const rtd::Phys &ph, const double *Us,
                     const double *xk, const double *Tk, double *lamU, double *lamx, double *lamT,
                     double gx, double *dn0, double *dS, unsigned *err, int64_t ncell,
                     cudaStream_t s)
{
    const int threads = 128;
    const int grid = (int)std::min<int64_t>((ncell + threads - 1) / threads, 148 * 16);
#define CA(g)                                                                                     \
    rta::k_chem_adj<g><<<grid, threads, 0, s>>>(boxes, ph, Us, xk, Tk, lamU, lamx, lamT, gx, dn0, \
                                                dS, err)
    switch (G) {
    case 1: CA(1); break;
    case 2: CA(2); break;
    case 3: CA(3); break;
    case 4: CA(4); break;
    default: return cudaErrorInvalidValue;
    }
#undef CA
    return cudaGetLastError();
}

cudaError_t transport_adj(int G, const rtd::BoxDev *boxes, const double *U, const double *lamS,
                          double *lamU, int64_t ncell, cudaStream_t s)
{
    const int threads = 256;
    const int grid = (int)std::min<int64_t>((G * ncell + threads - 1) / threads, 148 * 32);
    rta::k_transport_adj<<<grid, threads, 0, s>>>(boxes, G, U, lamS, lamU);
    return cudaGetLastError();
}

}  // namespace rtl
