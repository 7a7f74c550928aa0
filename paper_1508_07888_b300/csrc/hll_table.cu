// hll_table.cu -- host-side wave-speed table of the HLL flux.
//
// The HLL flux needs the extreme eigenvalues (signal speeds, units of c) of
// the Jacobian of the M1 flux along the face normal.  They depend on
// f = |F|/(cN) and mu = F_d/|F| only.  The table holds lambda_max at
// f_i = 1 - (i/nf)^2 (i = 0..nf, so i = 0 is f = 1) and mu_j = -1 + 2j/nm;
// the kernels interpolate it bilinearly in (sqrt(1 - f), mu), where it is
// smooth, and take lambda_min(f, mu) = -lambda_max(f, -mu).
//
// Jacobian of the x flux (F_x, P_xx, P_xy, P_xz) at N = 1, F = f (mu, nu, 0),
// nu = sqrt(1 - mu^2), with P = N a(w) I + b(w) F F^T / N, w = |F|^2/N^2,
// a = (1 + s - 2w)/(5 + 2s), b = (6 + 3/(2 + s))/(5 + 2s), s = sqrt(4 - 3w)
// (the Levermore closure): with u = F/N,
//   dP_ij/dN   = (a - 2 w a') d_ij - (b + 2 w b') u_i u_j
//   dP_ij/dF_k = 2 u_k (a' d_ij + b' u_i u_j) + b (d_ik u_j + u_i d_jk)
// (' = d/dw, here by forward-mode differentiation with dual numbers).  With
// F_z = 0 the F_z mode decouples (eigenvalue b u_x); the other three are the
// roots of the cubic characteristic polynomial of the (N, F_x, F_y) block,
// whose largest root Newton's method reaches monotonically from above.  At
// f = 1 all four eigenvalues equal mu (free streaming), a repeated root
// that is set exactly.
#include <cmath>

#include "../../include/rt_m1.h"

namespace {

typedef long double LD;

struct Dual {            // value and derivative with respect to w
    LD v, d;
};
Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
Dual cst(LD c) { return {c, 0}; }
Dual dsqrt(Dual a)
{
    const LD r = sqrtl(a.v);
    return {r, a.d / (2 * r)};
}

LD lambda_max_at(LD f, LD mu)
{
    if (f >= 1) return mu;
    const LD nu = sqrtl(fmaxl(0, 1 - mu * mu));
    const LD u[3] = {f * mu, f * nu, 0};
    const Dual w = {f * f, 1};
    const Dual s = dsqrt(cst(4) - cst(3) * w);
    const Dual den = cst(5) + cst(2) * s;
    const Dual a = (cst(1) + s - cst(2) * w) / den;
    const Dual b = (cst(6) + cst(3) / (cst(2) + s)) / den;
    // rows/columns (N, F_x, F_y) of the x-flux Jacobian
    LD J[3][3] = {{0, 1, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < 2; i++) {          // P_xx (row 1), P_xy (row 2)
        const int pi = 0, pj = i;          // P_{x, x} and P_{x, y}
        const LD dij = pi == pj ? 1 : 0;
        J[1 + i][0] = (a.v - 2 * w.v * a.d) * dij - (b.v + 2 * w.v * b.d) * u[pi] * u[pj];
        for (int k = 0; k < 2; k++)
            J[1 + i][1 + k] = 2 * u[k] * (a.d * dij + b.d * u[pi] * u[pj]) +
                              b.v * ((pi == k ? u[pj] : 0) + (pj == k ? u[pi] : 0));
    }
    const LD lz = b.v * u[0];              // the decoupled F_z mode
    // characteristic polynomial lambda^3 - c2 lambda^2 + c1 lambda - c0
    const LD c2 = J[0][0] + J[1][1] + J[2][2];
    const LD c1 = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) + (J[0][0] * J[2][2] - J[0][2] * J[2][0]) +
                  (J[1][1] * J[2][2] - J[1][2] * J[2][1]);
    const LD c0 = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                  J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    LD x = 2;                              // above every root (speeds <= 1)
    for (int it = 0; it < 400; it++) {
        const LD p = ((x - c2) * x + c1) * x - c0;
        const LD dp = (3 * x - 2 * c2) * x + c1;
        if (!(dp > 0)) break;
        const LD nx = x - p / dp;
        if (!(nx < x)) break;              // converged (monotone from above)
        x = nx;
    }
    return x > lz ? x : lz;
}

}  // namespace

extern "C" RT_API int rt_hll_speeds(int nf, int nm, double *lmax)
{
    if (nf < 1 || nm < 1 || !lmax) return RT_ERR_ARG;
    for (int i = 0; i <= nf; i++) {
        const LD z = (LD)i / nf;
        const LD f = 1 - z * z;
        for (int j = 0; j <= nm; j++) {
            const LD mu = -1 + 2 * (LD)j / nm;
            lmax[(size_t)i * (nm + 1) + j] = (double)lambda_max_at(f, mu);
        }
    }
    return RT_OK;
}
