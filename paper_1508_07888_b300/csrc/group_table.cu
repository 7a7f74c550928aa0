// group_table.cu -- host-side group averages of the hydrogen
// photo-ionisation cross-section over a black-body source spectrum
// (Eq. e:siggroup, the sigma_E and <E> definitions of Sec. 2.2.4, and the
// group photon share of Eq. e:sgroup).  Runs once, at set-up.
//
// Quadrature: 16-point Gauss-Legendre on 256 equal panels in u = ln E per
// group; nodes from Newton iteration on the Legendre recurrence.
#include <cmath>

#include "../../include/rt_m1.h"

namespace {

constexpr double KB = 1.380649e-16;
constexpr double EV = 1.602176634e-12;
constexpr double E_TH = 13.6;     // eV, hydrogen ionisation threshold
constexpr double SIG0 = 6.30e-18; // cm^2, threshold cross-section

// exact hydrogenic 1s photo-ionisation cross-section (Menzel-Pekeris form):
// sigma = sigma0 (E_th/E)^4 exp(4 - 4 atan(e)/e) / (1 - exp(-2 pi / e)),
// e = sqrt(E/E_th - 1)
double sigma_hydrogenic(double E)
{
    if (E < E_TH) return 0.0;
    const double r = E / E_TH;
    const double e = std::sqrt(r - 1.0);
    if (e < 1e-6) return SIG0;
    const double q = 1.0 / (r * r);
    return SIG0 * q * q * std::exp(4.0 - 4.0 * std::atan(e) / e) /
           (-std::expm1(-2.0 * M_PI / e));
}

void legendre_nodes(int n, double *x, double *w)
{
    for (int i = 0; i < n; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

extern "C" int rt_group_table(int G, const double *edges, double T_bb, double *sigN, double *sigE,
                              double *Eavg, double *frac)
{
    if (G < 1 || G > RT_MAX_GROUPS || !edges || !sigN || !sigE || !Eavg || !frac)
        return RT_ERR_ARG;
    if (!(T_bb > 0) || !(edges[0] >= E_TH)) return RT_ERR_ARG;
    for (int i = 0; i < G; i++)
        if (!(edges[i + 1] > edges[i]) || !std::isfinite(edges[i + 1])) return RT_ERR_ARG;
    const int NP = 256, NQ = 16;
    double xq[NQ], wq[NQ];
    legendre_nodes(NQ, xq, wq);
    const double kT = KB * T_bb / EV;   // eV
    double num[RT_MAX_GROUPS], tot = 0.0;
    for (int i = 0; i < G; i++) {
        const double u0 = std::log(edges[i]), u1 = std::log(edges[i + 1]);
        const double hp = (u1 - u0) / NP;
        double I0 = 0.0, Is = 0.0, IE = 0.0, IsE = 0.0;
        for (int p = 0; p < NP; p++) {
            const double mid = u0 + (p + 0.5) * hp;
            for (int q = 0; q < NQ; q++) {
                const double E = std::exp(mid + 0.5 * hp * xq[q]);
                // photons per unit u: E^2/(exp(E/kT) - 1) * dE/du, dE/du = E
                const double n = wq[q] * E * E * E / std::expm1(E / kT);
                const double s = sigma_hydrogenic(E);
                I0 += n;
                Is += s * n;
                IE += E * n;
                IsE += s * E * n;
            }
        }
        sigN[i] = Is / I0;
        Eavg[i] = IE / I0 * EV;
        sigE[i] = IsE / IE;
        num[i] = I0 * (0.5 * hp);   // photons of the group (panel half-width)
        tot += num[i];
    }
    for (int i = 0; i < G; i++) frac[i] = num[i] / tot;
    return RT_OK;
}
