// rate_table.cu -- host-side construction of the temperature-rate tables
// used by the chemistry kernel.
//
// The rate fits (Hui & Gnedin 1997 recombination, collisional ionisation and
// recombination cooling; exp(-118348/T)/(1 + sqrt(T/1e5)) excitation cooling;
// 1.42e-27 x 1.3 sqrt(T) bremsstrahlung) are evaluated here in long double and
// interpolated on 2^RTD_TAB_SUB equal intervals of T per binade, 1 K <= T <
// 2^30 K, each by a degree-5 Chebyshev polynomial in the local variable
// t = 2 (T - T_a)/(T_b - T_a) - 1 in [-1, 1), stored as monomial coefficients
// in t: c0 .. c2 in double, c3 .. c5 in float (the kernel evaluates the
// tail c3 + t (c4 + t c5) in FP32; on these narrow intervals it is below
// ~1e-6 of the value, so its FP32 rounding stays near 1e-13 of it).
// Tabulated functions (layout [interval][function][coefficient]):
//   0: alpha_A   1: alpha_B   2: recombination (case A or B) + free-free cooling
//   3: ln(beta) + T_HI/T               (beta = exp(f3 - T_HI/T))
//   4: ln(excitation cooling) + 118348/T
// The two exp(-c/T) factors stay outside the tables so every tabulated
// function is smooth in T.  The table is checked against the long-double
// fits before use; the kernel evaluates the fits directly when it is absent.
#include <cmath>

#include "launch.h"
#include "rt_device.h"

namespace {

typedef long double LD;
const LD THI = 157807.0L;

LD fit_aA(LD T)
{
    const LD l = 2 * THI / T;
    return 1.269e-13L * powl(l, 1.503L) / powl(1 + powl(l / 0.522L, 0.470L), 1.923L);
}
LD fit_aB(LD T)
{
    const LD l = 2 * THI / T;
    return 2.753e-14L * powl(l, 1.500L) / powl(1 + powl(l / 2.740L, 0.407L), 2.242L);
}
LD fit_kR(LD T, bool ots)
{
    const LD l = 2 * THI / T;
    const LD rec = ots ? 3.435e-30L * T * powl(l, 1.970L) / powl(1 + powl(l / 2.250L, 0.376L), 3.720L)
                       : 1.778e-29L * T * powl(l, 1.965L) / powl(1 + powl(l / 0.541L, 0.502L), 2.697L);
    return rec + 1.42e-27L * 1.3L * sqrtl(T);
}
LD fit_lnbeta_plus(LD T)   // ln(beta) + T_HI/T  (T_HI/T = lambda/2)
{
    const LD l = 2 * THI / T;
    return logl(21.11L) - 1.5L * logl(T) - 1.089L * logl(l) - 1.101L * log1pl(powl(l / 0.354L, 0.874L));
}
LD fit_lncce_plus(LD T)    // ln(excitation cooling) + 118348/T
{
    return logl(7.5e-19L) - log1pl(sqrtl(T / 1.0e5L));
}

LD fit(int f, LD T, bool ots)
{
    switch (f) {
    case 0: return fit_aA(T);
    case 1: return fit_aB(T);
    case 2: return fit_kR(T, ots);
    case 3: return fit_lnbeta_plus(T);
    default: return fit_lncce_plus(T);
    }
}

}  // namespace

namespace rtl {

// 2^(j/64) in long double (64-bit significand), split into the double hi
// nearest to it and the double lo nearest to the rest: hi + lo agrees with
// 2^(j/64) to about 2^-64 relative
void build_exp2_table(double2 *out)
{
    for (int j = 0; j < 64; j++) {
        const LD v = exp2l((LD)j / 64.0L);
        const double hi = (double)v;
        out[j] = make_double2(hi, (double)(v - (LD)hi));
    }
}

static_assert(RTD_TAB_NC == 6, "the coefficient layout holds degree 5: c0 .. c2 double, c3 .. c5 float");

// the kernel's evaluation of one polynomial at t (t32: t in float)
static double eval_coef(const rtd::RateCoef &c, double t, float t32)
{
    const float q = std::fmaf(std::fmaf(c.c5, t32, c.c4), t32, c.c3);
    return std::fma(std::fma(std::fma((double)q, t, c.c2), t, c.c1), t, c.c0);
}

// the kernel's FP32 evaluation of alpha_B from an interval's entries a[0..2]
static float eval_aB32(const rtd::RateCoef *a, float t32)
{
    const float q = std::fmaf(std::fmaf(a[1].c5, t32, a[1].c4), t32, a[1].c3);
    return std::fmaf(std::fmaf(std::fmaf(q, t32, a[2].b32), t32, a[1].b32), t32, a[0].b32);
}

// fills out[RTD_TAB_NINT][RTD_TAB_NF]; returns true when the table, evaluated
// the kernel's way, reproduces the long-double fits to 2e-13 (relative for
// functions 0-2, absolute for the logarithms 3-4) at 17 points per interval
// (the FP32 tail's rounding reaches 1.1e-13 on one interval, alpha_A near
// 7e7 K; elsewhere the error is ~3e-14),
// when alpha_B's FP32 copy (the b32 fields with entry 1's FP32 tail)
// reproduces it to 1e-6 relative at the same points (FP32 Horner of a degree-5
// polynomial in |t| <= 1: a few ulp of float), when both exp(-c/T) factors
// are exactly zero in double below RTD_TAB_TCUT, and when the terms they make
// are below 2^-60 of what they enter below RTD_TAB_TWARM at n0 dtau <=
// RTD_TAB_NDMAX.  Entry 3's b32 holds an upper bound of kR over the
// interval in FP32 (the largest fit value at 257 points, 1e-3 above it,
// rounded up), checked against the kernel's evaluation at the check points.
bool build_rate_table(bool ots, rtd::RateCoef *out)
{
    const int N = RTD_TAB_NC;
    // monomial coefficients of the Chebyshev polynomials T_0 .. T_{N-1}
    LD cheb[RTD_TAB_NC][RTD_TAB_NC] = {};
    cheb[0][0] = 1;
    cheb[1][1] = 1;
    for (int n = 2; n < N; n++)
        for (int i = 0; i < N; i++)
            cheb[n][i] = (i > 0 ? 2 * cheb[n - 1][i - 1] : 0) - cheb[n - 2][i];
    const int per = 1 << RTD_TAB_SUB;
    for (int j = 0; j < RTD_TAB_NINT; j++) {
        const LD lo = ldexpl(1.0L + (LD)(j % per) / per, RTD_TAB_E0 + j / per);
        const LD hi = ldexpl(1.0L + (LD)(j % per + 1) / per, RTD_TAB_E0 + j / per);
        LD aBm[3] = {0, 0, 0};                        // alpha_B's c0 .. c2
        for (int f = 0; f < RTD_TAB_NF; f++) {
            LD fv[RTD_TAB_NC], c[RTD_TAB_NC];
            for (int m = 0; m < N; m++) {
                const LD t = cosl(M_PIl * (m + 0.5L) / N);
                fv[m] = fit(f, lo + (t + 1) * 0.5L * (hi - lo), ots);
            }
            for (int n = 0; n < N; n++) {
                LD s = 0;
                for (int m = 0; m < N; m++) s += fv[m] * cosl(M_PIl * n * (m + 0.5L) / N);
                c[n] = (n == 0 ? 1.0L : 2.0L) * s / N;
            }
            // monomial coefficients in t
            LD mt[RTD_TAB_NC];
            for (int i = 0; i < N; i++) {
                LD s = 0;
                for (int n = 0; n < N; n++) s += c[n] * cheb[n][i];
                mt[i] = s;
            }
            rtd::RateCoef &o = out[(size_t)j * RTD_TAB_NF + f];
            o.c0 = (double)mt[0];
            o.c1 = (double)mt[1];
            o.c2 = (double)mt[2];
            o.c3 = (float)mt[3];
            o.c4 = (float)mt[4];
            o.c5 = (float)mt[5];
            o.b32 = 0.0f;
            if (f == 1)
                for (int i = 0; i < 3; i++) aBm[i] = mt[i];
            for (int k = 0; k <= 16; k++) {           // check, the kernel's way
                const double t = -1.0 + k / 8.0;
                const LD ex = fit(f, lo + ((LD)t + 1) * 0.5L * (hi - lo), ots);
                const double p = eval_coef(o, t, (float)t);
                const LD err = f <= 2 ? fabsl((p - ex) / ex) : fabsl(p - ex);
                if (!(err <= 2e-13L)) return false;
            }
        }
        rtd::RateCoef *a = out + (size_t)j * RTD_TAB_NF;
        for (int i = 0; i < 3; i++) a[i].b32 = (float)aBm[i];
        LD kmax = 0;
        for (int k = 0; k <= 256; k++) {
            const LD v = fit(2, lo + (hi - lo) * k / 256.0L, ots);
            kmax = v > kmax ? v : kmax;
        }
        kmax *= 1.001L;
        float kb = (float)kmax;
        if ((LD)kb < kmax) kb = std::nextafterf(kb, INFINITY);
        a[3].b32 = kb;
        for (int k = 0; k <= 16; k++)
            if (!(eval_coef(a[2], -1.0 + k / 8.0, (float)(-1.0 + k / 8.0)) <= (double)kb)) return false;
        for (int k = 0; k <= 16; k++) {
            const double t = -1.0 + k / 8.0;
            const LD ex = fit(1, lo + ((LD)t + 1) * 0.5L * (hi - lo), ots);
            if (!(fabsl(((LD)eval_aB32(a, (float)t) - ex) / ex) <= 1e-6L)) return false;
        }
    }
    // the factors the kernel skips below RTD_TAB_TCUT (both grow with T)
    const double tc = RTD_TAB_TCUT;
    if (std::exp((double)fit_lnbeta_plus(tc) - (double)THI / tc) != 0.0) return false;
    if (std::exp((double)fit_lncce_plus(tc) - 118348.0 / tc) != 0.0) return false;
    // below RTD_TAB_TWARM with n0 dtau <= RTD_TAB_NDMAX: beta n0 dtau (against
    // 1 in the x_HI denominator) and kC n0 dtau / (1.5 kB T) (the cooling
    // against the internal energy, x_HI, 1 - x_HI <= 1) below 2^-60; both
    // grow with T on [TCUT, TWARM], checked on a fine grid
    const LD kB = 1.380649e-16L, lim = ldexpl(1.0L, -60);
    LD prev_b = 0, prev_c = 0;
    for (int k = 0; k <= 4096; k++) {
        const LD T = RTD_TAB_TCUT + (RTD_TAB_TWARM - RTD_TAB_TCUT) * k / 4096.0L;
        const LD b = expl(fit_lnbeta_plus(T) - THI / T);
        const LD kc = kB * THI * b + expl(fit_lncce_plus(T) - 118348.0L / T);
        if (b < prev_b || kc < prev_c) return false;
        prev_b = b;
        prev_c = kc;
    }
    const LD Tw = RTD_TAB_TWARM;
    const LD bw = expl(fit_lnbeta_plus(Tw) - THI / Tw);
    const LD cw = (kB * THI * bw + expl(fit_lncce_plus(Tw) - 118348.0L / Tw)) / (1.5L * kB * Tw);
    if (!((LD)RTD_TAB_NDMAX * bw <= lim && (LD)RTD_TAB_NDMAX * cw <= lim)) return false;
    return true;
}

}  // namespace rtl
