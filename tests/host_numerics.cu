// Host-side checks of the chemistry kernel's numerical helpers, compiled by
// tests/test_host_numerics.py with nvcc and run on the CPU:
//   1. f2d (float -> double by integer operations, the conversion
//      instruction for subnormals, Inf and NaN) against the conversion
//      instruction, for every float;
//   2. d2f (double -> float, round to nearest even) against the conversion,
//      on exponents around the float range with exact ties, near-ties and
//      carries into the exponent, in the normal and the subnormal results;
//   3. exp_tab (the fast forms' exp, Tang's table-driven method) against expl
//      on 2e6 arguments, in ulps of the result, and its 2^(j/64) table;
//   4. the rate table (rate_table.cu) evaluated the kernel's way (interval
//      and local variable from T's bits, the polynomial's tail in FP32)
//      against the rate fits in long double at random temperatures.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_1508_07888_b300/csrc/launch.h"
#include "../paper_1508_07888_b300/csrc/rt_kernels.cuh"

typedef long double LD;
static const LD THI = 157807.0L;
// the fits, written out again from their published forms (Hui & Gnedin 1997
// case A/B recombination and collisional ionisation; excitation cooling and
// bremsstrahlung as documented in rate_table.cu)
static LD aA(LD T) { LD l = 2 * THI / T; return 1.269e-13L * powl(l, 1.503L) / powl(1 + powl(l / 0.522L, 0.470L), 1.923L); }
static LD aB(LD T) { LD l = 2 * THI / T; return 2.753e-14L * powl(l, 1.500L) / powl(1 + powl(l / 2.740L, 0.407L), 2.242L); }
static LD kR(LD T) { LD l = 2 * THI / T; return 1.778e-29L * T * powl(l, 1.965L) / powl(1 + powl(l / 0.541L, 0.502L), 2.697L) + 1.42e-27L * 1.3L * sqrtl(T); }
static LD beta(LD T) { LD l = 2 * THI / T; return 21.11L * powl(T, -1.5L) * expl(-l / 2) * powl(l, -1.089L) / powl(1 + powl(l / 0.354L, 0.874L), 1.101L); }
static LD cce(LD T) { return 7.5e-19L * expl(-118348.0L / T) / (1 + sqrtl(T / 1e5L)); }

int main()
{
    int fails = 0;
    unsigned long long bad = 0;
    for (unsigned long long u = 0; u <= 0xffffffffull; u++) {
        const float f = rtk::ffrom((unsigned)u);
        const double a = rtk::f2d(f), b = (double)f;
        if (f != f) { if (a == a) bad++; continue; }
        if (rtk::dbits(a) != rtk::dbits(b)) bad++;
    }
    printf("f2d: %llu mismatches over all floats\n", bad);
    fails += bad != 0;

    std::mt19937_64 g(7);
    unsigned long long bad2 = 0, n = 0;
    auto chk = [&](double d) {
        n++;
        const float a = rtk::d2f(d), b = (float)d;
        if (d != d) { if (a == a) bad2++; return; }
        if (rtk::fbits(a) != rtk::fbits(b)) bad2++;
    };
    for (int k = 0; k < 20000000; k++) {
        const unsigned long long r = g();
        const unsigned long long ex = 860 + (r % 330);
        unsigned long long m = g() & 0xfffffffffffffull;
        switch (k % 5) {
        case 1: m = (m & ~0x1fffffffull) | 0x10000000ull; break;
        case 2: m = (m & ~0x1fffffffull) | 0x0fffffffull; break;
        case 3: m = (m & ~0x1fffffffull) | 0x10000001ull; break;
        case 4: m = 0xfffffffffffffull - (g() & 0x3fffffffull); break;
        }
        chk(rtk::dfrom(((r >> 63) << 63) | (ex << 52) | m));
    }
    // ties, near-ties and carries at the rounding position of subnormal
    // results (exponents 873..896: the dropped bits are the low 926 - ex
    // bits of the 53-bit significand)
    for (unsigned long long ex = 870; ex <= 897; ex++) {
        const unsigned sft = ex <= 896 ? 926u - (unsigned)ex : 29u;
        for (int k = 0; k < 4000; k++) {
            const unsigned long long full = (g() & 0xfffffffffffffull) | (1ull << 52);
            const unsigned long long keep = sft < 53 ? full & ~((1ull << sft) - 1ull) : 0ull;
            const unsigned long long half = sft <= 53 ? 1ull << (sft - 1u) : 0ull;
            for (unsigned long long low : {half, half - 1ull, half + 1ull, 0ull, (half << 1) - 1ull}) {
                const unsigned long long m = ((keep | (sft <= 53 ? low : 0ull)) & 0xfffffffffffffull);
                chk(rtk::dfrom(((unsigned long long)(k & 1) << 63) | (ex << 52) | m));
            }
        }
    }
    for (unsigned long long ex = 0; ex < 2048; ex++)
        for (int s = 0; s < 2; s++)
            for (unsigned long long m : {0ull, 1ull, 0x10000000ull, 0xfffffffffffffull, 0x8000000000000ull})
                chk(rtk::dfrom(((unsigned long long)s << 63) | (ex << 52) | m));
    printf("d2f: %llu mismatches over %llu doubles\n", bad2, n);
    fails += bad2 != 0;

    {   // the fast forms' exp (Tang's table-driven method) against expl, in ulps of the result
        double2 e2[64];
        rtl::build_exp2_table(e2);
        // 2^(1/64), 2^(32/64), 2^(63/64) as hi + lo (60-digit decimal arithmetic); the
        // table is built in long double, so its lo parts agree to about 2^-64
        const double ref[3][2] = {{0x1.02c9a3e778061p+0, -0x1.19083535b085dp-56},
                                  {0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54},
                                  {0x1.fa7c1819e90d8p+0, 0x1.74853f3a5931ep-55}};
        const int rj[3] = {1, 32, 63};
        bool tab_ok = e2[0].x == 1.0 && e2[0].y == 0.0;
        for (int i = 0; i < 3; i++)
            tab_ok = tab_ok && e2[rj[i]].x == ref[i][0] && std::fabs(e2[rj[i]].y - ref[i][1]) <= std::ldexp(1.0, -62);
        std::uniform_real_distribution<double> ux(-600.0, 60.0);
        double worst = 0;
        for (int k = 0; k < 2000000; k++) {
            const double x = k < 1000 ? -511.99 + k * 0.5 : ux(g);
            const double a = rtk::exp_tab(x, e2);
            const LD ex = expl((LD)x);
            const double ulp = std::ldexp(1.0, std::ilogb((double)ex) - 52);
            worst = std::fmax(worst, (double)(fabsl((LD)a - ex) / (LD)ulp));
        }
        printf("exp_tab: max error %.3f ulp over 2e6 arguments in [-600, 60]; table %s\n", worst,
               tab_ok ? "ok" : "WRONG");
        fails += !(worst <= 1.0 && tab_ok);
    }

    for (int ots = 0; ots < 2; ots++) {
        std::vector<rtd::RateCoef> tab(rtl::rate_table_entries());
        if (!rtl::build_rate_table(ots != 0, tab.data())) { printf("table build failed\n"); return 1; }
        if (ots) continue;                      // the OTS table differs in kR only
        std::uniform_real_distribution<double> lu(0.0, 30.0 * 0.6931471805599453);
        double w[5] = {0, 0, 0, 0, 0}, w32 = 0;
        long long kr_over = 0;                  // kR above its interval's FP32 bound (entry 3's b32)
        for (int k = 0; k < 300000; k++) {
            const double T = std::exp(lu(g));
            const unsigned long long bits = rtk::dbits(T);
            const int e = (int)(bits >> 52) - 1023;
            if (e < RTD_TAB_E0 || e >= RTD_TAB_E1) continue;
            const int low = 52 - RTD_TAB_SUB;
            const int j = ((e - RTD_TAB_E0) << RTD_TAB_SUB) + (int)((bits >> low) & ((1 << RTD_TAB_SUB) - 1));
            // the kernel's local variable: t = 2 y - 3, and t32 from y's top 23 mantissa bits
            const unsigned long long ym = (bits & ((1ull << low) - 1)) << RTD_TAB_SUB;
            const double t = std::fma(2.0, rtk::dfrom(0x3FF0000000000000ull | ym), -3.0);
            const unsigned int y32 = 0x3F800000u | (unsigned int)(ym >> 29);
            float y32f;
            std::memcpy(&y32f, &y32, 4);
            const float t32 = std::fmaf(2.0f, y32f, -3.0f);
            const rtd::RateCoef *a = tab.data() + (size_t)j * RTD_TAB_NF;
            double gv[RTD_TAB_NF];
            for (int f = 0; f < RTD_TAB_NF; f++) {
                const rtd::RateCoef &c = a[f];
                const float q = std::fmaf(std::fmaf(c.c5, t32, c.c4), t32, c.c3);
                gv[f] = std::fma(std::fma(std::fma((double)q, t, c.c2), t, c.c1), t, c.c0);
            }
            const LD ex3[3] = {aA(T), aB(T), kR(T)};
            {   // the split form's FP32 alpha_B: the b32 fields with entry 1's FP32 tail
                const float q = std::fmaf(std::fmaf(a[1].c5, t32, a[1].c4), t32, a[1].c3);
                const float v = std::fmaf(std::fmaf(std::fmaf(q, t32, a[2].b32), t32, a[1].b32), t32, a[0].b32);
                w32 = std::fmax(w32, (double)fabsl(((LD)v - ex3[1]) / ex3[1]));
            }
            for (int f = 0; f < 3; f++) w[f] = std::fmax(w[f], (double)fabsl((gv[f] - ex3[f]) / ex3[f]));
            if (!(gv[2] <= (double)a[3].b32) || !((LD)a[3].b32 <= ex3[2] * 1.03L)) kr_over++;
            const double b = T >= RTD_TAB_TCUT ? std::exp(gv[3] - 157807.0 / T) : 0.0;
            const double c = T >= RTD_TAB_TCUT ? std::exp(gv[4] - 118348.0 / T) : 0.0;
            const LD eb = beta(T), ec = cce(T);
            // below the cut the fits are zero in double; above it, relative
            if (T < RTD_TAB_TCUT) {
                if ((double)eb != 0.0 || (double)ec != 0.0) w[3] = w[4] = 1.0;
            } else {
                if (eb > 1e-290L) w[3] = std::fmax(w[3], (double)fabsl((b - eb) / eb));
                if (ec > 1e-290L) w[4] = std::fmax(w[4], (double)fabsl((c - ec) / ec));
            }
        }
        printf("table: max rel err aA %.2e aB %.2e kR %.2e beta %.2e cce %.2e; FP32 aB %.2e; kR bound misses %lld\n",
               w[0], w[1], w[2], w[3], w[4], w32, kr_over);
        fails += kr_over != 0;
        // alpha, kR: interpolation error and the FP32 tail's rounding (the
        // table's own bound, 2e-13); beta, cce: exp of arguments up to ~800
        // in magnitude, whose own rounding (~1e-13 relative) dominates
        fails += !(w[0] < 2e-13 && w[1] < 2e-13 && w[2] < 2e-13 && w[3] < 1e-12 && w[4] < 1e-12 && w32 < 1e-6);
    }
    printf(fails ? "FAIL\n" : "OK\n");
    return fails ? 1 : 0;
}
