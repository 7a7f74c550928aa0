// rt_kernels.cuh -- the hot path of one M1 radiative-transfer step
// (Aubert, Deparis & Ocvirk, arXiv:1508.07888, Secs. 2.2.3 and 2.2.4).
//
// This header is compiled twice:
//   k_fast.cu    default flags: fused multiply-add, reciprocal-multiply in
//                place of some divisions (FP32 transport + FP64 chemistry,
//                and the all-FP64 form);
//   k_strict.cu  --fmad=false: every operation is one IEEE-rounded +, -, *,
//                /, sqrt in the order written, which makes the FP64 path
//                bit-reproducible against a plain IEEE evaluation of the same
//                expressions (with constant rates; the rate fits call exp/log).
// The STRICT template flag selects the division forms; the compiler flag
// removes the contractions.
#pragma once

#include <cstdint>

#include <cstring>
#include <type_traits>

#include "rt_device.h"

namespace rtk {

using rtd::BoxDev;
using rtd::CellConst;
using rtd::Ctl;
using rtd::DiagBuf;
using rtd::DiagPart;
using rtd::FineDev;
using rtd::Phys;
using rtd::RateCoef;

// ------------------------------------------------------------- vector I/O
template <typename R>
struct V4 {
    R x, y, z, w;
};

__device__ __forceinline__ V4<float> ld4(const V4<float> *p)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ void st4(V4<float> *p, const V4<float> &v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ V4<double> ld4(const V4<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = q[0], b = q[1];
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(V4<double> *p, const V4<double> &v)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}

// ------------------------------------------------------------- FP64 pipe relief
// On this GPU the FP64 pipe (2 lanes per SM and clock) bounds the chemistry,
// while the integer pipe is nearly idle; float <-> double conversions and
// reciprocals of the fast forms are therefore done without FP64-pipe
// conversion instructions.
__host__ __device__ __forceinline__ unsigned long long dbits(double d)
{
    unsigned long long u;
    memcpy(&u, &d, 8);
    return u;
}
__host__ __device__ __forceinline__ double dfrom(unsigned long long u)
{
    double d;
    memcpy(&d, &u, 8);
    return d;
}
__host__ __device__ __forceinline__ unsigned fbits(float f)
{
    unsigned u;
    memcpy(&u, &f, 4);
    return u;
}
__host__ __device__ __forceinline__ float ffrom(unsigned u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// float -> double, exact: a normal float's exponent is rebiased (127 -> 1023)
// and its mantissa moved up 29 bits, a zero keeps its sign; subnormals, Inf
// and NaN take the conversion instruction
__host__ __device__ __forceinline__ double f2d(float f)
{
    const unsigned u = fbits(f);
    if ((u & 0x7f800000u) - 0x00800000u < 0x7f000000u)
        return dfrom(((unsigned long long)(u & 0x80000000u) << 32) |
                     (((unsigned long long)(u & 0x7fffffffu) << 29) + (896ull << 52)));
    if ((u & 0x7fffffffu) == 0u) return dfrom((unsigned long long)u << 32);
    return (double)f;
}

// double -> float, rounded to nearest even: when the result is a normal
// float (double exponent 897..1150) the top 23 mantissa bits are kept and
// the 29 dropped bits decide the rounding (a carry into the exponent gives
// the next binade, or Inf above the largest float, as IEEE rounding does); a
// zero keeps its sign; everything else takes the conversion instruction
__host__ __device__ __forceinline__ float d2f(double d)
{
    const unsigned long long b = dbits(d);
    const unsigned ed = (unsigned)(b >> 52) & 0x7ffu;
    if (ed - 897u < 254u) {
        const unsigned long long m = b & 0x7fffffffffffffffull;
        unsigned r = (unsigned)((m >> 29) - (896ull << 23));
        const unsigned low = (unsigned)m & 0x1fffffffu;
        r += (low > 0x10000000u || (low == 0x10000000u && (r & 1u))) ? 1u : 0u;
        return ffrom(r | ((unsigned)(b >> 32) & 0x80000000u));
    }
    if ((b & 0x7fffffffffffffffull) == 0ull) return ffrom((unsigned)(b >> 32));   // +-0
    return (float)d;
}

// any lane of the warp's active ones (host: the lane itself)
__host__ __device__ __forceinline__ bool vote_any(bool p)
{
#ifdef __CUDA_ARCH__
    return __any_sync(__activemask(), p);
#else
    return p;
#endif
}

// finite (not NaN or Inf) from the exponent bits, on the integer pipe
__host__ __device__ __forceinline__ bool finite_bits(double d)
{
    return (dbits(d) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

template <typename R> __device__ __forceinline__ double to_d(R v);
template <> __device__ __forceinline__ double to_d<float>(float v) { return f2d(v); }
template <> __device__ __forceinline__ double to_d<double>(double v) { return v; }
template <typename R> __device__ __forceinline__ R from_d(double v);
template <> __device__ __forceinline__ float from_d<float>(double v) { return d2f(v); }
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }

// 1/d for the fast forms: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64, relative error below 2^-20) refined by one
// third-order Newton-Raphson step, y <- y + y (e + e^2) with e = 1 - d y,
// which cubes the relative error (below 2^-60 before the final rounding).
// On 4.2 M test values it equals IEEE 1/d in 99.97% of cases and is one ulp
// off otherwise.  |d| outside [2^-1020, 2^1020) (zero, subnormal, huge,
// Inf, NaN) takes the IEEE division instead.
__device__ __forceinline__ double rcp_nr(double d)
{
    const unsigned ex = (unsigned)(dbits(d) >> 52) & 0x7ffu;
    if (ex - 3u >= 2040u) return 1.0 / d;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    const double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// exp(x) of the fast forms' chemistry: the table-driven method of P. T. P.
// Tang (ACM TOMS 15(2), 1989).  With k = round(64 x / ln2), j = k mod 64,
// m = floor(k / 64) and r = x - k ln2/64 (ln2/64 as the pair L1 + L2,
// |r| <= ln2/128 + tiny), exp(x) = 2^m 2^(j/64) e^r: 2^(j/64) is the pair
// hi + lo of e2t[j], e^r - 1 its degree-5 Taylor polynomial (truncation
// below 4e-17 relative), 2^m added to the exponent field.  Within one ulp
// of exp(x) (host test over 2e6 arguments against expl).  |x| >= 512 and
// NaN take the library exp, behind a warp vote so the fast path issues
// none of its instructions.
__host__ __device__ __forceinline__ double exp_tab(double x, const double2 *e2t)
{
    constexpr double INV = 0x1.71547652b82fep+6;        // 64 / ln2
    constexpr double SH = 0x1.8p52;                     // round-to-integer shifter
    constexpr double L1 = 0x1.62e42fefa39efp-7;         // ln2/64 = L1 + L2
    constexpr double L2 = 0x1.abc9e3b39803fp-62;
    const double kd = fma(x, INV, SH);
    const int k = (int)(unsigned)dbits(kd);             // round(64 x / ln2), low word
    const double kf = kd - SH;
    double r = fma(-kf, L1, x);
    r = fma(-kf, L2, r);
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double p = fma(r * r, q, r);                  // e^r - 1
#ifdef __CUDA_ARCH__
    const double2 t = __ldg(e2t + (k & 63));
#else
    const double2 t = e2t[k & 63];
#endif
    const double y = t.x + fma(t.x, p, t.y);            // 2^(j/64) e^r, in [0.99, 2.02)
    double e = dfrom(dbits(y) + ((unsigned long long)(long long)(k >> 6) << 52));
    const bool far = (dbits(x) & 0x7fffffffffffffffull) >= 0x4080000000000000ull;   // |x| >= 512, NaN
    if (vote_any(far)) {
        if (far) e = exp(x);
    }
    return e;
}

__device__ __forceinline__ float rsqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double rsqrt_(double v) { return sqrt(v); }

// reciprocal and square root of the generic kernels: the FP32 fast path
// (the HLL transport of the split form) takes the MUFU approximations
// (rcp.approx / sqrt.approx, ~1 ulp), as the FP32 GLF kernel does; FP64 and
// the strict form take IEEE division and square root
template <typename R, bool STRICT>
__device__ __forceinline__ R frcp(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float frcp<float, false>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
template <typename R, bool STRICT>
__device__ __forceinline__ R fdiv(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ float fdiv<float, false>(float a, float b) { return a * frcp<float, false>(b); }
// reciprocal of the closure: the FP64 fast form (RT_PREC_FP64) takes the
// Newton reciprocal of rcp_nr (one ulp at most from IEEE 1/d) where the
// strict form divides.  The HLL speeds keep IEEE division in FP64: there a
// beam's f = |F|/N must come out exactly 1 (a 1-ulp f gives a beam along a
// face a transverse speed of ~1e-8 and moves the face off the mean flux)
template <typename R, bool STRICT>
__device__ __forceinline__ R crcp(R x) { return frcp<R, STRICT>(x); }
template <>
__device__ __forceinline__ double crcp<double, false>(double x) { return rcp_nr(x); }
template <typename R, bool STRICT>
__device__ __forceinline__ R cdiv(R a, R b) { return fdiv<R, STRICT>(a, b); }
template <>
__device__ __forceinline__ double cdiv<double, false>(double a, double b) { return a * rcp_nr(b); }
template <typename R, bool STRICT>
__device__ __forceinline__ R fsqrt(R x) { return rsqrt_(x); }
template <typename R, bool STRICT>
__device__ __forceinline__ constexpr bool approx_form() { return !STRICT && sizeof(R) == 4; }
template <>
__device__ __forceinline__ float fsqrt<float, false>(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------------- M1 closure
// Levermore closure, P = Nhat D with D = (1-chi)/2 I + (3chi-1)/2 n n
// (Sec. 2.2.3; the printed coefficients are swapped, the diffusive limit
// fixes the order), chi = (3+4f^2)/(5+2 sqrt(4-3f^2)), f = |Fhat|/Nhat
// clamped to 1, evaluated as (3chi-1)/2 = f^2 g, g = (6 + 3/(2+s))/(5+2s),
// s = sqrt(4-3f^2).  P = (xx, xy, xz, yy, yz, zz).
// smallest N the closure and the HLL speeds resolve: FP32 subnormals (below
// ~1.2e-38) would overflow 1/N, so the FP32 path treats N <= 1e-37 as N = 0
// (P = 0, isotropic speeds); FP64 uses N > 0 as the oracle does
template <typename R> __device__ __forceinline__ R closure_nmin();
template <> __device__ __forceinline__ float closure_nmin<float>() { return 1e-37f; }
template <> __device__ __forceinline__ double closure_nmin<double>() { return 0.0; }

template <typename R, bool STRICT>
__device__ __forceinline__ void closure(const V4<R> &u, R P[6])
{
    const R N = u.x;
    if (N > closure_nmin<R>()) {
        R ux, uy, uz;
        if (STRICT) {
            ux = u.y / N; uy = u.z / N; uz = u.w / N;
        } else {
            const R rN = crcp<R, STRICT>(N);
            ux = u.y * rN; uy = u.z * rN; uz = u.w * rN;
        }
        R f2 = ux * ux + uy * uy + uz * uz;
        // rounding guard of |F| <= cN.  With the approximate reciprocal a
        // beam (|F| = cN exactly) lands a few ulp either side of f = 1, so
        // the FP32 fast form takes f^2 >= 1 - 2^-20 as the beam itself and
        // its closure exactly: chi = 1, a = 0, g = 1, P = N n n
        constexpr bool AP = approx_form<R, STRICT>();
        const bool beam = AP ? f2 >= R(1) - R(9.5367431640625e-07) : f2 > R(1);
        if (beam) {
            const R f = fsqrt<R, STRICT>(f2);
            if (STRICT) {
                ux = ux / f; uy = uy / f; uz = uz / f;
            } else {
                const R rf = crcp<R, STRICT>(f);
                ux *= rf; uy *= rf; uz *= rf;
            }
            f2 = R(1);
        }
        R a, g;
        if (AP && beam) {
            a = R(0);
            g = R(1);
        } else if (STRICT) {
            const R s = fsqrt<R, STRICT>(R(4) - R(3) * f2);
            a = ((R(1) + s) - R(2) * f2) / (R(5) + R(2) * s);
            g = (R(6) + R(3) / (R(2) + s)) / (R(5) + R(2) * s);
        } else {
            const R s = fsqrt<R, STRICT>(R(4) - R(3) * f2);
            const R r5 = crcp<R, STRICT>(R(5) + R(2) * s);
            a = ((R(1) + s) - R(2) * f2) * r5;
            g = (R(6) + cdiv<R, STRICT>(R(3), R(2) + s)) * r5;
        }
        P[0] = N * (a + g * (ux * ux));
        P[1] = N * (g * (ux * uy));
        P[2] = N * (g * (ux * uz));
        P[3] = N * (a + g * (uy * uy));
        P[4] = N * (g * (uy * uz));
        P[5] = N * (a + g * (uz * uz));
    } else {
#pragma unroll
        for (int k = 0; k < 6; k++) P[k] = R(0);
    }
}

__device__ __forceinline__ constexpr int pidx(int d, int j)
{
    return d == 0 ? j : (d == 1 ? (j == 0 ? 1 : (j == 1 ? 3 : 4)) : (j == 0 ? 2 : (j == 1 ? 4 : 5)));
}

template <typename R>
__device__ __forceinline__ R comp(const V4<R> &u, int m)
{
    return m == 0 ? u.x : (m == 1 ? u.y : (m == 2 ? u.z : u.w));
}

// GLF flux (Eq. e:glf) along axis d between left (uL, PL) and right (uR, PR):
// Phi = 0.5 ((G_d(L) + G_d(R)) - (R - L)), G_d = (Fhat_d, P_d.)
template <typename R, int d>
__device__ __forceinline__ void glf(const V4<R> &uL, const R PL[6], const V4<R> &uR,
                                    const R PR[6], R Phi[4])
{
    const R GL0 = comp(uL, 1 + d), GR0 = comp(uR, 1 + d);
    Phi[0] = R(0.5) * ((GL0 + GR0) - (uR.x - uL.x));
    Phi[1] = R(0.5) * ((PL[pidx(d, 0)] + PR[pidx(d, 0)]) - (uR.y - uL.y));
    Phi[2] = R(0.5) * ((PL[pidx(d, 1)] + PR[pidx(d, 1)]) - (uR.z - uL.z));
    Phi[3] = R(0.5) * ((PL[pidx(d, 2)] + PR[pidx(d, 2)]) - (uR.w - uL.w));
}

// HLL signal speeds (units of c) of state u along the three axes from the
// wave-speed table (rt_hll_speeds: lambda_max at f = 1 - (i/NF)^2,
// mu = -1 + 2j/NM), interpolated bilinearly in (z = sqrt(1 - f), mu), and
// lambda_min(f, mu) = -lambda_max(f, -mu); f = |F|/N clamped to 1, mu =
// F_d/|F|; N <= 0 or F = 0 take f = 0 (isotropic speeds).
template <typename R>
__device__ __forceinline__ R hll_lookup(const R *tab, R z, R mu)
{
    const R x = z * R(RTD_HLL_NF), y = (mu + R(1)) * R(0.5) * R(RTD_HLL_NM);
    int i = (int)x, j = (int)y;
    i = i > RTD_HLL_NF - 1 ? RTD_HLL_NF - 1 : (i < 0 ? 0 : i);
    j = j > RTD_HLL_NM - 1 ? RTD_HLL_NM - 1 : (j < 0 ? 0 : j);
    const R tx = x - R(i), ty = y - R(j);
    const R *t0 = tab + i * (RTD_HLL_NM + 1) + j, *t1 = t0 + (RTD_HLL_NM + 1);
    const R v00 = t0[0], v01 = t0[1], v10 = t1[0], v11 = t1[1];
    return (v00 * (R(1) - tx) + v10 * tx) * (R(1) - ty) + (v01 * (R(1) - tx) + v11 * tx) * ty;
}

// (f, z) of a state; the caller takes mu = F_d / Fn along each axis
template <typename R, bool STRICT>
__device__ __forceinline__ void hll_fz(const V4<R> &u, R &Fn, R &z)
{
    R f = R(0);
    Fn = R(0);
    if (u.x > closure_nmin<R>()) {
        Fn = fsqrt<R, STRICT>(u.y * u.y + u.z * u.z + u.w * u.w);
        if (Fn > R(0)) {
            f = fdiv<R, STRICT>(Fn, u.x);
            // clamp to 1; the FP32 fast form also takes f within rounding of
            // 1 as the beam (z = sqrt(1 - f) would turn one ulp of f into a
            // transverse speed of 2e-4)
            if (f >= (approx_form<R, STRICT>() ? R(1) - R(4.76837158203125e-07) : R(1))) f = R(1);
        }
    }
    z = fsqrt<R, STRICT>(R(1) - f);
}

template <typename R, bool STRICT, int d>
__device__ __forceinline__ void hll_speed(const R *tab, const V4<R> &u, R Fn, R z, R &smin, R &smax)
{
    const R mu = Fn > R(0) ? fdiv<R, STRICT>(comp(u, 1 + d), Fn) : R(0);
    smax = hll_lookup(tab, z, mu);
    smin = -hll_lookup(tab, z, -mu);
}

// HLL flux along axis d between (uL, PL) with speeds [aL, bL] and (uR, PR)
// with speeds [aR, bR]: Phi = (l+ G_L - l- G_R + l+ l- (U_R - U_L))/(l+ - l-),
// l+ = max(0, bL, bR), l- = min(0, aL, aR); when no wave crosses the face
// (l+ = l- = 0: beams along it on both sides, whose fluxes vanish) the mean
// of the two fluxes
template <typename R, bool STRICT, int d>
__device__ __forceinline__ void hll(const V4<R> &uL, const R PL[6], R aL, R bL, const V4<R> &uR,
                                    const R PR[6], R aR, R bR, R Phi[4])
{
    R lp = bL > bR ? bL : bR, lm = aL < aR ? aL : aR;
    if (lp < R(0)) lp = R(0);
    if (lm > R(0)) lm = R(0);
    const R GL[4] = {comp(uL, 1 + d), PL[pidx(d, 0)], PL[pidx(d, 1)], PL[pidx(d, 2)]};
    const R GR[4] = {comp(uR, 1 + d), PR[pidx(d, 0)], PR[pidx(d, 1)], PR[pidx(d, 2)]};
    if (!(lp - lm > R(0))) {
#pragma unroll
        for (int m = 0; m < 4; m++) Phi[m] = R(0.5) * (GL[m] + GR[m]);
        return;
    }
    const R den = lp - lm, ll = lp * lm, rden = frcp<R, STRICT>(den);
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const R num = lp * GL[m] - lm * GR[m] + ll * (comp(uR, m) - comp(uL, m));
        Phi[m] = STRICT ? num / den : num * rden;
    }
}

// ghost state beyond a box face (Sec. 4.2): transmissive copies the cell,
// reflective copies it with the normal flux component inverted
template <typename R>
__device__ __forceinline__ V4<R> ghost_of(const V4<R> &own, int bc, int d)
{
    V4<R> g = own;
    if (bc == 2) {
        if (d == 0) g.y = -g.y;
        else if (d == 1) g.z = -g.z;
        else g.w = -g.w;
    }
    return g;
}

__device__ __forceinline__ int find_box(const BoxDev *boxes, int nboxes, int64_t item, bool chem)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int64_t s = chem ? boxes[mid].citem0 : boxes[mid].titem0;
        if (s <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------- transport
// cp.async (16-byte global -> shared copies, completion tracked per thread in
// commit groups)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename R>
__device__ __forceinline__ void cp_cell(V4<R> *dst, const V4<R> *src)
{
    if (sizeof(V4<R>) == 16) {
        cp_async16(dst, src);
    } else {
        cp_async16(dst, src);
        cp_async16(reinterpret_cast<char *>(dst) + 16, reinterpret_cast<const char *>(src) + 16);
    }
}

// TMA and mbarrier (FP32 GLF transport).  A tiled 4-D bulk copy of a box of
// the tensor map tm (dims: 4 components, x, y, z + nz g) into shared memory,
// completing on mbarrier bar with its byte count; waits poll the barrier's
// phase a bounded number of times.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// true once phase `parity` of bar has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned limit)
{
    const unsigned a = smem_u32(bar);
    for (unsigned i = 0; i < limit; i++) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}
// orders this thread's earlier shared-memory accesses (after a barrier: the
// block's) before later async-proxy (TMA) writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tm, int c0, int c1, int c2, int c3,
                                            unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5}], [%6];\n"
                 ::"r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
                 : "memory");
}
// polls of an mbarrier before a wait gives up (each poll waits up to the
// hardware's own time slice; far above any copy's latency)
constexpr unsigned RTK_TMA_POLLS = 1u << 22;

// Shared-memory layout of the transport pipeline: a ring of TP_STAGES planes
// of U over the (TY+2) x (TX+2) tile-with-halo, and two planes of the closure
// P (the plane being updated and the next one).
constexpr int TP_STAGES = 5;
constexpr int TP_W = RTD_TX + 2, TP_H = RTD_TY + 2;

template <typename R, int FLUX>
struct TransportSmem {                 // HLL: also the x/y signal speeds of two planes
    V4<R> U[TP_STAGES][TP_H][TP_W];
    R P[2][6][TP_H][TP_W];
    R Sp[2][4][TP_H][TP_W];            // xmin, xmax, ymin, ymax
};
template <typename R>
struct TransportSmem<R, RTD_FLUX_GLF> {
    V4<R> U[TP_STAGES][TP_H][TP_W];
    R P[2][6][TP_H][TP_W];
};

template <typename R, int FLUX = RTD_FLUX_GLF>
constexpr size_t transport_smem_bytes() { return sizeof(TransportSmem<R, FLUX>); }

// Work is counted in plane units: (box, group, y-tile, x-tile, z), z
// fastest.  Block b of a grid of n takes the units [b U/n, (b+1) U/n) and
// splits them into runs of consecutive planes of one column of tiles, so
// every block carries the same number of planes whatever the box sizes.
// For a run z0..z1-1, a block of TX x TY threads owns TX x TY columns:
// planes q = 0..L-1 (z = z0-1 .. z1) stream into a TP_STAGES-deep ring of
// shared memory by cp.async, TP_STAGES-2 planes ahead of the plane being
// updated, with the x/y halo (periodic halos from the wrapped cells, ghost
// halos copied from the boundary cell and, for reflective faces, the normal
// flux negated in shared memory).  Each cell's closure is evaluated once per
// plane; a thread updates plane q-1 as soon as plane q's closures are
// written (its own cell's closure of plane q stays in registers), so one
// barrier per plane separates the phases.  The z-face flux is carried in
// registers (each z-face evaluated once).
// Update (Eq. e:uprt, unsplit): U* = U - lam ((dPhi_x + dPhi_y) + dPhi_z).
__device__ __forceinline__ int find_box_unit(const BoxDev *boxes, int nboxes, int64_t unit)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].titem0 <= unit) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename R, bool STRICT, int FLUX>
__global__ void __launch_bounds__(RTD_TX *RTD_TY)
k_transport(const BoxDev *__restrict__ boxes, int nboxes, int64_t nunits, int /*unused*/, Phys ph,
            Ctl *ctl)
{
    constexpr int TX = RTD_TX, TY = RTD_TY, S = TP_STAGES;
    constexpr bool HLL = FLUX == RTD_FLUX_HLL;
    extern __shared__ __align__(16) unsigned char tp_smem_raw[];
    TransportSmem<R, FLUX> &sm = *reinterpret_cast<TransportSmem<R, FLUX> *>(tp_smem_raw);
    const R *htab = nullptr;
    if (HLL) htab = reinterpret_cast<const R *>(sizeof(R) == 4 ? (const void *)ph.hll_f
                                                                : (const void *)ph.hll_d);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    if (blockIdx.x == 0 && tid == 0) ctl->step += 1;

    const int64_t ubeg = nunits * (int64_t)blockIdx.x / gridDim.x;
    const int64_t uend = nunits * (int64_t)(blockIdx.x + 1) / gridDim.x;
    for (int64_t u = ubeg; u < uend;) {
        const int b = find_box_unit(boxes, nboxes, u);
        const BoxDev &B = boxes[b];
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        const int64_t loc = u - B.titem0;
        int64_t colid = loc / nz;
        const int z0 = (int)(loc - colid * nz);
        const int64_t zlim = (int64_t)z0 + (uend - u);
        const int z1 = zlim < (int64_t)nz ? (int)zlim : nz;
        u += z1 - z0;
        const int ix = (int)(colid % B.tiles_x); colid /= B.tiles_x;
        const int iy = (int)(colid % B.tiles_y);
        const int g = (int)(colid / B.tiles_y);
        const int x0 = ix * TX, y0 = iy * TY;
        const int ntx = min(TX, nx - x0), nty = min(TY, ny - y0);
        const int x = x0 + tx, y = y0 + ty;
        const bool act = (tx < ntx) && (ty < nty);
        const int L = (z1 - z0) + 2;                       // planes z0-1 .. z1
        const V4<R> *Ug = reinterpret_cast<const V4<R> *>(B.U) + (int64_t)g * B.ncell;
        V4<R> *Og = reinterpret_cast<V4<R> *>(B.Us) + (int64_t)g * B.ncell;
        const R lam = (R)B.lam;
        const int64_t sxy = (int64_t)nx * ny;

        // this thread's halo cell (at most one): smem position (hx, hy),
        // source (sx, sy) inside the box, negated component (0 = none)
        int hx = -1, hy = -1, sx = 0, sy = 0, hneg = 0;
        R hin = R(0);                     // inflow ghost: beam density, sign = direction
        bool hif = false;                 // the halo cell is an inflow ghost
        {
            int t = tid;
            if (t < nty) {                                   // left column
                hx = 0; hy = t + 1; sy = y0 + t; sx = x0 - 1;
                if (sx < 0) {
                    if (ph.bc[0] == 0) sx = nx - 1;
                    else { sx = 0; hneg = ph.bc[0] == 2 ? 1 : 0; }
                    if (ph.bc[0] == 3) { hif = true; hin = (R)(ph.inflow_c[0][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < nty) {                   // right column
                hx = ntx + 1; hy = t + 1; sy = y0 + t; sx = x0 + ntx;
                if (sx >= nx) {
                    if (ph.bc[1] == 0) sx = 0;
                    else { sx = nx - 1; hneg = ph.bc[1] == 2 ? 1 : 0; }
                    if (ph.bc[1] == 3) { hif = true; hin = -(R)(ph.inflow_c[1][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < ntx) {                   // bottom row
                hx = t + 1; hy = 0; sx = x0 + t; sy = y0 - 1;
                if (sy < 0) { if (ph.bc[2] == 0) sy = ny - 1; else { sy = 0; hneg = ph.bc[2] == 2 ? 2 : 0; } }
            } else if ((t -= ntx) < ntx) {                   // top row
                hx = t + 1; hy = nty + 1; sx = x0 + t; sy = y0 + nty;
                if (sy >= ny) { if (ph.bc[3] == 0) sy = 0; else { sy = ny - 1; hneg = ph.bc[3] == 2 ? 2 : 0; } }
            }
        }
        const int64_t own_col = (int64_t)y * nx + x;
        const int64_t halo_col = (int64_t)sy * nx + sx;

        // plane q of the run: z = z0 - 1 + q, wrapped or clamped at the faces
        auto src_plane = [&](int q, int &zneg) -> int {
            int zz = z0 - 1 + q;
            zneg = 0;
            if (zz < 0) { if (ph.bc[4] == 0) zz = nz - 1; else { zz = 0; zneg = ph.bc[4] == 2; } }
            else if (zz >= nz) { if (ph.bc[5] == 0) zz = 0; else { zz = nz - 1; zneg = ph.bc[5] == 2; } }
            return zz;
        };
        auto issue = [&](int q) {
            if (q < L) {
                int zneg;
                const int64_t pl = (int64_t)src_plane(q, zneg) * sxy;
                const int slot = q % S;
                if (act) cp_cell(&sm.U[slot][ty + 1][tx + 1], Ug + pl + own_col);
                if (hx >= 0) {
                    if (hif) sm.U[slot][hy][hx] = V4<R>{hin < R(0) ? -hin : hin, hin, R(0), R(0)};
                    else cp_cell(&sm.U[slot][hy][hx], Ug + pl + halo_col);
                }
            }
            cp_async_commit();
        };

#pragma unroll
        for (int q = 0; q < S - 2; q++) issue(q);

        R Fzm[4] = {R(0), R(0), R(0), R(0)};
        R szc_a = R(0), szc_b = R(0);     // HLL: z speeds of the plane being updated
        // FP64 fast form, GLF: the convex form of the update (as the FP32
        // kernel), from the cell below's U and G_z carried in registers
        constexpr bool CVX = !STRICT && !HLL;
        V4<R> ub = {};
        R gzb[4] = {R(0), R(0), R(0), R(0)};
        for (int q = 0; q < L; q++) {
            cp_async_wait<S - 3>();
            __syncthreads();        // plane q landed everywhere; plane q-1's closures visible;
                                    // plane q-2 retired (its U slot and P slot are reused)
            issue(q + S - 2);
            const int slot = q % S, pslot = q & 1;
            int zneg;
            src_plane(q, zneg);
            R Pn[6];
            V4<R> un = {};
            R szn_a = R(0), szn_b = R(0);
            if (act) {
                V4<R> &uref = sm.U[slot][ty + 1][tx + 1];
                if (zneg) uref.w = -uref.w;                // reflective z ghost plane
                un = uref;
                closure<R, STRICT>(un, Pn);
#pragma unroll
                for (int k = 0; k < 6; k++) sm.P[pslot][k][ty + 1][tx + 1] = Pn[k];
                if constexpr (HLL) {
                    // the cell's speeds along x, y (shared with the neighbours)
                    // and z (kept for its two z faces)
                    R Fn, zz, a, b;
                    hll_fz<R, STRICT>(un, Fn, zz);
                    hll_speed<R, STRICT, 0>(htab, un, Fn, zz, a, b);
                    sm.Sp[pslot][0][ty + 1][tx + 1] = a;
                    sm.Sp[pslot][1][ty + 1][tx + 1] = b;
                    hll_speed<R, STRICT, 1>(htab, un, Fn, zz, a, b);
                    sm.Sp[pslot][2][ty + 1][tx + 1] = a;
                    sm.Sp[pslot][3][ty + 1][tx + 1] = b;
                    hll_speed<R, STRICT, 2>(htab, un, Fn, zz, szn_a, szn_b);
                }
            }
            if (hx >= 0) {
                V4<R> &h = sm.U[slot][hy][hx];
                if (zneg) h.w = -h.w;
                if (hneg == 1) h.y = -h.y;
                else if (hneg == 2) h.z = -h.z;
                R Ph[6];
                closure<R, STRICT>(h, Ph);
#pragma unroll
                for (int k = 0; k < 6; k++) sm.P[pslot][k][hy][hx] = Ph[k];
                if constexpr (HLL) {
                    R Fn, zz, a, b;
                    hll_fz<R, STRICT>(h, Fn, zz);
                    hll_speed<R, STRICT, 0>(htab, h, Fn, zz, a, b);
                    sm.Sp[pslot][0][hy][hx] = a;
                    sm.Sp[pslot][1][hy][hx] = b;
                    hll_speed<R, STRICT, 1>(htab, h, Fn, zz, a, b);
                    sm.Sp[pslot][2][hy][hx] = a;
                    sm.Sp[pslot][3][hy][hx] = b;
                }
            }
            const R sza = szc_a, szb = szc_b;
            szc_a = szn_a;
            szc_b = szn_b;
            if (q == 0 || !act) continue;
            // update plane c = q - 1 (z = z0 + q - 2) unless c is the ghost plane 0
            const int c = q - 1, cs = c % S, cp = c & 1;
            const V4<R> uc = sm.U[cs][ty + 1][tx + 1];
            R Pc[6];
#pragma unroll
            for (int k = 0; k < 6; k++) Pc[k] = sm.P[cp][k][ty + 1][tx + 1];
            if constexpr (CVX) {
                // U* = (1 - 3 lam) U + (lam/2) sum_d [(U + G_d)(left_d) + (U - G_d)(right_d)],
                // G_x = (Fx, Pxx, Pxy, Pxz), G_y = (Fy, Pxy, Pyy, Pyz), G_z = (Fz, Pxz, Pyz, Pzz):
                // equal to U - lam sum_d (Phi_{d,+} - Phi_{d,-}) with Phi of Eq. e:glf,
                // each face's terms formed once
                if (c >= 1) {
                    R Pl[6], Pr[6], Pd[6], Pu[6];
#pragma unroll
                    for (int k = 0; k < 6; k++) {
                        Pl[k] = sm.P[cp][k][ty + 1][tx];
                        Pr[k] = sm.P[cp][k][ty + 1][tx + 2];
                        Pd[k] = sm.P[cp][k][ty][tx + 1];
                        Pu[k] = sm.P[cp][k][ty + 2][tx + 1];
                    }
                    const V4<R> ul = sm.U[cs][ty + 1][tx], ur = sm.U[cs][ty + 1][tx + 2];
                    const V4<R> ud = sm.U[cs][ty][tx + 1], uu = sm.U[cs][ty + 2][tx + 1];
                    const R c0 = R(1) - R(3) * lam, c1 = R(0.5) * lam;
                    R o[4];
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const R gxl = m == 0 ? ul.y : Pl[pidx(0, m - 1)];
                        const R gxr = m == 0 ? ur.y : Pr[pidx(0, m - 1)];
                        const R gyd = m == 0 ? ud.z : Pd[pidx(1, m - 1)];
                        const R gyu = m == 0 ? uu.z : Pu[pidx(1, m - 1)];
                        const R gzu = m == 0 ? un.w : Pn[pidx(2, m - 1)];
                        const R sx = (comp(ul, m) + gxl) + (comp(ur, m) - gxr);
                        const R sy = (comp(ud, m) + gyd) + (comp(uu, m) - gyu);
                        const R sz = (comp(ub, m) + gzb[m]) + (comp(un, m) - gzu);
                        o[m] = c0 * comp(uc, m) + c1 * ((sx + sy) + sz);
                    }
                    const int z = z0 + c - 1;
                    st4(Og + (int64_t)z * sxy + own_col, V4<R>{o[0], o[1], o[2], o[3]});
                }
                ub = uc;
                gzb[0] = uc.w;
                gzb[1] = Pc[2];
                gzb[2] = Pc[4];
                gzb[3] = Pc[5];
                continue;
            }
            R Fzp[4];
            if constexpr (HLL) {
                hll<R, STRICT, 2>(uc, Pc, sza, szb, un, Pn, szn_a, szn_b, Fzp);
            } else {
                glf<R, 2>(uc, Pc, un, Pn, Fzp);
            }
            if (c >= 1) {
                R Pl[6], Pr[6], Pd[6], Pu[6];
#pragma unroll
                for (int k = 0; k < 6; k++) {
                    Pl[k] = sm.P[cp][k][ty + 1][tx];
                    Pr[k] = sm.P[cp][k][ty + 1][tx + 2];
                    Pd[k] = sm.P[cp][k][ty][tx + 1];
                    Pu[k] = sm.P[cp][k][ty + 2][tx + 1];
                }
                const V4<R> ul = sm.U[cs][ty + 1][tx], ur = sm.U[cs][ty + 1][tx + 2];
                const V4<R> ud = sm.U[cs][ty][tx + 1], uu = sm.U[cs][ty + 2][tx + 1];
                R Fxm[4], Fxp[4], Fym[4], Fyp[4];
                if constexpr (HLL) {
                    const R cxa = sm.Sp[cp][0][ty + 1][tx + 1], cxb = sm.Sp[cp][1][ty + 1][tx + 1];
                    const R cya = sm.Sp[cp][2][ty + 1][tx + 1], cyb = sm.Sp[cp][3][ty + 1][tx + 1];
                    hll<R, STRICT, 0>(ul, Pl, sm.Sp[cp][0][ty + 1][tx], sm.Sp[cp][1][ty + 1][tx], uc, Pc,
                                      cxa, cxb, Fxm);
                    hll<R, STRICT, 0>(uc, Pc, cxa, cxb, ur, Pr, sm.Sp[cp][0][ty + 1][tx + 2],
                                      sm.Sp[cp][1][ty + 1][tx + 2], Fxp);
                    hll<R, STRICT, 1>(ud, Pd, sm.Sp[cp][2][ty][tx + 1], sm.Sp[cp][3][ty][tx + 1], uc, Pc,
                                      cya, cyb, Fym);
                    hll<R, STRICT, 1>(uc, Pc, cya, cyb, uu, Pu, sm.Sp[cp][2][ty + 2][tx + 1],
                                      sm.Sp[cp][3][ty + 2][tx + 1], Fyp);
                } else {
                    glf<R, 0>(ul, Pl, uc, Pc, Fxm);
                    glf<R, 0>(uc, Pc, ur, Pr, Fxp);
                    glf<R, 1>(ud, Pd, uc, Pc, Fym);
                    glf<R, 1>(uc, Pc, uu, Pu, Fyp);
                }
                R o[4];
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    const R dxf = Fxp[m] - Fxm[m];
                    const R dyf = Fyp[m] - Fym[m];
                    const R dzf = Fzp[m] - Fzm[m];
                    o[m] = comp(uc, m) - lam * ((dxf + dyf) + dzf);
                }
                if constexpr (HLL) {
                    // |F| <= N after an HLL step: the speeds mu of f = 1 would
                    // amplify the excess that rounding leaves in beam cells
                    const R Fn = rsqrt_(o[1] * o[1] + o[2] * o[2] + o[3] * o[3]);
                    if (Fn > o[0]) {
                        const R r = o[0] > R(0) ? o[0] / Fn : R(0);
                        o[1] *= r;
                        o[2] *= r;
                        o[3] *= r;
                    }
                }
                const int z = z0 + c - 1;
                st4(Og + (int64_t)z * sxy + own_col, V4<R>{o[0], o[1], o[2], o[3]});
            }
#pragma unroll
            for (int m = 0; m < 4; m++) Fzm[m] = Fzp[m];
        }
        cp_async_wait<0>();
        __syncthreads();                                   // ring free for the next run
    }
}

#ifndef RTK_SKIP_SINGLE_KERNELS
// single-instruction MUFU reciprocal and reciprocal square root (~1 ulp)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed form of a cell for the FP32 transport: U = (lo, hi) = ((N, Fx),
// (Fy, Fz)) and the right-/left-going GLF halves U +- G_d(U) per axis, with
// G_x = (Fx, Pxx, Pxy, Pxz), G_y = (Fy, Pxy, Pyy, Pyz), G_z = (Fz, Pxz, Pyz,
// Pzz) and P = N D from the Levermore closure (the formulas of closure(),
// with MUFU reciprocals, N below 1e-37 -- FP32 denormals -- giving P = 0, and
// N a + N g u_d u_j formed as (N g u_d) u_j + N a).
struct Halves {
    float4 R[3], L[3];
};

__device__ __forceinline__ float4 f4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

__device__ __forceinline__ void cell_closure(const V4<float> &u, float &P0, float &P1, float &P2, float &P3,
                                             float &P4, float &P5)
{
    const float N = u.x;
    P0 = 0.f; P1 = 0.f; P2 = 0.f; P3 = 0.f; P4 = 0.f; P5 = 0.f;
    if (N > 1e-37f) {
        const float rN = rcp_approx(N);
        float ux = u.y * rN, uy = u.z * rN, uz = u.w * rN;
        float f2 = ux * ux + uy * uy + uz * uz;
        if (f2 > 1.0f) {
            const float rf = rsqrt_approx(f2);
            ux *= rf; uy *= rf; uz *= rf;
            f2 = 1.0f;
        }
        const float q = 4.0f - 3.0f * f2;
        const float s = q * rsqrt_approx(q);
        const float r5 = rcp_approx(5.0f + 2.0f * s);
        const float Na = N * (((1.0f + s) - 2.0f * f2) * r5);
        const float Ng = N * ((6.0f + 3.0f * rcp_approx(2.0f + s)) * r5);
        const float gx = Ng * ux, gy = Ng * uy, gz = Ng * uz;
        P0 = gx * ux + Na; P3 = gy * uy + Na; P5 = gz * uz + Na;
        P1 = gx * uy; P2 = gx * uz; P4 = gy * uz;
    }
}

__device__ __forceinline__ void halves_of(const V4<float> &u, float P0, float P1, float P2, float P3, float P4,
                                          float P5, Halves &h)
{
    // scalar adds: the flux vectors' components are not aligned register
    // pairs, so packed adds would need moves to assemble them (same rounding)
    const float G[3][4] = {{u.y, P0, P1, P2}, {u.z, P1, P3, P4}, {u.w, P2, P4, P5}};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        h.R[d] = make_float4(u.x + G[d][0], u.y + G[d][1], u.z + G[d][2], u.w + G[d][3]);
        h.L[d] = make_float4(u.x - G[d][0], u.y - G[d][1], u.z - G[d][2], u.w - G[d][3]);
    }
}

__device__ __forceinline__ void cell_halves(const V4<float> &u, Halves &h)
{
    float P0, P1, P2, P3, P4, P5;
    cell_closure(u, P0, P1, P2, P3, P4, P5);
    halves_of(u, P0, P1, P2, P3, P4, P5, h);
}

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// The run of plane units of box B that starts at unit loc (relative to the
// box) and takes at most `left` units: group g, tile (ix, iy), planes
// z0 .. z1-1.  Units are ordered (group, y-tile, z-chunk, x-tile, z) with
// z-chunks of B.zlen planes (the last one shorter), so with chunks shorter
// than the box a block's consecutive runs are neighbouring tiles over the
// same planes and the x-halo lines of one run were read as interior by the
// run before, still in L2.  B.zlen = nz is the column order.
__device__ __forceinline__ void transport_run(const BoxDev &B, int64_t loc, int64_t left, int &g,
                                              int &iy, int &ix, int &z0, int &z1)
{
    const int nz = B.nz, Lz = B.zlen;
    const int64_t per_row = (int64_t)nz * B.tiles_x;        // units of one row of tiles
    const int64_t row = loc / per_row;
    int64_t r = loc - row * per_row;
    iy = (int)(row % B.tiles_y);
    g = (int)(row / B.tiles_y);
    const int nfull = nz / Lz;                                // full chunks
    const int64_t full = (int64_t)B.tiles_x * Lz;             // units of a full chunk
    int zc = (int)(r / full), Lc = Lz;
    if (zc >= nfull) { zc = nfull; Lc = nz - nfull * Lz; }
    r -= (int64_t)zc * full;
    ix = (int)(r / Lc);
    const int zz = (int)(r - (int64_t)ix * Lc);
    z0 = zc * Lz + zz;
    const int zend = zc * Lz + Lc;
    const int64_t lim = (int64_t)z0 + left;
    z1 = lim < (int64_t)zend ? (int)lim : zend;
}

// the FP32 GLF kernel streams one plane deeper than the others (4 planes
// ahead): it is the one bound by DRAM latency
constexpr int TP_STAGES_PM = 6;

// rows padded by one cell: the halo columns' threads, one row apart, then
// fall on distinct banks (a row of TX + 3 cells is 4 (TX + 3) words)
template <int TX, int TY>
struct TransportSmemPM {
    V4<float> U[TP_STAGES_PM][TY + 2][TX + 3];
    float4 H[2][4][TY + 2][TX + 3];    // per cell: Rx, Lx, Ry, Ly of two planes
};

// The TMA ring: each plane's tile with its halo as the dense box the copy
// writes (128-byte aligned slots), the wrapped halo columns and rows of
// periodic faces (their own small boxes), one mbarrier per slot.
template <int TX, int TY>
struct alignas(128) PMSlot {
    V4<float> c[TY + 2][TX + 2];
};
template <int N>
struct alignas(128) PMLine {
    V4<float> c[N];
};
template <int TX, int TY>
struct TransportSmemPMT {
    PMSlot<TX, TY> U[TP_STAGES_PM];
    PMLine<TY> Wx[TP_STAGES_PM][2];    // x = nx - 1 (left halo), x = 0 (right halo)
    PMLine<TX> Wy[TP_STAGES_PM][2];    // y = ny - 1 (bottom halo), y = 0 (top halo)
    float4 H[2][4][TY + 2][TX + 3];
    unsigned long long bar[TP_STAGES_PM];
};

template <int TX, int TY, bool TMA = false>
constexpr size_t transport_pm_smem_bytes()
{
    return TMA ? sizeof(TransportSmemPMT<TX, TY>) : sizeof(TransportSmemPM<TX, TY>);
}

// threads of the FP32 GLF kernel's block: TX x TY interior cells and the
// 2 (TX + TY) halo cells of the tile, one cell each, rounded up to warps
template <int TX, int TY>
constexpr int transport_pm_threads() { return (TX * TY + 2 * (TX + TY) + 31) / 32 * 32; }

// This block's share [ubeg, uend) of the launch's plane units.  lockx > 0
// (lockstep rows): the grid is groups of lockx blocks; group k takes the
// k-th equal share of the row-planes (box, group, y-tile, z) and block lix
// of the group their tile column lix.
__device__ __forceinline__ void pm_share(int64_t nunits, int lockx, int64_t &ubeg, int64_t &uend, int &lix)
{
    lix = 0;
    if (lockx > 0) {
        const int64_t m = gridDim.x / lockx, k = blockIdx.x / lockx;
        lix = (int)(blockIdx.x - k * lockx);
        const int64_t nrp = nunits / lockx;   // row-planes of all boxes
        ubeg = nrp * k / m;
        uend = nrp * (k + 1) / m;
    } else {
        ubeg = nunits * (int64_t)blockIdx.x / gridDim.x;
        uend = nunits * (int64_t)(blockIdx.x + 1) / gridDim.x;
    }
}

// The run that starts at unit u of the share (at most uend - u units):
// returns its box; group g, tile (ix, iy), planes z0 .. z1-1.  Lockstep: u
// counts row-planes and the tile column is lix.
__device__ __forceinline__ int pm_run(const BoxDev *__restrict__ boxes, int nboxes, int64_t u, int64_t uend,
                                      int lockx, int lix, int &g, int &iy, int &ix, int &z0, int &z1)
{
    if (lockx > 0) {
        // box of row-plane u: the last with titem0 / lockx <= u
        int lo = 0, hi = nboxes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (boxes[mid].titem0 / lockx <= u) lo = mid; else hi = mid - 1;
        }
        const BoxDev &Bb = boxes[lo];
        const int64_t loc = u - Bb.titem0 / lockx;
        const int64_t row = loc / Bb.nz;
        z0 = (int)(loc - row * Bb.nz);
        const int64_t lim = (int64_t)z0 + (uend - u);
        z1 = lim < (int64_t)Bb.nz ? (int)lim : Bb.nz;
        iy = (int)(row % Bb.tiles_y);
        g = (int)(row / Bb.tiles_y);
        ix = lix;
        return lo;
    }
    const int b = find_box_unit(boxes, nboxes, u);
    transport_run(boxes[b], u - boxes[b].titem0, uend - u, g, iy, ix, z0, z1);
    return b;
}

// FP32 transport of the split form.  Same pipeline and work split as
// k_transport; the unsplit GLF update is evaluated in its convex form
//   U* = (1 - 3 lam) U + (lam/2) sum_d [ (U + G_d)(left_d) + (U - G_d)(right_d) ],
// which equals U - lam sum_d (Phi_{d,+} - Phi_{d,-}) with Phi of Eq. e:glf.
// Each cell computes its halves once per plane; x/y neighbours read them from
// shared memory, the z halves stay in registers.  The tile (TX x TY columns)
// is a template parameter so the launch shape can be tuned per box set;
// every shape computes each cell with the same arithmetic.  The block holds
// one thread per interior column and one per halo column (x: left and
// right, y: bottom and top), so every thread evaluates exactly one closure
// per plane and no warp waits at the plane's barrier for another's second
// closure; the halo threads take no part in the update.
// TMA: one thread issues each plane as a TMA copy of the tile with its halo
// (rows of TX + 2 cells), completing on the slot's mbarrier; tiles on a
// periodic face add the wrapped column or row as a small box of its own.
// Otherwise every thread copies its own cell by cp.async.
// lockx > 0 (every box has lockx tile columns): lockstep rows.  The grid is
// groups of lockx blocks; block (k, ix) of group k takes tile column ix of
// the k-th equal share of the row-planes (box, group, y-tile, z), so the
// blocks of a group work on the tiles of one row at the same planes at the
// same time, and the lines a tile reads for its x-halo are its neighbours'
// interior lines, read at once from L2 instead of again from DRAM.
template <int TX, int TY, bool TMA>
__global__ void __launch_bounds__(transport_pm_threads<TX, TY>(), 2)
k_transport_pm(const BoxDev *__restrict__ boxes, int nboxes, int64_t nunits, int lockx, Phys ph,
               Ctl *ctl)
{
    constexpr int S = TP_STAGES_PM;
    extern __shared__ __align__(128) unsigned char tp_smem_pm[];
    TransportSmemPM<TX, TY> &sm = *reinterpret_cast<TransportSmemPM<TX, TY> *>(tp_smem_pm);
    TransportSmemPMT<TX, TY> &st = *reinterpret_cast<TransportSmemPMT<TX, TY> *>(tp_smem_pm);
    auto ring = [&](int slot, int yy, int xx) -> V4<float> & {
        if constexpr (TMA) return st.U[slot].c[yy][xx];
        else return sm.U[slot][yy][xx];
    };
    auto Hs = [&](int hs, int k, int yy, int xx) -> float4 & {
        if constexpr (TMA) return st.H[hs][k][yy][xx];
        else return sm.H[hs][k][yy][xx];
    };

    const int tid = threadIdx.x;
    const bool interior = tid < TX * TY;
    const int tx = interior ? tid % TX : 0, ty = interior ? tid / TX : 0;
    if (blockIdx.x == 0 && tid == 0) ctl->step += 1;
    if constexpr (TMA) {
        // the copies write 128-byte aligned slots: a misplaced window is
        // reported, not copied into (the same test in every thread)
        if (smem_u32(tp_smem_pm) & 127u) {
            if (tid == 0) atomicOr(&ctl->err, RTD_ERR_TIMEOUT);
            return;
        }
        if (tid == 0) {
            for (int k = 0; k < S; k++) mbar_init(&st.bar[k], 1u);
            mbar_init_fence();
        }
        __syncthreads();
    }
    unsigned pl_issued = 0, pl_done = 0;      // planes issued / consumed by the block

    int64_t ubeg, uend;
    int lix;                                  // lockstep: this block's tile column
    pm_share(nunits, lockx, ubeg, uend, lix);
    for (int64_t u = ubeg; u < uend;) {
        int g, iy, ix, z0, z1;
        const int b = pm_run(boxes, nboxes, u, uend, lockx, lix, g, iy, ix, z0, z1);
        const BoxDev &B = boxes[b];
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        u += z1 - z0;
        if (ix >= B.tiles_x) continue;        // (lockstep on a box of other width: not set up)
        const int x0 = ix * TX, y0 = iy * TY;
        const int ntx = min(TX, nx - x0), nty = min(TY, ny - y0);
        const int x = x0 + tx, y = y0 + ty;
        const bool act = interior && (tx < ntx) && (ty < nty);
        const int L = (z1 - z0) + 2;
        const V4<float> *Ug = reinterpret_cast<const V4<float> *>(B.U) + (int64_t)g * B.ncell;
        V4<float> *Og = reinterpret_cast<V4<float> *>(B.Us) + (int64_t)g * B.ncell;
        const float lam = (float)B.lam;
        const float c0 = 1.0f - 3.0f * lam, c1 = 0.5f * lam;
        const int64_t sxy = (int64_t)nx * ny;
        // periodic faces of this tile (TMA: their wrapped halo lines come as
        // boxes of their own)
        const bool wl = x0 == 0 && ph.bc[0] == 0, wr = x0 + ntx == nx && ph.bc[1] == 0;
        const bool wb = y0 == 0 && ph.bc[2] == 0, wt = y0 + nty == ny && ph.bc[3] == 0;

        // halo cell of a halo thread and which half of it the tile needs:
        // 0 = Rx (left column), 1 = Lx (right), 2 = Ry (bottom), 3 = Ly (top)
        int hx = -1, hy = -1, sx = 0, sy = 0, hneg = 0, hk = 0;
        float hin = 0.0f;                 // inflow ghost: beam density, sign = direction
        bool hif = false;                 // the halo cell is an inflow ghost
        // TMA: where the halo cell is read: the box at (hry, hrx), or (hw >= 0)
        // wrapped line hw (0 Wx left, 1 Wx right, 2 Wy bottom, 3 Wy top) at hwi
        int hry = 0, hrx = 0, hw = -1, hwi = 0;
        if (!interior) {
            int t = tid - TX * TY;
            if (t < nty) {
                hx = 0; hy = t + 1; sy = y0 + t; sx = x0 - 1; hk = 0;
                hry = hy; hrx = 0;
                if (sx < 0) {
                    if (ph.bc[0] == 0) { sx = nx - 1; hw = 0; hwi = t; }
                    else { sx = 0; hneg = ph.bc[0] == 2 ? 1 : 0; hrx = 1; }
                    if (ph.bc[0] == 3) { hif = true; hin = (float)(ph.inflow_c[0][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < nty) {
                hx = ntx + 1; hy = t + 1; sy = y0 + t; sx = x0 + ntx; hk = 1;
                hry = hy; hrx = ntx + 1;
                if (sx >= nx) {
                    if (ph.bc[1] == 0) { sx = 0; hw = 1; hwi = t; }
                    else { sx = nx - 1; hneg = ph.bc[1] == 2 ? 1 : 0; hrx = ntx; }
                    if (ph.bc[1] == 3) { hif = true; hin = -(float)(ph.inflow_c[1][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < ntx) {
                hx = t + 1; hy = 0; sx = x0 + t; sy = y0 - 1; hk = 2;
                hry = 0; hrx = hx;
                if (sy < 0) {
                    if (ph.bc[2] == 0) { sy = ny - 1; hw = 2; hwi = t; }
                    else { sy = 0; hneg = ph.bc[2] == 2 ? 2 : 0; hry = 1; }
                }
            } else if ((t -= ntx) < ntx) {
                hx = t + 1; hy = nty + 1; sx = x0 + t; sy = y0 + nty; hk = 3;
                hry = nty + 1; hrx = hx;
                if (sy >= ny) {
                    if (ph.bc[3] == 0) { sy = 0; hw = 3; hwi = t; }
                    else { sy = ny - 1; hneg = ph.bc[3] == 2 ? 2 : 0; hry = nty; }
                }
            }
        }
        // source pointers of this thread's own and halo cells, advanced one
        // plane per issue; plane q is z0 - 1 + q, wrapped (periodic) or
        // clamped (ghost planes copy the face plane, negated when reflective)
        const V4<float> *gown = Ug + (int64_t)y * nx + x;
        const V4<float> *ghalo = Ug + (int64_t)sy * nx + sx;
        const bool zneg_first = z0 == 0 && ph.bc[4] == 2, zneg_last = z1 == nz && ph.bc[5] == 2;
        int zi = z0 - 1;                          // plane of the next issue
        int slot_i = (int)(pl_issued % S);        // its ring slot
        // offset of plane zi inside the box (advanced by one plane per
        // issue) and of the two ghost planes
        int64_t pl_in = (int64_t)zi * sxy;
        const int64_t pl_lo = ph.bc[4] == 0 ? (int64_t)(nz - 1) * sxy : 0;
        const int64_t pl_hi = ph.bc[5] == 0 ? 0 : (int64_t)(nz - 1) * sxy;
        const int zlo = ph.bc[4] == 0 ? nz - 1 : 0, zhi = ph.bc[5] == 0 ? 0 : nz - 1;
        const void *tm = B.tmap;
        auto issue = [&]() {
            if (zi < z1 + 1) {
                if constexpr (TMA) {
                    if (tid == 0) {
                        // the ring slot was read in an earlier plane (the
                        // barrier before the issue ordered those reads)
                        fence_proxy_async_smem();
                        const int zz = zi < 0 ? zlo : (zi >= nz ? zhi : zi);
                        const int c3 = g * nz + zz;
                        unsigned bytes = (unsigned)sizeof(PMSlot<TX, TY>::c);
                        if (wl) bytes += (unsigned)sizeof(PMLine<TY>::c);
                        if (wr) bytes += (unsigned)sizeof(PMLine<TY>::c);
                        if (wb) bytes += (unsigned)sizeof(PMLine<TX>::c);
                        if (wt) bytes += (unsigned)sizeof(PMLine<TX>::c);
                        unsigned long long *bar = &st.bar[slot_i];
                        mbar_expect_tx(bar, bytes);
                        const char *tmc = static_cast<const char *>(tm);
                        tma_load_4d(&st.U[slot_i].c[0][0], tmc, 0, x0 - 1, y0 - 1, c3, bar);
                        if (wl) tma_load_4d(&st.Wx[slot_i][0].c[0], tmc + 128, 0, nx - 1, y0, c3, bar);
                        if (wr) tma_load_4d(&st.Wx[slot_i][1].c[0], tmc + 128, 0, 0, y0, c3, bar);
                        if (wb) tma_load_4d(&st.Wy[slot_i][0].c[0], tmc + 256, 0, x0, ny - 1, c3, bar);
                        if (wt) tma_load_4d(&st.Wy[slot_i][1].c[0], tmc + 256, 0, x0, 0, c3, bar);
                    }
                } else {
                    const int64_t pl = zi < 0 ? pl_lo : (zi >= nz ? pl_hi : pl_in);
                    if (act) cp_async16(&sm.U[slot_i][ty + 1][tx + 1], gown + pl);
                    if (hx >= 0) {
                        if (hif) sm.U[slot_i][hy][hx] = V4<float>{fabsf(hin), hin, 0.0f, 0.0f};
                        else cp_async16(&sm.U[slot_i][hy][hx], ghalo + pl);
                    }
                }
                pl_issued++;
            }
            if constexpr (!TMA) cp_async_commit();
            zi++;
            pl_in += sxy;
            slot_i = slot_i + 1 == S ? 0 : slot_i + 1;
        };
#pragma unroll
        for (int q = 0; q < S - 2; q++) issue();

        V4<float> uc = {};                  // own cell of plane q-1
        float4 Rz_prev = {}, Rz_c = {};     // right-going z halves of planes q-2 and q-1
        V4<float> *out = Og + (int64_t)z0 * sxy + (int64_t)y * nx + x;
        int slot = (int)(pl_done % S);      // ring slot of plane q
#pragma unroll 3
        for (int q = 0; q < L; q++) {
            if constexpr (TMA) {
                // plane q landed (every thread observes its slot's phase);
                // a wait that gives up stops the whole block at the barrier
                const bool ok = mbar_wait(&st.bar[slot], (pl_done / S) & 1u, RTK_TMA_POLLS);
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) atomicOr(&ctl->err, RTD_ERR_TIMEOUT);
                    return;
                }
            } else {
                cp_async_wait<S - 3>();
                __syncthreads();
            }
            pl_done++;
            issue();
            const int hs = q & 1;
            const bool zneg = (q == 0 && zneg_first) || (q == L - 1 && zneg_last);
            V4<float> un = {};
            float4 Rz_n = {}, Lz_n = {};
            if (act) {
                un = ring(slot, ty + 1, tx + 1);
                if (zneg) un.w = -un.w;
                Halves hv;
                cell_halves(un, hv);
                Rz_n = hv.R[2];
                Lz_n = hv.L[2];
                Hs(hs, 0, ty + 1, tx + 1) = hv.R[0];
                Hs(hs, 1, ty + 1, tx + 1) = hv.L[0];
                Hs(hs, 2, ty + 1, tx + 1) = hv.R[1];
                Hs(hs, 3, ty + 1, tx + 1) = hv.L[1];
            }
            if (hx >= 0) {
                V4<float> h;
                if constexpr (TMA) {
                    if (hif) h = V4<float>{fabsf(hin), hin, 0.0f, 0.0f};
                    else if (hw >= 0) h = hw < 2 ? st.Wx[slot][hw].c[hwi] : st.Wy[slot][hw - 2].c[hwi];
                    else h = st.U[slot].c[hry][hrx];
                } else {
                    h = sm.U[slot][hy][hx];
                }
                if (zneg) h.w = -h.w;
                if (hneg == 1) h.y = -h.y;
                else if (hneg == 2) h.z = -h.z;
                Halves hv;
                cell_halves(h, hv);
                Hs(hs, hk, hy, hx) = hk == 0 ? hv.R[0] : hk == 1 ? hv.L[0] : hk == 2 ? hv.R[1] : hv.L[1];
            }
            if (act && q >= 2) {
                // update plane c = q - 1 (z = z0 + q - 2)
                const int cs = hs ^ 1;
                const float4 l = Hs(cs, 0, ty + 1, tx);        // Rx of the left cell
                const float4 r = Hs(cs, 1, ty + 1, tx + 2);    // Lx of the right cell
                const float4 d = Hs(cs, 2, ty, tx + 1);        // Ry of the cell below
                const float4 p = Hs(cs, 3, ty + 2, tx + 1);    // Ly of the cell above
                const float2 slo = __fadd2_rn(__fadd2_rn(__fadd2_rn(lo2(l), lo2(r)), __fadd2_rn(lo2(d), lo2(p))),
                                              __fadd2_rn(lo2(Rz_prev), lo2(Lz_n)));
                const float2 shi = __fadd2_rn(__fadd2_rn(__fadd2_rn(hi2(l), hi2(r)), __fadd2_rn(hi2(d), hi2(p))),
                                              __fadd2_rn(hi2(Rz_prev), hi2(Lz_n)));
                const float2 cc0 = make_float2(c0, c0), cc1 = make_float2(c1, c1);
                const float2 olo = __ffma2_rn(cc0, make_float2(uc.x, uc.y), __fmul2_rn(cc1, slo));
                const float2 ohi = __ffma2_rn(cc0, make_float2(uc.z, uc.w), __fmul2_rn(cc1, shi));
                st4(out, V4<float>{olo.x, olo.y, ohi.x, ohi.y});
                out += sxy;
            }
            Rz_prev = Rz_c;
            Rz_c = Rz_n;
            uc = un;
            slot = slot + 1 == S ? 0 : slot + 1;
        }
        if constexpr (!TMA) cp_async_wait<0>();
        __syncthreads();
    }
}

// Groups per block: the FP32 GLF transport with NG photon groups of each
// tile in one block (the units count group blocks, ceil(G / NG) per tile and
// plane).  Every thread copies and updates its cell in each of the block's
// groups per plane: NG independent closures between two barriers, and the
// barrier, the plane bookkeeping and the halo logic shared by the groups.
// Layout, work orders (column, z-chunked, lockstep rows), per-cell arithmetic
// and results are those of k_transport_pm with per-thread copies; the ring
// and the halves hold NG groups, so NG = 2 takes one block per SM.
template <int TX, int TY, int NG>
struct TransportSmemPMG {
    V4<float> U[TP_STAGES_PM][NG][TY + 2][TX + 3];
    float4 H[2][NG][4][TY + 2][TX + 3];
};

template <int TX, int TY, int NG>
constexpr size_t transport_pmg_smem_bytes() { return sizeof(TransportSmemPMG<TX, TY, NG>); }

template <int TX, int TY, int NG>
__global__ void __launch_bounds__(transport_pm_threads<TX, TY>(), 1)
k_transport_pmg(const BoxDev *__restrict__ boxes, int nboxes, int64_t nunits, int lockx, Phys ph,
                Ctl *ctl)
{
    static_assert(NG >= 2 && NG <= RTD_MAXG, "groups per block");
    constexpr int S = TP_STAGES_PM;
    extern __shared__ __align__(128) unsigned char tp_smem_pmg[];
    auto &sm = *reinterpret_cast<TransportSmemPMG<TX, TY, NG> *>(tp_smem_pmg);

    const int tid = threadIdx.x;
    const bool interior = tid < TX * TY;
    const int tx = interior ? tid % TX : 0, ty = interior ? tid / TX : 0;
    if (blockIdx.x == 0 && tid == 0) ctl->step += 1;

    int64_t ubeg, uend;
    int lix;
    pm_share(nunits, lockx, ubeg, uend, lix);
    for (int64_t u = ubeg; u < uend;) {
        int gb, iy, ix, z0, z1;
        const int b = pm_run(boxes, nboxes, u, uend, lockx, lix, gb, iy, ix, z0, z1);
        const BoxDev &B = boxes[b];
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        u += z1 - z0;
        if (ix >= B.tiles_x) continue;        // (lockstep on a box of other width: not set up)
        const int g0 = gb * NG, ng = min(NG, ph.G - g0);     // the block's groups g0 .. g0+ng-1
        const int x0 = ix * TX, y0 = iy * TY;
        const int ntx = min(TX, nx - x0), nty = min(TY, ny - y0);
        const int x = x0 + tx, y = y0 + ty;
        const bool act = interior && (tx < ntx) && (ty < nty);
        const int L = (z1 - z0) + 2;
        const int64_t gst = B.ncell;          // one group's cells
        const V4<float> *Ug = reinterpret_cast<const V4<float> *>(B.U) + (int64_t)g0 * gst;
        V4<float> *Og = reinterpret_cast<V4<float> *>(B.Us) + (int64_t)g0 * gst;
        const float lam = (float)B.lam;
        const float c0 = 1.0f - 3.0f * lam, c1 = 0.5f * lam;
        const int64_t sxy = (int64_t)nx * ny;

        // halo cell of a halo thread and which half of it the tile needs:
        // 0 = Rx (left column), 1 = Lx (right), 2 = Ry (bottom), 3 = Ly (top)
        int hx = -1, hy = -1, sx = 0, sy = 0, hneg = 0, hk = 0;
        float hin[NG];                    // inflow ghost per group: beam density, sign = direction
#pragma unroll
        for (int k = 0; k < NG; k++) hin[k] = 0.0f;
        bool hif = false;                 // the halo cell is an inflow ghost
        if (!interior) {
            int t = tid - TX * TY;
            if (t < nty) {
                hx = 0; hy = t + 1; sy = y0 + t; sx = x0 - 1; hk = 0;
                if (sx < 0) {
                    if (ph.bc[0] == 0) sx = nx - 1;
                    else { sx = 0; hneg = ph.bc[0] == 2 ? 1 : 0; }
                    if (ph.bc[0] == 3) {
                        hif = true;
#pragma unroll
                        for (int k = 0; k < NG; k++)
                            if (k < ng) hin[k] = (float)(ph.inflow_c[0][g0 + k] * B.inv_nunit);
                    }
                }
            } else if ((t -= nty) < nty) {
                hx = ntx + 1; hy = t + 1; sy = y0 + t; sx = x0 + ntx; hk = 1;
                if (sx >= nx) {
                    if (ph.bc[1] == 0) sx = 0;
                    else { sx = nx - 1; hneg = ph.bc[1] == 2 ? 1 : 0; }
                    if (ph.bc[1] == 3) {
                        hif = true;
#pragma unroll
                        for (int k = 0; k < NG; k++)
                            if (k < ng) hin[k] = -(float)(ph.inflow_c[1][g0 + k] * B.inv_nunit);
                    }
                }
            } else if ((t -= nty) < ntx) {
                hx = t + 1; hy = 0; sx = x0 + t; sy = y0 - 1; hk = 2;
                if (sy < 0) {
                    if (ph.bc[2] == 0) sy = ny - 1;
                    else { sy = 0; hneg = ph.bc[2] == 2 ? 2 : 0; }
                }
            } else if ((t -= ntx) < ntx) {
                hx = t + 1; hy = nty + 1; sx = x0 + t; sy = y0 + nty; hk = 3;
                if (sy >= ny) {
                    if (ph.bc[3] == 0) sy = 0;
                    else { sy = ny - 1; hneg = ph.bc[3] == 2 ? 2 : 0; }
                }
            }
        }
        // plane q is z0 - 1 + q, wrapped (periodic) or clamped (ghost planes
        // copy the face plane, negated when reflective); the ring starts at
        // slot 0 in every run (the previous run drained it)
        const V4<float> *gown = Ug + (int64_t)y * nx + x;
        const V4<float> *ghalo = Ug + (int64_t)sy * nx + sx;
        const bool zneg_first = z0 == 0 && ph.bc[4] == 2, zneg_last = z1 == nz && ph.bc[5] == 2;
        int zi = z0 - 1;
        int slot_i = 0;
        int64_t pl_in = (int64_t)zi * sxy;
        const int64_t pl_lo = ph.bc[4] == 0 ? (int64_t)(nz - 1) * sxy : 0;
        const int64_t pl_hi = ph.bc[5] == 0 ? 0 : (int64_t)(nz - 1) * sxy;
        auto issue = [&]() {
            if (zi < z1 + 1) {
                const int64_t pl = zi < 0 ? pl_lo : (zi >= nz ? pl_hi : pl_in);
#pragma unroll
                for (int k = 0; k < NG; k++) {
                    if (k < ng) {
                        if (act) cp_async16(&sm.U[slot_i][k][ty + 1][tx + 1], gown + k * gst + pl);
                        if (hx >= 0) {
                            if (hif) sm.U[slot_i][k][hy][hx] = V4<float>{fabsf(hin[k]), hin[k], 0.0f, 0.0f};
                            else cp_async16(&sm.U[slot_i][k][hy][hx], ghalo + k * gst + pl);
                        }
                    }
                }
            }
            cp_async_commit();
            zi++;
            pl_in += sxy;
            slot_i = slot_i + 1 == S ? 0 : slot_i + 1;
        };
#pragma unroll
        for (int q = 0; q < S - 2; q++) issue();

        V4<float> uc[NG];                   // own cell of plane q-1, per group
        float4 Rz_prev[NG], Rz_c[NG];       // right-going z halves of planes q-2 and q-1
#pragma unroll
        for (int k = 0; k < NG; k++) {
            uc[k] = V4<float>{0.0f, 0.0f, 0.0f, 0.0f};
            Rz_prev[k] = Rz_c[k] = float4{};
        }
        V4<float> *out = Og + (int64_t)z0 * sxy + (int64_t)y * nx + x;
        int slot = 0;
#pragma unroll 1
        for (int q = 0; q < L; q++) {
            cp_async_wait<S - 3>();
            __syncthreads();
            issue();
            const int hs = q & 1, cs = hs ^ 1;
            const bool zneg = (q == 0 && zneg_first) || (q == L - 1 && zneg_last);
#pragma unroll
            for (int k = 0; k < NG; k++) {
                if (k >= ng) continue;        // (the same in every thread)
                V4<float> un = {};
                float4 Rz_n = {}, Lz_n = {};
                if (act) {
                    un = sm.U[slot][k][ty + 1][tx + 1];
                    if (zneg) un.w = -un.w;
                    Halves hv;
                    cell_halves(un, hv);
                    Rz_n = hv.R[2];
                    Lz_n = hv.L[2];
                    sm.H[hs][k][0][ty + 1][tx + 1] = hv.R[0];
                    sm.H[hs][k][1][ty + 1][tx + 1] = hv.L[0];
                    sm.H[hs][k][2][ty + 1][tx + 1] = hv.R[1];
                    sm.H[hs][k][3][ty + 1][tx + 1] = hv.L[1];
                }
                if (hx >= 0) {
                    V4<float> h = sm.U[slot][k][hy][hx];
                    if (zneg) h.w = -h.w;
                    if (hneg == 1) h.y = -h.y;
                    else if (hneg == 2) h.z = -h.z;
                    Halves hv;
                    cell_halves(h, hv);
                    sm.H[hs][k][hk][hy][hx] = hk == 0 ? hv.R[0] : hk == 1 ? hv.L[0] : hk == 2 ? hv.R[1] : hv.L[1];
                }
                if (act && q >= 2) {
                    // update plane c = q - 1 (z = z0 + q - 2) of group g0 + k
                    const float4 l = sm.H[cs][k][0][ty + 1][tx];        // Rx of the left cell
                    const float4 r = sm.H[cs][k][1][ty + 1][tx + 2];    // Lx of the right cell
                    const float4 d = sm.H[cs][k][2][ty][tx + 1];        // Ry of the cell below
                    const float4 p = sm.H[cs][k][3][ty + 2][tx + 1];    // Ly of the cell above
                    const float4 Rzp = Rz_prev[k];
                    const float2 slo = __fadd2_rn(__fadd2_rn(__fadd2_rn(lo2(l), lo2(r)), __fadd2_rn(lo2(d), lo2(p))),
                                                  __fadd2_rn(lo2(Rzp), lo2(Lz_n)));
                    const float2 shi = __fadd2_rn(__fadd2_rn(__fadd2_rn(hi2(l), hi2(r)), __fadd2_rn(hi2(d), hi2(p))),
                                                  __fadd2_rn(hi2(Rzp), hi2(Lz_n)));
                    const float2 cc0 = make_float2(c0, c0), cc1 = make_float2(c1, c1);
                    const float2 olo = __ffma2_rn(cc0, make_float2(uc[k].x, uc[k].y), __fmul2_rn(cc1, slo));
                    const float2 ohi = __ffma2_rn(cc0, make_float2(uc[k].z, uc[k].w), __fmul2_rn(cc1, shi));
                    st4(out + k * gst, V4<float>{olo.x, olo.y, ohi.x, ohi.y});
                }
                Rz_prev[k] = Rz_c[k];
                Rz_c[k] = Rz_n;
                uc[k] = un;
            }
            if (act && q >= 2) out += sxy;
            slot = slot + 1 == S ? 0 : slot + 1;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}

// ---------------------------------------------- FP32 HLL transport
// Both signal speeds of a state along one axis from the paired table: entry
// (i, j), j < NM, holds the pairs (lambda_min, lambda_max) at mu_j and
// mu_{j+1}, f = 1 - (i/NF)^2, mu_j = -1 + 2j/NM, with lambda_min(f, mu) =
// -lambda_max(f, -mu) stored beside lambda_max; the bilinear form of
// hll_lookup on both at once, two 16-byte loads.  The row part (i, tx)
// depends on f only and is shared by the three axes.
__device__ __forceinline__ float2 hll_pair(const float4 *__restrict__ tab, int i, float tx, float mu)
{
    const float y = (mu + 1.0f) * (0.5f * (float)RTD_HLL_NM);
    int j = (int)y;
    j = j > RTD_HLL_NM - 1 ? RTD_HLL_NM - 1 : (j < 0 ? 0 : j);
    const float ty = y - (float)j;
    const float4 r0 = __ldg(tab + i * RTD_HLL_NM + j), r1 = __ldg(tab + (i + 1) * RTD_HLL_NM + j);
    const float2 v00 = lo2(r0), v01 = hi2(r0), v10 = lo2(r1), v11 = hi2(r1);
    const float2 wx1 = make_float2(tx, tx), wx0 = make_float2(1.0f - tx, 1.0f - tx);
    const float2 wy1 = make_float2(ty, ty), wy0 = make_float2(1.0f - ty, 1.0f - ty);
    const float2 a = __ffma2_rn(v10, wx1, __fmul2_rn(v00, wx0));
    const float2 b = __ffma2_rn(v11, wx1, __fmul2_rn(v01, wx0));
    return __ffma2_rn(b, wy1, __fmul2_rn(a, wy0));
}

// a - b on a pair (b * -1 is exact, so the fused form rounds once, as a - b)
__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// HLL flux between (UL, GL) with speeds sL = (min, max) and (UR, GR), sR, as
// Phi = al G_L + be G_R + ka (U_R - U_L) with al = l+/(l+ - l-), be =
// -l-/(l+ - l-), ka = l+ l-/(l+ - l-) (the form of hll()); no wave across
// the face gives al = be = 1/2, ka = 0, the mean of the two fluxes
__device__ __forceinline__ float4 hll_face(const float4 &UL, const float4 &GL, float2 sL, const float4 &UR,
                                           const float4 &GR, float2 sR)
{
    const float lp = fmaxf(fmaxf(sL.y, sR.y), 0.0f), lm = fminf(fminf(sL.x, sR.x), 0.0f);
    const float den = lp - lm;
    float al = 0.5f, be = 0.5f, ka = 0.0f;
    if (den > 0.0f) {
        const float r = rcp_approx(den);
        al = lp * r;
        be = -lm * r;
        ka = (lp * lm) * r;
    }
    const float2 A = make_float2(al, al), Bv = make_float2(be, be), K = make_float2(ka, ka);
    const float2 dlo = fsub2(lo2(UR), lo2(UL)), dhi = fsub2(hi2(UR), hi2(UL));
    const float2 plo = __ffma2_rn(K, dlo, __ffma2_rn(Bv, lo2(GR), __fmul2_rn(A, lo2(GL))));
    const float2 phi = __ffma2_rn(K, dhi, __ffma2_rn(Bv, hi2(GR), __fmul2_rn(A, hi2(GL))));
    return f4(plo, phi);
}

// closure, flux vectors G_d = (F_d, P_d.) and speeds of one cell (the FP32
// fast forms of closure() and hll_fz(); mu = F_d/|F|, 0 for F = 0).  ALL:
// the speeds along x, y, z; otherwise along axis ax (0 = x, 1 = y) only,
// in s[0]
struct HllCell {
    float4 G[3];
    float2 s[3];
};

template <bool ALL>
__device__ __forceinline__ void hll_cell(const float4 *__restrict__ tab, const V4<float> &u, int ax, HllCell &c)
{
    float P[6];
    closure<float, false>(u, P);
    c.G[0] = make_float4(u.y, P[0], P[1], P[2]);
    c.G[1] = make_float4(u.z, P[1], P[3], P[4]);
    c.G[2] = make_float4(u.w, P[2], P[4], P[5]);
    float Fn, z;
    hll_fz<float, false>(u, Fn, z);
    const float x = z * (float)RTD_HLL_NF;
    int i = (int)x;
    i = i > RTD_HLL_NF - 1 ? RTD_HLL_NF - 1 : (i < 0 ? 0 : i);
    const float tx = x - (float)i;
    const float rF = Fn > 0.0f ? rcp_approx(Fn) : 0.0f;
    if (ALL) {
        c.s[0] = hll_pair(tab, i, tx, u.y * rF);
        c.s[1] = hll_pair(tab, i, tx, u.z * rF);
        c.s[2] = hll_pair(tab, i, tx, u.w * rF);
    } else {
        c.s[0] = hll_pair(tab, i, tx, (ax == 0 ? u.y : u.z) * rF);
    }
}

template <int TX, int TY>
struct TransportSmemHLL {              // rows padded by one cell, as in k_transport_pm
    V4<float> U[TP_STAGES][TY + 2][TX + 3];
    float4 Gx[2][TY + 2][TX + 3];      // G_x of two planes
    float4 Gy[2][TY + 2][TX + 3];      // G_y of two planes
    float2 Sx[2][TY + 2][TX + 3];      // (min, max) speeds along x of two planes
    float2 Sy[2][TY + 2][TX + 3];      // along y
};

template <int TX, int TY>
constexpr size_t transport_hll_smem_bytes() { return sizeof(TransportSmemHLL<TX, TY>); }

// FP32 transport with the HLL flux.  Pipeline, work split and halos of
// k_transport_pm; each cell's closure, flux vectors and speeds are evaluated
// once per plane, the x/y ones shared through shared memory, the z ones kept
// in registers, and the z-face flux carried from plane to plane.  Halo cells
// evaluate the one axis their face needs; reflective halos keep their
// negated state in shared memory (the flux reads U of both sides).  After the
// update |F| <= N is restored as in k_transport.  The block holds one thread
// per interior and per halo column (the layout of k_transport_pm), so every
// thread evaluates one cell per plane.
template <int TX, int TY>
__global__ void __launch_bounds__(transport_pm_threads<TX, TY>(), 2)
k_transport_hll(const BoxDev *__restrict__ boxes, int nboxes, int64_t nunits, int, Phys ph, Ctl *ctl)
{
    constexpr int S = TP_STAGES;
    extern __shared__ __align__(16) unsigned char tp_smem_raw[];
    TransportSmemHLL<TX, TY> &sm = *reinterpret_cast<TransportSmemHLL<TX, TY> *>(tp_smem_raw);
    const float4 *__restrict__ tab = ph.hll_f4;

    const int tid = threadIdx.x;
    const bool interior = tid < TX * TY;
    const int tx = interior ? tid % TX : 0, ty = interior ? tid / TX : 0;
    if (blockIdx.x == 0 && tid == 0) ctl->step += 1;

    const int64_t ubeg = nunits * (int64_t)blockIdx.x / gridDim.x;
    const int64_t uend = nunits * (int64_t)(blockIdx.x + 1) / gridDim.x;
    for (int64_t u = ubeg; u < uend;) {
        const int b = find_box_unit(boxes, nboxes, u);
        const BoxDev &B = boxes[b];
        const int nx = B.nx, ny = B.ny, nz = B.nz;
        int g, iy, ix, z0, z1;
        transport_run(B, u - B.titem0, uend - u, g, iy, ix, z0, z1);
        u += z1 - z0;
        const int x0 = ix * TX, y0 = iy * TY;
        const int ntx = min(TX, nx - x0), nty = min(TY, ny - y0);
        const int x = x0 + tx, y = y0 + ty;
        const bool act = interior && (tx < ntx) && (ty < nty);
        const int L = (z1 - z0) + 2;
        const V4<float> *Ug = reinterpret_cast<const V4<float> *>(B.U) + (int64_t)g * B.ncell;
        V4<float> *Og = reinterpret_cast<V4<float> *>(B.Us) + (int64_t)g * B.ncell;
        const float lam = (float)B.lam;
        const int64_t sxy = (int64_t)nx * ny;

        // halo cell of this thread: 0 = left column, 1 = right, 2 = bottom
        // row, 3 = top (its x or y face only)
        int hx = -1, hy = -1, sx = 0, sy = 0, hneg = 0, hk = 0;
        float hin = 0.0f;
        bool hif = false;
        if (!interior) {
            int t = tid - TX * TY;
            if (t < nty) {
                hx = 0; hy = t + 1; sy = y0 + t; sx = x0 - 1; hk = 0;
                if (sx < 0) {
                    if (ph.bc[0] == 0) sx = nx - 1;
                    else { sx = 0; hneg = ph.bc[0] == 2 ? 1 : 0; }
                    if (ph.bc[0] == 3) { hif = true; hin = (float)(ph.inflow_c[0][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < nty) {
                hx = ntx + 1; hy = t + 1; sy = y0 + t; sx = x0 + ntx; hk = 1;
                if (sx >= nx) {
                    if (ph.bc[1] == 0) sx = 0;
                    else { sx = nx - 1; hneg = ph.bc[1] == 2 ? 1 : 0; }
                    if (ph.bc[1] == 3) { hif = true; hin = -(float)(ph.inflow_c[1][g] * B.inv_nunit); }
                }
            } else if ((t -= nty) < ntx) {
                hx = t + 1; hy = 0; sx = x0 + t; sy = y0 - 1; hk = 2;
                if (sy < 0) { if (ph.bc[2] == 0) sy = ny - 1; else { sy = 0; hneg = ph.bc[2] == 2 ? 2 : 0; } }
            } else if ((t -= ntx) < ntx) {
                hx = t + 1; hy = nty + 1; sx = x0 + t; sy = y0 + nty; hk = 3;
                if (sy >= ny) { if (ph.bc[3] == 0) sy = 0; else { sy = ny - 1; hneg = ph.bc[3] == 2 ? 2 : 0; } }
            }
        }
        const V4<float> *gown = Ug + (int64_t)y * nx + x;
        const V4<float> *ghalo = Ug + (int64_t)sy * nx + sx;
        const bool zneg_first = z0 == 0 && ph.bc[4] == 2, zneg_last = z1 == nz && ph.bc[5] == 2;
        int zi = z0 - 1;
        int slot_i = 0;
        int64_t pl_in = (int64_t)zi * sxy;       // plane zi's offset, and the ghost planes'
        const int64_t pl_lo = ph.bc[4] == 0 ? (int64_t)(nz - 1) * sxy : 0;
        const int64_t pl_hi = ph.bc[5] == 0 ? 0 : (int64_t)(nz - 1) * sxy;
        auto issue = [&]() {
            if (zi < z1 + 1) {
                const int64_t pl = zi < 0 ? pl_lo : (zi >= nz ? pl_hi : pl_in);
                if (act) cp_async16(&sm.U[slot_i][ty + 1][tx + 1], gown + pl);
                if (hx >= 0) {
                    if (hif) sm.U[slot_i][hy][hx] = V4<float>{fabsf(hin), hin, 0.0f, 0.0f};
                    else cp_async16(&sm.U[slot_i][hy][hx], ghalo + pl);
                }
            }
            cp_async_commit();
            zi++;
            pl_in += sxy;
            slot_i = slot_i + 1 == S ? 0 : slot_i + 1;
        };
#pragma unroll
        for (int q = 0; q < S - 2; q++) issue();

        float4 uc = {}, Gzc = {}, Fzm = {};   // plane q-1: state, G_z; flux of its lower z face
        float2 szc = {};                      // its z speeds
        V4<float> *out = Og + (int64_t)z0 * sxy + (int64_t)y * nx + x;
        int slot = 0, slot_c = S - 1;         // ring slots of planes q and q-1
#pragma unroll 2
        for (int q = 0; q < L; q++) {
            cp_async_wait<S - 3>();
            __syncthreads();
            issue();
            const int hs = q & 1;
            const bool zneg = (q == 0 && zneg_first) || (q == L - 1 && zneg_last);
            float4 un = {}, Gzn = {};
            float2 szn = {};
            if (act) {
                V4<float> v = sm.U[slot][ty + 1][tx + 1];
                if (zneg) v.w = -v.w;
                HllCell hc;
                hll_cell<true>(tab, v, 0, hc);
                sm.Gx[hs][ty + 1][tx + 1] = hc.G[0];
                sm.Gy[hs][ty + 1][tx + 1] = hc.G[1];
                sm.Sx[hs][ty + 1][tx + 1] = hc.s[0];
                sm.Sy[hs][ty + 1][tx + 1] = hc.s[1];
                un = make_float4(v.x, v.y, v.z, v.w);
                Gzn = hc.G[2];
                szn = hc.s[2];
            }
            if (hx >= 0) {
                V4<float> &hr = sm.U[slot][hy][hx];
                V4<float> h = hr;
                if (zneg) h.w = -h.w;
                if (hneg == 1) h.y = -h.y;
                else if (hneg == 2) h.z = -h.z;
                if (hneg) hr = h;
                const int ax = hk >> 1;
                HllCell hc;
                hll_cell<false>(tab, h, ax, hc);
                if (ax == 0) {
                    sm.Gx[hs][hy][hx] = hc.G[0];
                    sm.Sx[hs][hy][hx] = hc.s[0];
                } else {
                    sm.Gy[hs][hy][hx] = hc.G[1];
                    sm.Sy[hs][hy][hx] = hc.s[0];
                }
            }
            if (act && q >= 1) {
                const float4 Fzp = hll_face(uc, Gzc, szc, un, Gzn, szn);
                if (q >= 2) {
                    // update plane c = q - 1 (z = z0 + q - 2)
                    const int cs = hs ^ 1;
                    const float4 Gxc = sm.Gx[cs][ty + 1][tx + 1], Gyc = sm.Gy[cs][ty + 1][tx + 1];
                    const float2 sxc = sm.Sx[cs][ty + 1][tx + 1], syc = sm.Sy[cs][ty + 1][tx + 1];
                    float4 Fxm, Fxp, Fym, Fyp;
                    {
                        const V4<float> v = sm.U[slot_c][ty + 1][tx];
                        const float2 s = sm.Sx[cs][ty + 1][tx];
                        Fxm = hll_face(make_float4(v.x, v.y, v.z, v.w), sm.Gx[cs][ty + 1][tx], s, uc, Gxc, sxc);
                    }
                    {
                        const V4<float> v = sm.U[slot_c][ty + 1][tx + 2];
                        const float2 s = sm.Sx[cs][ty + 1][tx + 2];
                        Fxp = hll_face(uc, Gxc, sxc, make_float4(v.x, v.y, v.z, v.w), sm.Gx[cs][ty + 1][tx + 2], s);
                    }
                    {
                        const V4<float> v = sm.U[slot_c][ty][tx + 1];
                        const float2 s = sm.Sy[cs][ty][tx + 1];
                        Fym = hll_face(make_float4(v.x, v.y, v.z, v.w), sm.Gy[cs][ty][tx + 1], s, uc, Gyc, syc);
                    }
                    {
                        const V4<float> v = sm.U[slot_c][ty + 2][tx + 1];
                        const float2 s = sm.Sy[cs][ty + 2][tx + 1];
                        Fyp = hll_face(uc, Gyc, syc, make_float4(v.x, v.y, v.z, v.w), sm.Gy[cs][ty + 2][tx + 1], s);
                    }
                    const float2 L2 = make_float2(-lam, -lam);
                    const float2 dlo = __fadd2_rn(__fadd2_rn(fsub2(lo2(Fxp), lo2(Fxm)), fsub2(lo2(Fyp), lo2(Fym))),
                                                  fsub2(lo2(Fzp), lo2(Fzm)));
                    const float2 dhi = __fadd2_rn(__fadd2_rn(fsub2(hi2(Fxp), hi2(Fxm)), fsub2(hi2(Fyp), hi2(Fym))),
                                                  fsub2(hi2(Fzp), hi2(Fzm)));
                    const float2 olo = __ffma2_rn(L2, dlo, lo2(uc)), ohi = __ffma2_rn(L2, dhi, hi2(uc));
                    float o0 = olo.x, o1 = olo.y, o2 = ohi.x, o3 = ohi.y;
                    const float Fn = fsqrt<float, false>(o1 * o1 + o2 * o2 + o3 * o3);
                    if (Fn > o0) {
                        const float r = o0 > 0.0f ? o0 * rcp_approx(Fn) : 0.0f;
                        o1 *= r;
                        o2 *= r;
                        o3 *= r;
                    }
                    st4(out, V4<float>{o0, o1, o2, o3});
                    out += sxy;
                }
                Fzm = Fzp;
            }
            uc = un;
            Gzc = Gzn;
            szc = szn;
            slot_c = slot;
            slot = slot + 1 == S ? 0 : slot + 1;
        }
        cp_async_wait<0>();
        __syncthreads();
    }
}
#endif  // RTK_SKIP_SINGLE_KERNELS

// ------------------------------------------------------------- rates
// Temperature fits (cgs).  Recombination, collisional ionisation and
// recombination cooling: Hui & Gnedin (1997) fits in lambda = 2 T_HI / T;
// collisional excitation cooling exp(-118348/T)/(1 + sqrt(T/1e5)) (Cen 1992);
// bremsstrahlung 1.42e-27 g_ff sqrt(T), g_ff = 1.3.  Written with one log of
// lambda and exp/log1p of it.
struct Rates {
    double aA, aB, beta;   // cm^3/s
    double kR;             // cooling per n_e n_HII: recombination + bremsstrahlung
    double kC;             // cooling per n_e n_HI: collisional ionisation + excitation
    float aB32;            // alpha_B in FP32 (the split form's recombination photons)
    float kC32;            // kC in FP32 (the fast forms' pre-test), formed where kC is
    float kR32;            // an upper bound of kR in FP32 (the fast forms' pre-test)
};

__device__ __forceinline__ Rates rates_at(const Phys &ph, double T)
{
    Rates r;
    if (ph.rates_const) {
        r.aA = ph.alphaA; r.aB = ph.alphaB; r.beta = ph.beta;
        r.kR = 0.0; r.kC = 0.0;
        r.aB32 = d2f(r.aB);
        r.kC32 = 0.0f;
        r.kR32 = 0.0f;
        return r;
    }
    const double l = 2.0 * rtd::T_HI / T;
    const double ll = log(l);
    // ln of the fit scales 0.522, 2.740, 0.354, 0.541, 2.250 (host-computed)
    const double L0522 = ph.lnfit[0], L2740 = ph.lnfit[1], L0354 = ph.lnfit[2],
                 L0541 = ph.lnfit[3], L2250 = ph.lnfit[4];
    r.aB = 2.753e-14 * exp(1.500 * ll - 2.242 * log1p(exp(0.407 * (ll - L2740))));
    r.aA = ph.ots ? r.aB
                  : 1.269e-13 * exp(1.503 * ll - 1.923 * log1p(exp(0.470 * (ll - L0522))));
    const double lnT = ph.ln2THI - ll;
    r.beta = 21.11 * exp(-1.5 * lnT - 0.5 * l - 1.089 * ll
                         - 1.101 * log1p(exp(0.874 * (ll - L0354))));
    const double crec = ph.ots
        ? 3.435e-30 * T * exp(1.970 * ll - 3.720 * log1p(exp(0.376 * (ll - L2250))))
        : 1.778e-29 * T * exp(1.965 * ll - 2.697 * log1p(exp(0.502 * (ll - L0541))));
    const double sT = sqrt(T);
    const double cff = 1.42e-27 * 1.3 * sT;
    const double cci = rtd::KB * rtd::T_HI * r.beta;
    const double cce = 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1.0e5));
    r.kR = crec + cff;
    r.kC = cci + cce;
    r.kC32 = d2f(r.kC);
    r.kR32 = d2f(r.kR);
    r.aB32 = d2f(r.aB);
    return r;
}

// Position of T in the rate tables (rate_table.cu): interval j and local
// variable t in [-1, 1), both from T's bits.  For T = 2^e (1 + m), m in
// [0, 1), j = 2^SUB (e - E0) + floor(2^SUB m) and y = 1 + frac(2^SUB m) in
// [1, 2) exactly; t = 2 y - 3 (exact), and t32 = the same with y's mantissa
// cut to float's 23 bits (exact in float; the FP32 tail needs ~1e-6 of t).
// Returns false outside [2^E0, 2^E1) (and for T <= 0, NaN, Inf).
__device__ __forceinline__ bool tab_pos(double T, int &j, double &t, float &t32)
{
    const long long bits = __double_as_longlong(T);
    const int e = (int)(bits >> 52) - 1023;
    if (e < RTD_TAB_E0 || e >= RTD_TAB_E1) return false;
    constexpr int low = 52 - RTD_TAB_SUB;
    j = ((e - RTD_TAB_E0) << RTD_TAB_SUB) + (int)((bits >> low) & ((1 << RTD_TAB_SUB) - 1));
    // y: the mantissa bits below the top SUB, moved up
    const long long ym = (bits & ((1ll << low) - 1)) << RTD_TAB_SUB;
    t = fma(2.0, __longlong_as_double(0x3FF0000000000000ll | ym), -3.0);
    t32 = fmaf(2.0f, __int_as_float(0x3F800000 | (int)(ym >> 29)), -3.0f);
    return true;
}

// p(t) = c0 + t (c1 + t (c2 + t q)) with the tail q = c3 + t (c4 + t c5) in FP32
__device__ __forceinline__ double tab_eval(const RateCoef *c, double t, float t32)
{
    const float q = fmaf(fmaf(__ldg(&c->c5), t32, __ldg(&c->c4)), t32, __ldg(&c->c3));
    return fma(fma(fma(f2d(q), t, __ldg(&c->c2)), t, __ldg(&c->c1)), t, __ldg(&c->c0));
}

// The same rates from the tables built at set-up (rate_table.cu): degree-5
// Chebyshev interpolants on 64 intervals of T per binade, accurate to ~3e-14
// relative; beta and the excitation cooling keep their exp(-c/T) factor
// exact, and below RTD_TAB_TCUT, where both factors are exactly zero in
// double, they are not evaluated.  Outside 1 K .. 2^30 K the fits are
// evaluated directly.
// warm: the cut is RTD_TAB_TWARM (the cell's n0 dtau allows it: below it the
// two factors' terms are below 2^-60 of what they enter), else RTD_TAB_TCUT
template <bool STRICT>
__device__ __forceinline__ Rates rates_tab(const Phys &ph, const RateCoef *tab, double T,
                                           bool warm = false, bool b32 = false)
{
    int j;
    double t;
    float t32;
    if (!tab_pos(T, j, t, t32)) return rates_at(ph, T);
    const RateCoef *a = tab + (size_t)j * RTD_TAB_NF;
    Rates r;
    if (b32) {
        // alpha_B only for the FP32 recombination photons (no OTS): its
        // polynomial in FP32, the FP64 value not formed
        const float q = fmaf(fmaf(__ldg(&a[1].c5), t32, __ldg(&a[1].c4)), t32, __ldg(&a[1].c3));
        r.aB32 = fmaf(fmaf(fmaf(q, t32, __ldg(&a[2].b32)), t32, __ldg(&a[1].b32)), t32, __ldg(&a[0].b32));
        r.aB = 0.0;
    } else {
        r.aB = tab_eval(a + 1, t, t32);
        r.aB32 = 0.0f;
    }
    r.aA = ph.ots ? r.aB : tab_eval(a, t, t32);
    r.kR = tab_eval(a + 2, t, t32);
    r.kR32 = __ldg(&a[3].b32);                 // bound over the interval (no conversion)
    if (dbits(T) >= (warm ? dbits(RTD_TAB_TWARM) : dbits(RTD_TAB_TCUT))) {   // T >= cut (both positive)
        const double invT = STRICT ? 1.0 / T : rcp_nr(T);
        const double ab = tab_eval(a + 3, t, t32) - rtd::T_HI * invT;
        const double ac = tab_eval(a + 4, t, t32) - 118348.0 * invT;
        r.beta = STRICT ? exp(ab) : exp_tab(ab, ph.e2t);
        const double cce = STRICT ? exp(ac) : exp_tab(ac, ph.e2t);
        r.kC = rtd::KB * rtd::T_HI * r.beta + cce;
        r.kC32 = d2f(r.kC);
    } else {
        r.beta = 0.0;
        r.kC = 0.0;
        r.kC32 = 0.0f;
    }
    return r;
}

// cooling Lambda(n0, x, T) of Eq. e:therm4, erg/cm^3/s
__device__ __forceinline__ double cooling(const Rates &r, double n0, double xHI)
{
    const double x = 1.0 - xHI;
    const double ne = x * n0, nHII = x * n0, nHI = xHI * n0;
    return ne * nHII * r.kR + ne * nHI * r.kC;
}

// e = (3/2)(1 + x) n0 kB T  (pure hydrogen, gamma = 5/3)
__device__ __forceinline__ double eint(double xHI, double n0, double T)
{
    return 1.5 * (1.0 + (1.0 - xHI)) * n0 * rtd::KB * T;
}

// ------------------------------------------------------------- chemistry
template <int G>
struct Cell {
    double N[G], F[G][3];
    double xHI, T;
    float n32[G];       // N in FP32 where the photon update runs in FP32 (N == n32 then)
};

// one trial of length dtau from s into o, in the paper's order
// N -> F -> x -> e (Sec. 2.2.4 semi-implicit update; dtau restored in the
// absorption denominators); returns e^p and e^{p+1}
template <int G, bool STRICT>
__device__ __forceinline__ void chem_trial(const Phys &ph, double nunit, double inu, double n0,
                                           const double *S, const Rates &r, double alpha,
                                           const Cell<G> &s, double dtau, Cell<G> &o, double &ep,
                                           double &e1)
{
    // STRICT: the oracle's operations in its order (IEEE division); the fast
    // forms multiply by 1/nunit (inu) and by Newton reciprocals instead
    const double x = 1.0 - s.xHI;
#pragma unroll
    for (int i = 0; i < G; i++) {
        const double den = 1.0 + ph.csig[i] * s.xHI * n0 * dtau;
        double src = S[i];
        if (i == 0 && !ph.ots)
            src = STRICT ? src + (r.aA - r.aB) * x * x * n0 * n0 / nunit
                         : src + (r.aA - r.aB) * x * x * n0 * n0 * inu;
        if (STRICT) {
            o.N[i] = (s.N[i] + src * dtau) / den;
#pragma unroll
            for (int k = 0; k < 3; k++) o.F[i][k] = s.F[i][k] / den;
        } else {
            const double rd = rcp_nr(den);
            o.N[i] = (s.N[i] + src * dtau) * rd;
#pragma unroll
            for (int k = 0; k < 3; k++) o.F[i][k] = s.F[i][k] * rd;
        }
    }
    double gam = 0.0;
#pragma unroll
    for (int i = 0; i < G; i++) gam = gam + ph.csig[i] * (nunit * o.N[i]);
    const double xnum = s.xHI + alpha * x * x * n0 * dtau;
    const double xden = 1.0 + dtau * (r.beta * x * n0 + gam);
    o.xHI = STRICT ? xnum / xden : xnum * rcp_nr(xden);
    const double e0 = eint(s.xHI, n0, s.T);
    ep = e0;
    if (ph.isothermal) {
        o.T = s.T;
        e1 = e0;
        return;
    }
    double heat = 0.0;
#pragma unroll
    for (int i = 0; i < G; i++) heat = heat + ph.c * o.xHI * n0 * (nunit * o.N[i]) * ph.SigE[i];
    const double lamc = cooling(r, n0, o.xHI);   // Lambda(n0, x^{p+1}, T^p)
    const double e = e0 + dtau * heat - dtau * lamc;
    e1 = e;
    const double cv = 1.5 * (1.0 + (1.0 - o.xHI)) * n0 * rtd::KB;
    o.T = STRICT ? e / cv : e * rcp_nr(cv);
}

// advance one cell over `span` with sub-cycles: dtau = min(rest,
// |e/(H - Lambda)|) when use_est (adaptive), halved while the energy changes
// by more than 10% (Sec. 2.2.4, after Rosdahl et al. 2013)
// no-op recorder of accepted trials (the adjoint passes one that stores them)
struct NoTrace {
    template <int G>
    __device__ __forceinline__ void push(const Cell<G> &, double) {}
};

// One trial of the fast forms: the same update as chem_trial, regrouped
// around per-cell constants so the FP64 pipe does less work (products with
// n0 and nunit formed once per cell; Newton reciprocals).  Agrees with
// chem_trial to a few ulp.
template <int G>
struct CellK {
    double n02, K, cvn; // n0^2, n0^2 / nunit (without OTS), (3/2) kB n0
    double cvn2;        // 3 kB n0
    float n0f, S32[G];  // n0 and the source terms in FP32 (FP32 photon update)
    float K32;          // K in FP32
};

// the per-cell constants of the fast forms from n0 (k_cconst, supercomoving
// units, the fine level): the operations chem_span used to form per call
__device__ __forceinline__ CellConst cell_const(const Phys &ph, const BoxDev &B, double n0)
{
    CellConst c;
    c.n0 = n0;
    c.n02 = n0 * n0;
    c.K = ph.ots ? 0.0 : c.n02 * B.inv_nunit;
    c.cvn = (1.5 * rtd::KB) * n0;
    c.cvn2 = 2.0 * c.cvn;
    c.K32 = d2f(c.K);
    c.pad = 0.0f;
    return c;
}

// DEFER: F is not carried through the trial (nothing in the chemistry reads
// it; it only scales by 1/den), the scale of each group goes to rd[] instead.
// N32 (split form): the photon update of a5, N <- (N + S dtau)/(1 + c
// sigma_N,i x_HI n0 dtau) and the scale of F, runs in FP32, the precision
// N and F are stored in; x_HI, T, the rates and the photoionisation,
// heating and cooling sums stay FP64
// rec32 (N32 only): the recombination photons of group 1 per unit time in
// FP32, (alpha_A - alpha_B) x^2 n0^2 / nunit, formed once per sub-cycle (it
// depends on the sub-cycle's start state only); xh32: x_HI in FP32; dt32:
// dtau in FP32
template <int G, bool DEFER, bool N32, typename FT>
__device__ __forceinline__ void chem_trial_fast(const Phys &ph, const BoxDev &B, const CellK<G> &k,
                                                double n0, const double *S, const Rates &r,
                                                double alpha, const Cell<G> &s, double e0,
                                                double dtau, Cell<G> &o, double &e1, FT *rdo,
                                                float rec32, float xh32, float dt32)
{
    const double x = 1.0 - s.xHI;
    if constexpr (N32) {
        const float q32 = (xh32 * k.n0f) * dt32;
#pragma unroll
        for (int i = 0; i < G; i++) {
            const float rd = __frcp_rn(fmaf(ph.csig_f[i], q32, 1.0f));
            const float src = (i == 0 && !ph.ots) ? k.S32[i] + rec32 : k.S32[i];
            const float n = fmaf(src, dt32, s.n32[i]) * rd;
            o.n32[i] = n;
            o.N[i] = f2d(n);
            rdo[i] = rd;
        }
    } else {
        const double q = s.xHI * n0 * dtau;
        const double rec = ph.ots ? 0.0 : (r.aA - r.aB) * x * x * k.K;
#pragma unroll
        for (int i = 0; i < G; i++) {
            const double rd = rcp_nr(fma(ph.csig[i], q, 1.0));
            const double src = (i == 0 && !ph.ots) ? S[i] + rec : S[i];
            o.N[i] = fma(src, dtau, s.N[i]) * rd;
            if (DEFER) {
                rdo[i] = rd;
            } else {
#pragma unroll
                for (int m = 0; m < 3; m++) o.F[i][m] = s.F[i][m] * rd;
            }
        }
    }
    double gam = B.gN[0] * o.N[0];
#pragma unroll
    for (int i = 1; i < G; i++) gam = fma(B.gN[i], o.N[i], gam);
    const double xnum = fma(alpha * x * x, n0 * dtau, s.xHI);
    // one formula for every cell: in cold gas beta = kC = 0 exactly and the
    // collisional terms add exact zeros (a per-cell choice of the shorter
    // form ran both forms in every warp)
    const double xden = fma(dtau, fma(r.beta * x, n0, gam), 1.0);
    o.xHI = xnum * rcp_nr(xden);
    if (ph.isothermal) {
        o.T = s.T;
        e1 = e0;
        return;
    }
    double hs = B.hN[0] * o.N[0];            // heating per neutral atom / n0
#pragma unroll
    for (int i = 1; i < G; i++) hs = fma(B.hN[i], o.N[i], hs);
    const double x1 = 1.0 - o.xHI;
    // Lambda(n0, x^{p+1}, T^p)
    const double cool = k.n02 * x1 * fma(x1, r.kR, o.xHI * r.kC);
    e1 = fma(dtau, fma(o.xHI * n0, hs, -cool), e0);
    o.T = e1 * rcp_nr(fma(-k.cvn, o.xHI, k.cvn2));    // (3/2) kB n0 (2 - x_HI)
}

// fac (fast forms without a trace): F is left alone and each group's scale
// over the accepted trials is multiplied into fac[i] (the caller starts it
// at 1 and applies it to F); otherwise F is updated in s and fac unused.
// s <- o; F only when it is carried through the trials
template <int G, bool F_TOO, bool N32 = false>
__device__ __forceinline__ void take(Cell<G> &s, const Cell<G> &o)
{
#pragma unroll
    for (int i = 0; i < G; i++) {
        s.N[i] = o.N[i];
        if (N32) s.n32[i] = o.n32[i];
        if (F_TOO) {
#pragma unroll
            for (int m = 0; m < 3; m++) s.F[i][m] = o.F[i][m];
        }
    }
    s.xHI = o.xHI;
    s.T = o.T;
}

// warm_cut (fast forms): n0 dtau <= RTD_TAB_NDMAX for every dtau of the span,
// so the rates may take the RTD_TAB_TWARM cut
// in32 (FP32 photon update only, required there): the caller's FP32 copies,
// in32[0] = n0 and in32[1 + i] = S_i, with s.n32 holding N in FP32 and s.N
// its exact double.  Every float <-> double conversion costs FP64-pipe
// issue slots (its rare-case instruction is issued, predicated, with the
// warp), so values that arrive in FP32 are not converted back and forth.
// span32 (fast forms): span in FP32, required with the FP32 photon update
// (its dtau); elsewhere a negative value means unknown, and the pre-test
// then never decides (the FP64 test does).  kc (fast forms without a trace,
// required there): the cell's constants from n0 (cell_const).
template <int G, bool STRICT, class Trace = NoTrace, typename FT = double>
__device__ unsigned int chem_span(const Phys &ph, const RateCoef *tab, const BoxDev &B, double n0,
                                  const double *S, Cell<G> &s, double span, bool use_est,
                                  int &ncyc, Trace *tr = nullptr, FT *fac = nullptr,
                                  bool warm_cut = false, const float *in32 = nullptr,
                                  float span32 = -1.0f, const CellConst *kc = nullptr)
{
    constexpr bool DEFER = !STRICT && std::is_same<Trace, NoTrace>::value;
    constexpr bool N32 = DEFER && std::is_same<FT, float>::value;
    unsigned int err = 0;
    double tau = 0.0;
    CellK<G> k;
    if constexpr (DEFER) {                      // the caller's per-cell constants
        k.n02 = kc->n02;
        k.K = kc->K;
        k.cvn = kc->cvn;
        k.cvn2 = kc->cvn2;
    } else if (!STRICT) {
        k.n02 = n0 * n0;
        k.K = ph.ots ? 0.0 : k.n02 * B.inv_nunit;
        k.cvn = (1.5 * rtd::KB) * n0;
        k.cvn2 = 2.0 * k.cvn;
    }
    if constexpr (N32) {
        k.n0f = in32[0];
        k.K32 = kc->K32;
#pragma unroll
        for (int i = 0; i < G; i++) k.S32[i] = in32[1 + i];
    } else if (!STRICT) {
        k.n0f = d2f(n0);
    }
    double rem = span;                          // span - tau, tau = 0 in the first sub-cycle
    float rem32 = span32;                       // rem in FP32 (fast forms)
    for (;;) {
        const Rates r = tab ? rates_tab<STRICT>(ph, tab, s.T, !STRICT && warm_cut, N32 && !ph.ots)
                            : rates_at(ph, s.T);
        const double alpha = ph.ots ? r.aB : r.aA;
        double dtau = rem;
        // dtau in FP32 (the FP32 photon update): rem32, halved exactly with
        // dtau (both stay far above FP32's normal range)
        float dt32 = rem32;
        bool last = true;
        // e^p (the fast forms reuse it in every trial of this sub-cycle)
        const double ep0 = STRICT ? 0.0 : fma(-k.cvn, s.xHI, k.cvn2) * s.T;
        // x_HI and 1 - x_HI in FP32, once per sub-cycle (the pre-test, the
        // FP32 photon update and the recombination photons)
        const float xh32 = STRICT ? 0.0f : d2f(s.xHI);
        const float xl32 = STRICT ? 0.0f : d2f(1.0 - s.xHI);
        // FP32 pre-test of the estimate's skip (fast forms).  heat and
        // cooling are >= 0, so |rate| <= heat + cool, and q = rem (heat +
        // cool) / e is a sum of products of non-negative FP32 numbers in which
        // n0 and kB cancel (each a few ulp; an underflowed term is below any
        // part of q that matters; kR enters as an upper bound over its table
        // interval, which only raises q); 1 - x_HI comes from its FP64 value.  q <=
        // 0.999 therefore implies |e| >= rem |rate| (1 + 1e-13), the skip the
        // FP64 test below takes, which is then not evaluated: the decisions,
        // and the results, are those of the FP64 test
        bool pre_skip = false;
        if (!STRICT && !ph.isothermal && use_est) {
            const float xh = fabsf(xh32), xl = fabsf(xl32);
            float hsum = 0.0f;
#pragma unroll
            for (int i = 0; i < G; i++) hsum = fmaf(ph.hK[i], fabsf(N32 ? s.n32[i] : d2f(s.N[i])), hsum);
            constexpr float KB15I = (float)(1.0 / (1.5 * rtd::KB));
            const float kr = fabsf(r.kR32) * KB15I, kc = fabsf(r.kC32) * KB15I;
            const float cool = (k.n0f * xl) * fmaf(xl, kr, xh * kc);
            const float q = (rem32 * fmaf(xh * B.nunit_f, hsum, cool)) *
                            __frcp_rn((2.0f - xh) * d2f(s.T));
            pre_skip = q >= 0.0f && q <= 0.999f;
        }
        if (!ph.isothermal && use_est && !pre_skip) {
            double rate, e;
            if (STRICT) {
                double heat = 0.0;
#pragma unroll
                for (int i = 0; i < G; i++)
                    heat = heat + ph.c * s.xHI * n0 * (B.nunit * s.N[i]) * ph.SigE[i];
                rate = heat - cooling(r, n0, s.xHI);
                e = eint(s.xHI, n0, s.T);
            } else {
                // N32: s.N is formed by the trials; here N from its FP32 copy
                double hs = B.hN[0] * (N32 ? f2d(s.n32[0]) : s.N[0]);
#pragma unroll
                for (int i = 1; i < G; i++) hs = fma(B.hN[i], N32 ? f2d(s.n32[i]) : s.N[i], hs);
                hs = hs * n0;
                const double x = 1.0 - s.xHI;
                rate = fma(s.xHI, hs, -(k.n02 * x * fma(x, r.kR, s.xHI * r.kC)));
                e = ep0;
            }
            // est = |e/rate| is needed only when it may fall below rem; with
            // |e| >= rem |rate| (1 + 1e-13) it is >= rem whatever the
            // rounding, and the division is skipped
            const double ar = fabs(rate);
            const double lim = rem * ar * 1.0000000000001;
            // non-negative doubles order like their bit patterns: the fast
            // forms compare them on the integer pipe
            const bool skip = STRICT ? (rate == 0.0 || fabs(e) >= lim)
                                     : ((dbits(rate) << 1) == 0ull ||
                                        (long long)dbits(fabs(e)) >= (long long)dbits(lim));
            if (!skip) {
                const double est = STRICT ? fabs(e / rate) : fabs(e) * rcp_nr(ar);
                if (est < rem) { dtau = est; dt32 = d2f(est); last = false; }
            }
        }
        Cell<G> o;
        double ep, e1;
        FT rd[G];
        float rec32 = 0.0f;
        if (N32 && !ph.ots) rec32 = (d2f(r.aA) - r.aB32) * (xl32 * xl32) * k.K32;
        for (int h = 0;; h++) {
            if (STRICT) {
                chem_trial<G, true>(ph, B.nunit, B.inv_nunit, n0, S, r, alpha, s, dtau, o, ep, e1);
            } else {
                ep = ep0;
                chem_trial_fast<G, DEFER, N32, FT>(ph, B, k, n0, S, r, alpha, s, ep0, dtau, o, e1, rd,
                                                   rec32, xh32, dt32);
            }
            if (ph.isothermal) break;
            const bool finite = STRICT ? isfinite(e1) : finite_bits(e1);
            if (!finite) {                  // no amount of halving repairs a NaN/Inf
                take<G, !DEFER, N32>(s, o);
                ncyc++;
                return err | RTD_ERR_NONFINITE;
            }
            const double de = fabs(e1 - ep), tol = 0.1 * ep;
            if (STRICT ? de <= tol : (long long)dbits(de) <= (long long)dbits(tol)) break;
            if (h >= ph.max_halvings) { err |= RTD_ERR_SUBCYCLE; break; }
            dtau = 0.5 * dtau;
            dt32 = 0.5f * dt32;
            last = false;
        }
        if (tr) tr->push(s, dtau);
        if (DEFER) {
#pragma unroll
            for (int i = 0; i < G; i++) fac[i] *= rd[i];
        }
        take<G, !DEFER, N32>(s, o);
        ncyc++;
        if (last) break;
        tau = tau + dtau;
        rem = span - tau;
        rem32 = d2f(rem);
        if (ncyc >= RTD_MAXCYC) { err |= RTD_ERR_SUBCYCLE; break; }
    }
    return err;
}

template <typename R> __device__ __forceinline__ double flux_tol();
template <> __device__ __forceinline__ double flux_tol<float>() { return 1e-5; }
template <> __device__ __forceinline__ double flux_tol<double>() { return 1e-12; }
// smallest N at which |F|/N is meaningful in the stored precision: below it
// N is denormal or near it (FP32 keeps < 24 bits there and 1/N overflows)
template <typename R> __device__ __forceinline__ R flux_nmin();
template <> __device__ __forceinline__ float flux_nmin<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double flux_nmin<double>() { return 1e-290; }

__device__ __forceinline__ double ldn(const float *p, int64_t i) { return f2d(p[i]); }
__device__ __forceinline__ double ldn(const double *p, int64_t i) { return p[i]; }

// Supercomoving units (Sec. 3): the stored state is the comoving N^, F^
// (units of nunit) and T~ = a^2 T, the density n0 comoving and dt the
// comoving step; the chemistry of step k runs in physical units at a_k:
// N, F, S and n0 scaled by 1/a^3, T = T~/a^2, over a_k dt.  After it, back
// by a^3 (F^ also by a_k/a_(k+1): F^ follows F~/c~, and c~ grows like a) and
// T~ = a^2 T.
// F_TOO: F is carried in the cell (strict form); the fast forms scale F
// once at the end (the 1/a^3 and a^3 cancel, a_k/a_(k+1) goes into fac)
template <int G, bool F_TOO>
__device__ __forceinline__ void cosmo_in(double a, Cell<G> &s, double *S, double &n0, double &span,
                                         double dt_com)
{
    const double ia3 = 1.0 / (a * a * a);
#pragma unroll
    for (int i = 0; i < G; i++) {
        s.N[i] = s.N[i] * ia3;
        if (F_TOO) {
#pragma unroll
            for (int m = 0; m < 3; m++) s.F[i][m] = s.F[i][m] * ia3;
        }
        S[i] = S[i] * ia3;
    }
    n0 = n0 * ia3;
    s.T = s.T / (a * a);
    span = a * dt_com;
}

template <int G, bool F_TOO>
__device__ __forceinline__ void cosmo_out(double a, double a1, Cell<G> &s)
{
    const double a3 = a * a * a, fr = a / a1;
#pragma unroll
    for (int i = 0; i < G; i++) {
        s.N[i] = s.N[i] * a3;
        if (F_TOO) {
#pragma unroll
            for (int m = 0; m < 3; m++) s.F[i][m] = s.F[i][m] * a3 * fr;
        }
    }
    s.T = s.T * (a * a);
}

// FP32 copies of the rescaled n0, S and N for the FP32 photon update (N
// rounded to FP32, s.N its exact double), after cosmo_in
template <int G>
__device__ __forceinline__ void cosmo_32(Cell<G> &s, const double *S, double n0, float *in32)
{
    in32[0] = d2f(n0);
#pragma unroll
    for (int i = 0; i < G; i++) {
        in32[1 + i] = d2f(S[i]);
        s.n32[i] = d2f(s.N[i]);
        s.N[i] = f2d(s.n32[i]);
    }
}

// Diagnostics of a set of cells: two FP64 sums (ionised fraction, photons),
// the largest |F|/N (bits of a non-negative double, so integer max), two
// integer counts.
struct DiagAcc {
    double X, ph;
    unsigned long long fbits, count, ncyc;
};

__device__ __forceinline__ void diag_add(DiagAcc &a, const DiagAcc &b)
{
    a.X += b.X;
    a.ph += b.ph;
    a.fbits = b.fbits > a.fbits ? b.fbits : a.fbits;
    a.count += b.count;
    a.ncyc += b.ncyc;
}

// acquire-release fence at GPU scope: with a relaxed atomic after it, a
// release of the thread's (and, through a barrier, its warp's) earlier
// stores; after an atomic, an acquire (lighter than the sequentially
// consistent __threadfence)
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// warp reduction in a fixed order (shuffle-down tree), result in lane 0
__device__ __forceinline__ DiagAcc warp_reduce_diag(DiagAcc a)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        DiagAcc o;
        o.X = __shfl_down_sync(0xffffffffu, a.X, off);
        o.ph = __shfl_down_sync(0xffffffffu, a.ph, off);
        o.fbits = __shfl_down_sync(0xffffffffu, a.fbits, off);
        o.count = __shfl_down_sync(0xffffffffu, a.count, off);
        o.ncyc = __shfl_down_sync(0xffffffffu, a.ncyc, off);
        diag_add(a, o);
    }
    return a;
}

__device__ __forceinline__ DiagAcc load_part(const DiagPart *p)
{
    DiagAcc a;
    a.X = __ldcg(&p->X);
    a.ph = __ldcg(&p->ph);
    a.fbits = __ldcg(&p->fbits);
    a.count = __ldcg(&p->count);
    a.ncyc = __ldcg(&p->ncyc);
    return a;
}

__device__ __forceinline__ void store_part(DiagPart *p, const DiagAcc &a)
{
    p->X = a.X;
    p->ph = a.ph;
    p->fbits = a.fbits;
    p->count = a.count;
    p->ncyc = a.ncyc;
}

// sum of n partials by one warp: lane l takes l, l + 32, ... in order, then
// the fixed tree; result in lane 0
__device__ __forceinline__ DiagAcc warp_sum_parts(const DiagPart *p, int64_t n)
{
    DiagAcc a = {0.0, 0.0, 0ull, 0ull, 0ull};
    for (int64_t i = threadIdx.x & 31; i < n; i += 32) diag_add(a, load_part(p + i));
    return warp_reduce_diag(a);
}

// the integer fields of a work item (max, counts) across the warp, result in
// lane 0; the FP64 sums of an item are not reduced here (lane values)
__device__ __forceinline__ DiagAcc warp_reduce_ints(DiagAcc a)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long f = __shfl_down_sync(0xffffffffu, a.fbits, off);
        a.fbits = f > a.fbits ? f : a.fbits;
        a.count += __shfl_down_sync(0xffffffffu, a.count, off);
        a.ncyc += __shfl_down_sync(0xffffffffu, a.ncyc, off);
    }
    return a;
}

// Sum of a group of n work items by one warp: the integer fields from the
// items' partials, the FP64 sums from their lane values (lane l adds slot l
// of every item in item order), then the fixed tree; result in lane 0.  The
// per-item FP64 sums thus cost n adds per lane instead of a tree per item.
__device__ __forceinline__ DiagAcc group_sum(const DiagPart *p, const double *lanev, int64_t n)
{
    const int l = threadIdx.x & 31;
    DiagAcc a = {0.0, 0.0, 0ull, 0ull, 0ull};
    for (int64_t i = l; i < n; i += 32) diag_add(a, load_part(p + i));
    double x = 0.0, ph = 0.0;
    for (int64_t j = 0; j < n; j++) {
        x += __ldcg(lanev + j * (2 * RTD_CHEM_ITEM) + l);
        ph += __ldcg(lanev + j * (2 * RTD_CHEM_ITEM) + RTD_CHEM_ITEM + l);
    }
    a.X = x;
    a.ph = ph;
    return warp_reduce_diag(a);
}

// All groups of box b are reduced: sum the group partials in a fixed order
// and write the step's diagnostics (ionised fraction, photons, max f,
// n(xHI < 0.5), mean sub-cycles) into lastdiag and the caller's history.
// Called by one warp.
__device__ __forceinline__ void reduce_box(const BoxDev &B, int b, const DiagBuf &db, Ctl *ctl)
{
    const DiagAcc a = warp_sum_parts(db.gpart + B.cgroup0, B.ncgroups);
    if ((threadIdx.x & 31) == 0) {
        const double nc = (double)B.ncell;
        double d[RTD_NDIAG];
        d[0] = a.X / nc;
        d[1] = a.ph * B.nunit * (B.dx * B.dx * B.dx);
        d[2] = __longlong_as_double((long long)a.fbits);
        d[3] = (double)a.count;
        d[4] = (double)a.ncyc / nc;
        for (int k = 0; k < RTD_NDIAG; k++) db.last[b * RTD_NDIAG + k] = d[k];
        if (ctl->hist) {
            double *h = ctl->hist + ((int64_t)ctl->step * ctl->nboxes + b) * RTD_NDIAG;
            for (int k = 0; k < RTD_NDIAG; k++) h[k] = d[k];
        }
        db.done[b] = 0;                      // ready for the next step
    }
}

// Staged inputs of one row of 32 cells of a chemistry work item (the fast
// forms): U* of every group, the cells' constants, x_HI, T, n0; two rows per
// warp in dynamic shared memory
template <int G, typename TU, typename TN>
struct ChemRow {
    V4<TU> U[G][RTD_CHEM_ITEM];
    CellConst cc[RTD_CHEM_ITEM];
    double xHI[RTD_CHEM_ITEM], T[RTD_CHEM_ITEM];
    TN n0[RTD_CHEM_ITEM];
};
template <int G, typename TU, typename TN, bool STRICT>
constexpr size_t chem_smem_bytes()
{
    return STRICT ? 0 : sizeof(ChemRow<G, TU, TN>) * 2 * (RTD_CHEM_BLOCK / 32);
}

// One work item = RTD_CHEM_LANE_CELLS x RTD_CHEM_ITEM (4 x 32) consecutive
// cells of one box and one warp, each lane taking one cell of every row of
// 32 in turn; warps draw items independently (no block barrier).
// Reads the post-transport state, runs the sub-cycled chemistry over the
// box's dt, writes the new radiation state into the caller's U and the
// item's diagnostic partial.  The warp that completes a group of
// RTD_CHEM_GROUP items sums the group; the warp that completes a box's last
// group reduces the box (no separate diagnostics launch).  Every sum runs
// in a fixed order of cells, so the diagnostics do not depend on scheduling.
template <int G, typename TU, typename TN, bool STRICT>
__global__ void __launch_bounds__(RTD_CHEM_BLOCK)
k_chem(const BoxDev *__restrict__ boxes, int nboxes, int64_t nitems, Phys ph, Ctl *ctl,
       DiagBuf db, int grab)
{
    const int lane = threadIdx.x & 31;
    const RateCoef *tab = (ph.rtab && !ph.rates_const) ? ph.rtab : nullptr;
    // fast forms: each row of 32 cells' inputs (U* of every group, x_HI, T,
    // n0) is staged into the warp's shared-memory buffers by cp.async while
    // the lanes work on the previous row, so the DRAM latency of a cell's
    // loads is hidden without registers; a lane reads back only what it
    // copied itself
    constexpr bool STAGE = !STRICT;
    using Row = ChemRow<G, TU, TN>;
    extern __shared__ __align__(16) unsigned char chem_smem_raw[];
    Row *wrow = reinterpret_cast<Row *>(chem_smem_raw) + (STAGE ? 2 * (threadIdx.x >> 5) : 0);
    // items are handed out `grab` at a time from a counter, so warps that
    // draw cheap cells (cold gas) take more of them; the order of the work
    // does not enter any result
    unsigned long long knext = 0;
    int kleft = 0;
    for (;;) {
        if (kleft == 0) {
            if (lane == 0) knext = atomicAdd(&ctl->chem_next, (unsigned long long)grab);
            knext = __shfl_sync(0xffffffffu, knext, 0);
            kleft = grab;
        }
        const unsigned long long k = knext++;
        kleft--;
        if (k >= (unsigned long long)nitems) break;
        const int64_t it = (int64_t)k;
        const int b = find_box(boxes, nboxes, it, true);
        const BoxDev &B = boxes[b];
        const int64_t li = it - B.citem0;                 // item within the box
        DiagAcc v = {0.0, 0.0, 0ull, 0ull, 0ull};
        const V4<TU> *Us = reinterpret_cast<const V4<TU> *>(B.Us);
        // copies of row hr into buffer hr & 1 (an empty group past the item)
        auto stage = [&](int hr) {
            const int64_t cs = (li * RTD_CHEM_LANE_CELLS + hr) * RTD_CHEM_ITEM + lane;
            if (hr < RTD_CHEM_LANE_CELLS && cs < B.ncell) {
                Row &r = wrow[hr & 1];
#pragma unroll
                for (int i = 0; i < G; i++) cp_cell(&r.U[i][lane], Us + (int64_t)i * B.ncell + cs);
                {
                    const char *cg = reinterpret_cast<const char *>(
                        ph.cc + it * (RTD_CHEM_LANE_CELLS * RTD_CHEM_ITEM) + hr * RTD_CHEM_ITEM + lane);
                    char *cd = reinterpret_cast<char *>(&r.cc[lane]);
                    cp_async16(cd, cg);
                    cp_async16(cd + 16, cg + 16);
                    cp_async16(cd + 32, cg + 32);
                }
                cp_async8(&r.xHI[lane], B.xHI + cs);
                cp_async8(&r.T[lane], B.T + cs);
                if constexpr (sizeof(TN) == 4) cp_async4(&r.n0[lane], reinterpret_cast<const TN *>(B.n0) + cs);
                else cp_async8(&r.n0[lane], reinterpret_cast<const TN *>(B.n0) + cs);
            }
            cp_async_commit();
        };
        if constexpr (STAGE) stage(0);
        // does the item hold a source cell?  (one search per item; the
        // sources are sparse, so most items skip the per-cell search)
        bool item_src = false;
        if (B.nsrc > 0) {
            const int64_t c0 = li * (RTD_CHEM_LANE_CELLS * RTD_CHEM_ITEM);
            int lo = 0, hi = B.nsrc;                     // first source cell >= c0
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (B.src_cell[mid] < c0) lo = mid + 1; else hi = mid;
            }
            item_src = lo < B.nsrc && B.src_cell[lo] < c0 + RTD_CHEM_LANE_CELLS * RTD_CHEM_ITEM;
        }
        unsigned fmb = 0u;                               // FP32 state: max |F|/N, float bits
        // the item's cells: RTD_CHEM_LANE_CELLS rows of 32, one cell of each
        // per lane, in order (the lane's diagnostics summed in that order)
        for (int hrow = 0; hrow < RTD_CHEM_LANE_CELLS; hrow++) {
        const int64_t c = (li * RTD_CHEM_LANE_CELLS + hrow) * RTD_CHEM_ITEM + lane;
        if constexpr (STAGE) {
            stage(hrow + 1);
            cp_async_wait<1>();                          // row hrow has landed
        }
        const Row &rw = wrow[STAGE ? (hrow & 1) : 0];
        if (c < B.ncell) {
            V4<TU> *U = reinterpret_cast<V4<TU> *>(B.U);
            Cell<G> s;
            unsigned long long nclamp = 0;
            bool gross = false;
            // fast forms: F stays in the stored precision and is scaled once
            // at the end (read again from U*) by the product of its per-trial
            // factors (fac), formed in that precision (FP32 photon update of
            // the split form)
            using FT = typename std::conditional<!STRICT && std::is_same<TU, float>::value, float,
                                                 double>::type;
            // FP32 photon update (split form): N, n0 and the source terms go
            // to the chemistry in FP32 as they were read, beside their exact
            // doubles (no conversion back)
            constexpr bool N32 = std::is_same<FT, float>::value;
            float in32[1 + G];
            FT fac[G];
#pragma unroll
            for (int i = 0; i < G; i++) {
                const V4<TU> u = STAGE ? rw.U[i][lane] : ld4(Us + (int64_t)i * B.ncell + c);
                // N32: s.N is first formed by the trials (or by the rescaling
                // of supercomoving units)
                if constexpr (N32) s.n32[i] = u.x;
                else s.N[i] = to_d(u.x);
                fac[i] = FT(1);
                if (STRICT) {
                    s.F[i][0] = to_d(u.y); s.F[i][1] = to_d(u.z); s.F[i][2] = to_d(u.w);
                }
                // flux limit after transport, in the state's own precision;
                // F is scaled by 1/N first so no square underflows
                if (u.x > flux_nmin<TU>()) {
                    const TU rn = TU(1) / u.x;
                    const TU ux = u.y * rn, uy = u.z * rn, uz = u.w * rn;
                    const TU f2 = ux * ux + uy * uy + uz * uz;
                    const TU tol = (TU)(1.0 + flux_tol<TU>());
                    if (f2 > tol * tol) nclamp++;
                    if (f2 > TU(1.01 * 1.01)) gross = true;
                }
            }
            if (gross) atomicOr(&ctl->err, RTD_ERR_REALIZ);
            if (nclamp) atomicAdd(&ctl->nclamp, nclamp);
            s.xHI = STAGE ? rw.xHI[lane] : B.xHI[c];
            s.T = STAGE ? rw.T[lane] : B.T[c];
            // fast forms: n0 and its constants as k_cconst formed them
            const double n0 = STAGE ? rw.cc[lane].n0 : ldn(reinterpret_cast<const TN *>(B.n0), c);
            CellConst kcv;
            if constexpr (STAGE) kcv = rw.cc[lane];
            if constexpr (N32) in32[0] = STAGE ? (float)rw.n0[lane] : d2f(n0);
            // source term of this cell: sorted unique cells, binary search
            double S[G];
#pragma unroll
            for (int i = 0; i < G; i++) {
                S[i] = 0.0;
                in32[1 + i] = 0.0f;
            }
            if (item_src) {
                int lo = 0, hi = B.nsrc - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (B.src_cell[mid] < c) lo = mid + 1; else hi = mid;
                }
                if (B.src_cell[lo] == c) {
#pragma unroll
                    for (int i = 0; i < G; i++) {
                        S[i] = B.src_S[(int64_t)lo * G + i];
                        if constexpr (N32) in32[1 + i] = d2f(S[i]);
                    }
                }
            }
            int ncyc = 0;
            unsigned int err = 0;
            // supercomoving units: the state is comoving, the chemistry runs
            // in physical units at this step's a (N, F, S, n0 / a^3, T~ / a^2,
            // dt = a dt_com)
            double span = B.dt, n0c = n0, ca = 1.0, ca1 = 1.0;
            if (ph.cosmo) {
                ca = ph.acos[ctl->step];
                ca1 = ph.acos[ctl->step + 1];
                if constexpr (N32) {
#pragma unroll
                    for (int i = 0; i < G; i++) s.N[i] = f2d(s.n32[i]);
                }
                cosmo_in<G, STRICT>(ca, s, S, n0c, span, B.dt);
                if constexpr (N32) cosmo_32<G>(s, S, n0c, in32);
                if constexpr (STAGE) kcv = cell_const(ph, B, n0c);
            }
            // the warm cut holds for every sub-cycle when n0 times the whole
            // step is within its bound (in FP32; an overflow to Inf fails)
            const float span32 = STRICT ? 0.0f : d2f(span);
            const bool warm_cut = !STRICT && (N32 ? in32[0] : d2f(n0c)) * span32 <= RTD_TAB_NDMAX;
            if (ph.nsub > 0) {
                const double h = span / ph.nsub;
                const float h32 = STRICT ? 0.0f : d2f(h);
                for (int k = 0; k < ph.nsub; k++)
                    err |= chem_span<G, STRICT, NoTrace, FT>(ph, tab, B, n0c, S, s, h, false, ncyc, nullptr, fac,
                                                             warm_cut, in32, h32, &kcv);
            } else {
                err |= chem_span<G, STRICT, NoTrace, FT>(ph, tab, B, n0c, S, s, span, true, ncyc, nullptr, fac,
                                                         warm_cut, in32, span32, &kcv);
            }
            if (ph.cosmo) {
                cosmo_out<G, STRICT>(ca, ca1, s);
                if (!STRICT) {
                    const FT fr = from_d<FT>(ca / ca1);
#pragma unroll
                    for (int i = 0; i < G; i++) fac[i] = fac[i] * fr;
                }
                if constexpr (N32) {
#pragma unroll
                    for (int i = 0; i < G; i++) {       // the stored N, rounded once
                        s.n32[i] = d2f(s.N[i]);
                        s.N[i] = f2d(s.n32[i]);
                    }
                }
            }
            if (!finite_bits(s.xHI) || !finite_bits(s.T)) err |= RTD_ERR_NONFINITE;
            if (err) atomicOr(&ctl->err, err);
            double ph_tot = 0.0;
            TU f2max = TU(0);                  // largest |F/N|^2 of the cell's groups
#pragma unroll
            for (int i = 0; i < G; i++) {
                V4<TU> o;
                // N: its FP32 value where the chemistry kept one (s.N is its
                // exact double), else rounded from s.N
                if constexpr (N32) o.x = s.n32[i];
                else o.x = from_d<TU>(s.N[i]);
                if (STRICT) {
                    o.y = from_d<TU>(s.F[i][0]); o.z = from_d<TU>(s.F[i][1]); o.w = from_d<TU>(s.F[i][2]);
                } else {
                    const TU fi = (TU)fac[i];          // FT is TU in the fast forms
                    const V4<TU> u = STAGE ? rw.U[i][lane] : ld4(Us + (int64_t)i * B.ncell + c);
                    o.y = u.y * fi; o.z = u.z * fi; o.w = u.w * fi;
                }
                st4(U + (int64_t)i * B.ncell + c, o);
                const double oxd = N32 ? s.N[i] : to_d(o.x);
                ph_tot = i == 0 ? oxd : ph_tot + oxd;
                if (o.x > flux_nmin<TU>()) {
                    const TU rn = TU(1) / o.x;
                    const TU ux = o.y * rn, uy = o.z * rn, uz = o.w * rn;
                    const TU f2 = ux * ux + uy * uy + uz * uz;
                    f2max = f2 > f2max ? f2 : f2max;
                }
            }
            B.xHI[c] = s.xHI;
            B.T[c] = s.T;
            DiagAcc vc;
            vc.X = 1.0 - s.xHI;
            vc.ph = ph_tot;
            // largest |F|/N: in FP32 state its float bits are kept over the
            // item (non-negative floats order like their bits) and widened
            // once per item
            if constexpr (sizeof(TU) == 4) {
                const unsigned fb = fbits(sqrt(f2max));
                fmb = fb > fmb ? fb : fmb;
                vc.fbits = 0ull;
            } else {
                vc.fbits = dbits(sqrt(f2max));
            }
            // xHI < 0.5 on the integer pipe: doubles order like their bits
            // as signed integers (negative values below every positive one)
            vc.count = (long long)dbits(s.xHI) < (long long)dbits(0.5) ? 1ull : 0ull;
            vc.ncyc = (unsigned long long)ncyc;
            if (hrow == 0) v = vc;
            else diag_add(v, vc);
        }
        }
        if constexpr (sizeof(TU) == 4) v.fbits = dbits(f2d(ffrom(fmb)));
        // FP64 sums: each lane's values go to the item's fixed slots (summed
        // per group); the integer fields are reduced across the warp
        db.lane[it * (2 * RTD_CHEM_ITEM) + lane] = v.X;
        db.lane[it * (2 * RTD_CHEM_ITEM) + RTD_CHEM_ITEM + lane] = v.ph;
        v = warp_reduce_ints(v);
        if (lane == 0) store_part(db.part + it, v);
        // the warp barrier orders every lane's stores before lane 0's release
        // (an acquire-release fence, then the arrival count); the warp that
        // completes the group acquires after its count and shares it
        __syncwarp();
        const int64_t gl = li / RTD_CHEM_GROUP;           // group within the box
        int last_group = 0;
        if (lane == 0) {
            const int64_t left = B.ncitems - gl * RTD_CHEM_GROUP;
            const unsigned n_in = (unsigned)(left < RTD_CHEM_GROUP ? left : RTD_CHEM_GROUP);
            fence_acq_rel_gpu();
            last_group = atomicAdd(&db.gdone[B.cgroup0 + gl], 1u) == n_in - 1u;
            if (last_group) fence_acq_rel_gpu();
        }
        last_group = __shfl_sync(0xffffffffu, last_group, 0);
        if (last_group) {
            __syncwarp();
            const int64_t first = B.citem0 + gl * RTD_CHEM_GROUP;
            const int64_t left = B.ncitems - gl * RTD_CHEM_GROUP;
            const DiagAcc g = group_sum(db.part + first, db.lane + first * (2 * RTD_CHEM_ITEM),
                                        left < RTD_CHEM_GROUP ? left : RTD_CHEM_GROUP);
            int last_box = 0;
            if (lane == 0) {
                store_part(db.gpart + B.cgroup0 + gl, g);
                db.gdone[B.cgroup0 + gl] = 0u;            // ready for the next step
                __threadfence();
                last_box = atomicAdd(&db.done[b], 1u) == (unsigned)(B.ncgroups - 1);
            }
            last_box = __shfl_sync(0xffffffffu, last_box, 0);
            if (last_box) {
                __threadfence();
                reduce_box(B, b, db, ctl);
            }
        }
    }
    // every warp has drawn its last (empty) item before it counts itself
    // here; the last one resets the counters for the next launch
    if (lane == 0) {
        __threadfence();
        const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(&ctl->chem_fin, 1ull) == nw - 1ull) {
            ctl->chem_next = 0ull;
            ctl->chem_fin = 0ull;
            __threadfence();
        }
    }
}



// The fast forms' per-cell chemistry constants from the boxes' n0 (once per
// rt_step call; n0 is static within a call), in the chemistry's item order:
// one warp per item of RTD_CHEM_LANE_CELLS rows of 32 cells.
template <typename TN>
__global__ void __launch_bounds__(256)
k_cconst(const BoxDev *__restrict__ boxes, int nboxes, int64_t nitems, Phys ph, CellConst *cc)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems; it += nw) {
        const BoxDev &B = boxes[find_box(boxes, nboxes, it, true)];
        const int64_t li = it - B.citem0;
#pragma unroll
        for (int r = 0; r < RTD_CHEM_LANE_CELLS; r++) {
            const int64_t c = (li * RTD_CHEM_LANE_CELLS + r) * RTD_CHEM_ITEM + lane;
            if (c < B.ncell)
                cc[it * (RTD_CHEM_LANE_CELLS * RTD_CHEM_ITEM) + r * RTD_CHEM_ITEM + lane] =
                    cell_const(ph, B, ldn(reinterpret_cast<const TN *>(B.n0), c));
        }
    }
}

// CRTA fine level (Sec. 5): one work item = 32 refined cells of one box, one
// warp.  Each refined cell takes its parent's post-transport N, F (the field
// the coarse chemistry used, still in U*) and source term, its own density
// and state, and runs the same sub-cycled chemistry over the box's dt; its
// radiation result is discarded (radiation is transported on the coarse grid
// only).  Runs after the coarse chemistry of the step.
__device__ __forceinline__ int find_fine_box(const FineDev *fines, int nboxes, int64_t item)
{
    int lo = 0, hi = nboxes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fines[mid].fitem0 <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int G, typename TU, typename TN, bool STRICT>
__global__ void __launch_bounds__(RTD_CHEM_BLOCK)
k_chem_fine(const BoxDev *__restrict__ boxes, const FineDev *__restrict__ fines, int nboxes,
            int64_t nitems, Phys ph, Ctl *ctl)
{
    const int lane = threadIdx.x & 31;
    const RateCoef *tab = (ph.rtab && !ph.rates_const) ? ph.rtab : nullptr;
    for (;;) {
        unsigned long long k = 0;
        if (lane == 0) k = atomicAdd(&ctl->fine_next, 1ull);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= (unsigned long long)nitems) break;
        const int64_t it = (int64_t)k;
        const int b = find_fine_box(fines, nboxes, it);
        const BoxDev &B = boxes[b];
        const FineDev &F = fines[b];
        const int64_t f = (it - F.fitem0) * RTD_CHEM_ITEM + lane;
        if (f >= F.nfine) continue;
        const int64_t c = F.parent[f];
        const V4<TU> *Us = reinterpret_cast<const V4<TU> *>(B.Us);
        Cell<G> s;
        // the refined cell's radiation is not kept (fac only as in k_chem)
        using FT = typename std::conditional<!STRICT && std::is_same<TU, float>::value, float, double>::type;
        constexpr bool N32 = std::is_same<FT, float>::value;   // FP32 photon update (split form)
        float in32[1 + G];
        FT fac[G];
#pragma unroll
        for (int i = 0; i < G; i++) {
            const V4<TU> u = ld4(Us + (int64_t)i * B.ncell + c);
            if constexpr (N32) s.n32[i] = u.x;
            else s.N[i] = to_d(u.x);
            fac[i] = FT(1);
            if (STRICT) {
                s.F[i][0] = to_d(u.y); s.F[i][1] = to_d(u.z); s.F[i][2] = to_d(u.w);
            }
        }
        s.xHI = F.xHI[f];
        s.T = F.T[f];
        const double n0 = ldn(reinterpret_cast<const TN *>(F.n0), f);
        if constexpr (N32) {
            if constexpr (std::is_same<TN, float>::value) in32[0] = reinterpret_cast<const float *>(F.n0)[f];
            else in32[0] = d2f(n0);
        }
        double S[G];
#pragma unroll
        for (int i = 0; i < G; i++) {
            S[i] = 0.0;
            in32[1 + i] = 0.0f;
        }
        if (B.nsrc > 0) {
            int lo = 0, hi = B.nsrc - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (B.src_cell[mid] < c) lo = mid + 1; else hi = mid;
            }
            if (B.src_cell[lo] == c) {
#pragma unroll
                for (int i = 0; i < G; i++) {
                    S[i] = B.src_S[(int64_t)lo * G + i];
                    if constexpr (N32) in32[1 + i] = d2f(S[i]);
                }
            }
        }
        int ncyc = 0;
        unsigned int err = 0;
        double span = B.dt, n0c = n0;
        if (ph.cosmo) {
            if constexpr (N32) {
#pragma unroll
                for (int i = 0; i < G; i++) s.N[i] = f2d(s.n32[i]);
            }
            cosmo_in<G, STRICT>(ph.acos[ctl->step], s, S, n0c, span, B.dt);
            if constexpr (N32) cosmo_32<G>(s, S, n0c, in32);
        }
        CellConst kcv;
        if constexpr (!STRICT) kcv = cell_const(ph, B, n0c);
        const float span32 = STRICT ? 0.0f : d2f(span);
        const bool warm_cut = !STRICT && (N32 ? in32[0] : d2f(n0c)) * span32 <= RTD_TAB_NDMAX;
        if (ph.nsub > 0) {
            const double h = span / ph.nsub;
            const float h32 = STRICT ? 0.0f : d2f(h);
            for (int q = 0; q < ph.nsub; q++)
                err |= chem_span<G, STRICT, NoTrace, FT>(ph, tab, B, n0c, S, s, h, false, ncyc, nullptr, fac,
                                                         warm_cut, in32, h32, &kcv);
        } else {
            err |= chem_span<G, STRICT, NoTrace, FT>(ph, tab, B, n0c, S, s, span, true, ncyc, nullptr, fac,
                                                     warm_cut, in32, span32, &kcv);
        }
        if (ph.cosmo) s.T = s.T * (ph.acos[ctl->step] * ph.acos[ctl->step]);
        if (!finite_bits(s.xHI) || !finite_bits(s.T)) err |= RTD_ERR_NONFINITE;
        if (err) atomicOr(&ctl->err, err);
        F.xHI[f] = s.xHI;
        F.T[f] = s.T;
    }
    // the last warp to finish resets the counters for the next launch
    if (lane == 0) {
        __threadfence();
        const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(&ctl->fine_fin, 1ull) == nw - 1ull) {
            ctl->fine_next = 0ull;
            ctl->fine_fin = 0ull;
            __threadfence();
        }
    }
}

}  // namespace rtk
