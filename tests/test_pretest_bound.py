"""The chemistry's FP32 pre-test of the dtau estimate's skip (fast forms).

The kernel skips the FP64 estimate when an FP32 upper bound of
q = rem (heat + cool) / e is at most 0.999, arguing that heat, cool >= 0
make |heat - cool| <= heat + cool, that every term of q is a product or sum
of non-negative FP32 numbers (a few ulp each, n0 and kB cancelled), and that
q <= 0.999 therefore implies the FP64 skip |e| >= rem |rate| (1 + 1e-13).

This checks that implication on random and adversarial states: the bound is
formed in float32 with one rounding per operation (as the kernel's
operations round), the skip in float64 in the kernel's order.  No GPU."""
import numpy as np

KB = 1.380649e-16
F = np.float32


def fmaf(a, b, c):
    """a b + c rounded once to float32 (the float32 product is exact in
    float64; the float64 sum then rounds at 2^-53, far inside the margin)."""
    return F(float(a) * float(b) + float(c))


def bound_q(rem, xHI, T, n0, nunit, N, hK, kR, kC):
    """The kernel's FP32 bound, operation by operation."""
    xh = F(abs(xHI))
    xl = F(abs(1.0 - xHI))
    hsum = F(0.0)
    for h, n in zip(hK, N):
        hsum = fmaf(F(h), F(abs(n)), hsum)
    kb15i = F(1.0 / (1.5 * KB))
    kr = F(F(abs(kR)) * kb15i)           # kR here: the kernel's FP32 upper bound of kR
    kc = F(F(abs(kC)) * kb15i)
    cool = F(F(F(n0) * xl) * fmaf(xl, kr, F(xh * kc)))
    num = fmaf(F(xh * F(nunit)), hsum, cool)
    den = F(F(F(2.0) - xh) * F(T))
    with np.errstate(divide="ignore", over="ignore", invalid="ignore"):
        return F(F(F(rem) * num) * F(F(1.0) / den))


def fp64_skips(rem, xHI, T, n0, nunit, N, hN, kR, kC):
    """The kernel's FP64 skip test (fast forms)."""
    cvn = (1.5 * KB) * n0
    e = cvn * (2.0 - xHI) * T
    hs = hN[0] * N[0]
    for h, n in zip(hN[1:], N[1:]):
        hs = h * n + hs
    hs = hs * n0
    x = 1.0 - xHI
    rate = xHI * hs - (n0 * n0) * x * (x * kR + xHI * kC)
    lim = rem * abs(rate) * 1.0000000000001
    return rate == 0.0 or abs(e) >= lim


def test_pretest_implies_the_fp64_skip():
    rng = np.random.Generator(np.random.PCG64(31))
    c = 2.99792458e10 * 0.1
    hits = 0
    for k in range(200000):
        G = 3
        nunit = 10.0 ** rng.uniform(-8, 2)
        SigE = 10.0 ** rng.uniform(-30, -26, G)
        hN = c * nunit * SigE
        hK = np.abs(c * SigE / (1.5 * KB))
        mode = k % 4
        xHI = (1.0 - 10.0 ** rng.uniform(-12, 0)) if mode == 0 else 10.0 ** rng.uniform(-12, 0)
        T = 10.0 ** rng.uniform(0, 8)
        n0 = 10.0 ** rng.uniform(-6, 3)
        N = [float(F(10.0 ** rng.uniform(-40, 3))) for _ in range(G)]
        if mode == 3:
            N = [0.0] * G
        kR = 10.0 ** rng.uniform(-28, -21)
        kC = 0.0 if mode == 2 else 10.0 ** rng.uniform(-40, -18)
        rem = 10.0 ** rng.uniform(8, 15)
        if mode == 1:
            # heating close to cooling: |rate| far below heat + cool
            heat = xHI * n0 * sum(h * n for h, n in zip(hN, N))
            cool = n0 * n0 * (1.0 - xHI) * ((1.0 - xHI) * kR + xHI * kC)
            if heat > 0 and cool > 0:
                N = [n * cool / heat * (1.0 + rng.uniform(-1e-9, 1e-9)) for n in N]
                N = [float(F(n)) for n in N]
        # the kernel's kR in the pre-test: an upper bound over its table
        # interval (up to ~1% above kR, rounded up in FP32)
        kRb = float(np.nextafter(F(kR * (1.0 + rng.uniform(0.0, 1e-2))), np.float32(np.inf)))
        q = bound_q(rem, xHI, T, n0, nunit, N, hK, kRb, kC)
        if q >= 0.0 and q <= F(0.999):
            hits += 1
            assert fp64_skips(rem, xHI, T, n0, nunit, N, hN, kR, kC), (k, q)
    assert hits > 20000
