"""Pins of the oracle's atomic-rate and cooling fits (reading R8) against
physics that does not come from the fits themselves.

The paper cites its rate compilations (Sec. 2.2.4) without printing them; the
oracle uses the Hui & Gnedin (1997) fits for alpha_A, alpha_B, beta and the
recombination cooling, the exp(-118348/T)/(1 + sqrt(T/1e5)) form for the
collisional-excitation cooling, and 1.42e-27 g_ff sqrt(T), g_ff = 1.3, for the
free-free cooling.  Each function is checked here against an independent
source, chosen so that a wrong exponent, a wrong constant, a dropped factor or
the case A/B constants swapped fails at least one check:

* the case A - case B difference of the recombination rate and of the
  recombination cooling is recombination straight to 1s.  Its rate
  coefficient and its kinetic-energy loss follow from the exact hydrogenic 1s
  photo-ionisation cross-section (Osterbrock & Ferland 2006, Eq. 2.4; the
  threshold value 2^9 pi^2 alpha a0^2/(3 e^4) = 6.304e-18 cm^2) through the
  Milne relation sigma_rec = (g_1s/g_+)(h nu/(m c v))^2 a_nu (Osterbrock &
  Ferland 2006, Sec. 2.1; Rybicki & Lightman 1979, Sec. 10.5) averaged over a
  Maxwellian.  At 1e4 K that gives 1.580e-13 cm^3/s, Osterbrock & Ferland's
  Table 2.1 value of alpha_{1^2S};
* case B (all levels n >= 2): the Kramers cross-section with unit Gaunt
  factor, a_n(nu) = (64 pi/(3 sqrt 3)) alpha a0^2 n (nu_n/nu)^3 (Rybicki &
  Lightman 1979, Eq. 10.54), through the same Milne relation and summed over
  n.  Its rate is close to alpha_B, and the mean kinetic energy carried off per
  recombination, Lambda_B/(alpha_B kT), much closer, since the Gaunt factors
  nearly cancel in the ratio;
* collisional ionisation: the Maxwellian average of Lotz's (1967, ApJS 14,
  207) empirical cross-section for H I (a = 4.0e-14 cm^2 eV^2, b = 0.60,
  c = 0.56) and Voronov's (1997, ADNDT 65, 1) fit for H (A = 2.91e-8 cm^3/s,
  X = 0.232, K = 0.39, P = 0); and at low T the Arrhenius energy of the rate
  equals the ionisation energy;
* collisional-ionisation cooling: each ionisation costs the ionisation energy
  of hydrogen, Ry/(1 + m_e/m_p) = 13.598 eV (CODATA 2018);
* collisional-excitation cooling: the Arrhenius energy at low T is the
  Lyman-alpha excitation energy (3/4) Ry/(1 + m_e/m_p) = 10.199 eV, and the
  implied effective collision strength of 1s -> n >= 2 at 5e3-2e4 K is of the
  size of the n = 2 collision strengths, 1s-2s ~0.3 plus 1s-2p ~0.5 (R-matrix
  results of Anderson et al. 2000, J. Phys. B 33, 1255);
* free-free: the classical emissivity (Rybicki & Lightman 1979, Eq. 5.15b)
  2^5 pi e^6/(3 h m c^3) (2 pi k/(3 m))^(1/2) g_B sqrt(T), evaluated from
  CODATA constants (1.4256e-27 cgs), with the Gaunt factor g_B = 1.3 the
  oracle states.

Tolerances are the spread measured between the fits and these sources (given
beside each check), not the other way round.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O

# CODATA 2018, cgs and eV
KB_EV = 8.617333262e-5
KB = 1.380649e-16
ERG_PER_EV = 1.602176634e-12
ME_C2_EV = 510998.95
C_CGS = 2.99792458e10
ALPHA_FS = 7.2973525693e-3
A0_CM = 5.29177210903e-9
RY_INF_EV = 13.605693122994
MP_OVER_ME = 1836.15267343
E_CHARGE = 4.80320471e-10
H_PLANCK = 6.62607015e-27
M_E = 9.1093837015e-28

RY_H = RY_INF_EV / (1.0 + 1.0 / MP_OVER_ME)      # ionisation energy of H, 13.598 eV
E_LYA = 0.75 * RY_H                               # 1s -> 2 excitation energy
SIGMA_1S = 2 ** 9 * math.pi ** 2 / (3 * math.e ** 4) * ALPHA_FS * A0_CM ** 2
KRAMERS = 64 * math.pi / (3 * math.sqrt(3)) * ALPHA_FS * A0_CM ** 2


def sigma_1s(hnu):
    """Exact hydrogenic 1s photo-ionisation cross-section (cm^2), hnu in eV."""
    x = hnu / RY_H
    if x <= 1.0:
        return SIGMA_1S if x == 1.0 else 0.0
    eps = math.sqrt(x - 1.0)
    return SIGMA_1S * x ** -4 * math.exp(4 - 4 * math.atan(eps) / eps) / -math.expm1(-2 * math.pi / eps)


def maxwell_flux(u, kT):
    """v f(v) dv in terms of u = E/kT: the Maxwellian's speed-weighted
    density per unit u (cm/s), E the electron kinetic energy."""
    E = u * kT
    return C_CGS * math.sqrt(2 * E / ME_C2_EV) * 2 * math.sqrt(u / math.pi) * math.exp(-u)


def milne_1s(T):
    """(rate coefficient cm^3/s, kinetic-energy loss erg cm^3/s) of
    recombination to 1s: Milne relation with g_1s = 2, g_+ = 1."""
    kT = KB_EV * T

    def srec(u):
        E = u * kT
        hnu = RY_H + E
        return 2.0 * hnu ** 2 / (2 * ME_C2_EV * E) * sigma_1s(hnu)

    rate = integrate.quad(lambda u: srec(u) * maxwell_flux(u, kT), 0, 60, limit=400,
                          epsrel=1e-9, epsabs=0)[0]
    loss = integrate.quad(lambda u: srec(u) * maxwell_flux(u, kT) * u * kT * ERG_PER_EV, 0, 60,
                          limit=400, epsrel=1e-9, epsabs=0)[0]
    return rate, loss


def _ey_e1(y):
    """e^y E1(y), y > 0 (asymptotic series beyond y = 50, error < 1e-7)."""
    y = np.asarray(y, dtype=float)
    big = y > 50
    out = np.empty_like(y)
    out[~big] = np.exp(y[~big]) * special.exp1(y[~big])
    yb = y[big]
    out[big] = (1 - 1 / yb + 2 / yb ** 2 - 6 / yb ** 3 + 24 / yb ** 4) / yb
    return out


def kramers_case_b(T, nmax=1500):
    """(rate, kinetic-energy loss) of recombination to every level n >= 2 with
    Kramers cross-sections (unit Gaunt factor) and g_n = 2 n^2.  With
    a_n = KRAMERS n (chi_n/hnu)^3 the Maxwellian integral is closed:
    rate_n = g_n KRAMERS n chi_n^3/(2 m c^2) * (2c/sqrt(pi)) sqrt(2/(m c^2)) (kT)^(-3/2) e^y E1(y)
    loss_n = the same with e^y E1(y) replaced by kT (1 - y e^y E1(y)), y = chi_n/kT."""
    kT = KB_EV * T
    n = np.arange(2, nmax + 1, dtype=float)
    chi = RY_H / n ** 2
    y = chi / kT
    g = _ey_e1(y)
    pre = (2 * n ** 2) * KRAMERS * n * chi ** 3 / (2 * ME_C2_EV) * (2 * C_CGS / math.sqrt(math.pi)) \
        * math.sqrt(2 / ME_C2_EV) * kT ** -1.5
    rate = np.sum(pre * g)
    loss = np.sum(pre * kT * (1 - y * g)) * ERG_PER_EV
    return float(rate), float(loss)


def test_physics_helpers_reproduce_textbook_values():
    # the exact 1s threshold cross-section and alpha_{1^2S}(1e4 K) of
    # Osterbrock & Ferland (2006), Eq. 2.4 and Table 2.1
    assert SIGMA_1S == pytest.approx(6.30e-18, rel=2e-3, abs=0)
    assert milne_1s(1e4)[0] == pytest.approx(1.58e-13, rel=5e-3, abs=0)
    # recombination to 1s at low T: sigma_rec ~ 1/E makes the mean energy kT
    r, l = milne_1s(100.0)
    assert l / (r * KB * 100.0) == pytest.approx(1.0, abs=2e-3)
    # Kramers case B at 1e4 K lies within the Gaunt factors (~5%) of the
    # tabulated alpha_B = 2.59e-13
    assert kramers_case_b(1e4)[0] == pytest.approx(2.59e-13, rel=0.06, abs=0)


# Each pin below is a function of a rate provider rate(name, T), so that the
# same checks run on the oracle and, in the last test, on copies of the oracle
# with a mistake planted in one fit.

def chk_a_minus_b_rate(rate, T):
    """alpha_A - alpha_B against the exact 1s Milne rate (measured: 3% at
    100 K, 8% at 1e4 K, 0.6% at 1e6 K)."""
    fit = rate("alphaA", T) - rate("alphaB", T)
    assert fit == pytest.approx(milne_1s(T)[0], rel=0.10, abs=0)


def chk_a_minus_b_cooling(rate, T, tol):
    """The case A/B split of the recombination cooling: Lambda_A - Lambda_B
    against the kinetic energy carried off by recombination to 1s (measured:
    <= 5.5% over 3e3-1e6 K, 6% at 1e3 K; 18% at 100 K, where it is a
    difference of two fits each worth several times it)."""
    fit = rate("cool_recA", T) - rate("cool_recB", T)
    assert fit == pytest.approx(milne_1s(T)[1], rel=tol, abs=0)


def chk_case_b(rate, T):
    """alpha_B within the Gaunt factors of the Kramers sum (measured 0.95-1.02)
    and the mean energy per case-B recombination Lambda_B/(alpha_B kT) within
    5% of its Kramers value (measured 0.4-2.1%, 3.8% at 1e5 K)."""
    r, loss = kramers_case_b(T)
    aB = rate("alphaB", T)
    assert aB == pytest.approx(r, rel=0.07, abs=0)
    kT = KB * T
    assert rate("cool_recB", T) / (aB * kT) == pytest.approx(loss / (r * kT), rel=0.05, abs=0)


def chk_case_a_energy(rate, T):
    """Lambda_A/(alpha_A kT) against the exact 1s part plus the Kramers n >= 2
    part (measured within 3%)."""
    r1, l1 = milne_1s(T)
    rb, lb = kramers_case_b(T)
    kT = KB * T
    want = (l1 + lb) / ((r1 + rb) * kT)
    assert rate("cool_recA", T) / (rate("alphaA", T) * kT) == pytest.approx(want, rel=0.05, abs=0)


def _lotz_sigma(E):
    """Lotz (1967) empirical ionisation cross-section of H I, cm^2 (E in eV)."""
    P = 13.6
    if E <= P:
        return 0.0
    return 4.0e-14 * math.log(E / P) / (E * P) * (1 - 0.60 * math.exp(-0.56 * (E / P - 1)))


def _lotz_rate(T):
    kT = KB_EV * T
    lo = 13.6 / kT
    return integrate.quad(lambda u: _lotz_sigma(u * kT) * maxwell_flux(u, kT), lo, lo + 80,
                          limit=400, epsrel=1e-9, epsabs=0)[0]


def _voronov_rate(T):
    U = 13.6 / (KB_EV * T)
    return 2.91e-8 * U ** 0.39 * math.exp(-U) / (0.232 + U)


def chk_beta(rate, T):
    """beta(T) against the Maxwellian average of Lotz's cross-section
    (measured ratio 1.04-1.15) and Voronov's fit (1.00-1.22)."""
    b = rate("beta", T)
    assert b == pytest.approx(_lotz_rate(T), rel=0.20, abs=0)
    assert b == pytest.approx(_voronov_rate(T), rel=0.25, abs=0)


def _arrhenius_eV(rate, name, T1=3000.0, T2=6000.0):
    r1, r2 = rate(name, T1), rate(name, T2)
    return -math.log(r1 / r2) / (1 / T1 - 1 / T2) * KB_EV


def chk_thresholds(rate):
    """At low T a collisional rate is its threshold's Boltzmann factor times a
    slowly varying prefactor, so its Arrhenius energy between 3000 and 6000 K
    is the threshold energy, up to ~0.2 eV from a prefactor T^s, |s| <= 0.5:
    13.598 eV for ionisation, 10.199 eV (Lyman alpha) for excitation
    (measured 13.79 and 10.17 eV)."""
    assert _arrhenius_eV(rate, "beta") == pytest.approx(RY_H, abs=0.3)
    assert _arrhenius_eV(rate, "cool_colion") == pytest.approx(RY_H, abs=0.3)
    assert _arrhenius_eV(rate, "cool_colexc") == pytest.approx(E_LYA, abs=0.3)


def chk_colion(rate, T):
    """Each collisional ionisation costs the ionisation energy of H."""
    assert rate("cool_colion", T) / rate("beta", T) == pytest.approx(RY_H * ERG_PER_EV, rel=1e-4, abs=0)


def chk_colexc(rate, T):
    """Lambda_exc = E_Lya q, q = 8.629e-6 Upsilon/(g_1 sqrt(T)) e^(-E_Lya/kT),
    g_1 = 2: the effective collision strength the fit implies (measured 0.62,
    0.81, 1.04 at 5e3, 1e4, 2e4 K) must be of the size of the n = 2 collision
    strengths (1s-2s ~0.3 + 1s-2p ~0.5), here between 0.5 and 1.2."""
    q_per_ups = 8.629e-6 / (2 * math.sqrt(T)) * math.exp(-E_LYA / (KB_EV * T))
    ups = rate("cool_colexc", T) / (q_per_ups * E_LYA * ERG_PER_EV)
    assert 0.5 <= ups <= 1.2, ups


def chk_free_free(rate):
    """Rybicki & Lightman Eq. 5.15b from CODATA constants (1.4256e-27) with the
    stated g_B = 1.3, and its sqrt(T) law."""
    pref = (2 ** 5 * math.pi * E_CHARGE ** 6 / (3 * H_PLANCK * M_E * C_CGS ** 3)
            * math.sqrt(2 * math.pi * KB / (3 * M_E)))
    assert pref == pytest.approx(1.4256e-27, rel=1e-4, abs=0)
    for T in (1e2, 1e4, 1e6):
        assert rate("cool_brems", T) == pytest.approx(pref * 1.3 * math.sqrt(T), rel=5e-3, abs=0)
        assert rate("cool_brems", 4 * T) / rate("cool_brems", T) == pytest.approx(2.0, rel=1e-12, abs=0)


T_AB_RATE = [100.0, 1e3, 5e3, 1e4, 2e4, 1e5, 1e6]
T_AB_COOL = [(100.0, 0.22), (1e3, 0.10), (3e3, 0.08), (1e4, 0.08), (2e4, 0.08), (1e5, 0.08),
             (1e6, 0.08)]
T_CASE_B = [100.0, 300.0, 1e3, 5e3, 1e4, 2e4, 1e5, 1e6]
T_CASE_A = [100.0, 1e3, 1e4, 1e5, 1e6]
T_BETA = [8e3, 1e4, 2e4, 5e4, 1e5, 3e5, 1e6, 1e7]
T_COLION = [5e3, 1e4, 1e5, 1e6]
T_COLEXC = [5e3, 1e4, 2e4]


def all_pins():
    """(name, zero-argument check of a rate provider) for every pin above."""
    out = []
    out += [(f"a-b rate {T:g}", lambda r, T=T: chk_a_minus_b_rate(r, T)) for T in T_AB_RATE]
    out += [(f"a-b cooling {T:g}", lambda r, T=T, t=t: chk_a_minus_b_cooling(r, T, t))
            for T, t in T_AB_COOL]
    out += [(f"case B {T:g}", lambda r, T=T: chk_case_b(r, T)) for T in T_CASE_B]
    out += [(f"case A energy {T:g}", lambda r, T=T: chk_case_a_energy(r, T)) for T in T_CASE_A]
    out += [(f"beta {T:g}", lambda r, T=T: chk_beta(r, T)) for T in T_BETA]
    out += [("thresholds", chk_thresholds), ("free-free", chk_free_free)]
    out += [(f"colion {T:g}", lambda r, T=T: chk_colion(r, T)) for T in T_COLION]
    out += [(f"colexc {T:g}", lambda r, T=T: chk_colexc(r, T)) for T in T_COLEXC]
    return out


@pytest.mark.parametrize("T", T_AB_RATE)
def test_case_a_minus_b_rate_is_recombination_to_1s(T):
    chk_a_minus_b_rate(O.rate, T)


@pytest.mark.parametrize("T,tol", T_AB_COOL)
def test_case_a_minus_b_cooling_is_recombination_to_1s(T, tol):
    chk_a_minus_b_cooling(O.rate, T, tol)


@pytest.mark.parametrize("T", T_CASE_B)
def test_case_b_rate_and_energy_per_recombination_against_kramers(T):
    chk_case_b(O.rate, T)


@pytest.mark.parametrize("T", T_CASE_A)
def test_case_a_energy_per_recombination(T):
    chk_case_a_energy(O.rate, T)


@pytest.mark.parametrize("T", T_BETA)
def test_collisional_ionisation_against_cross_section_and_voronov(T):
    chk_beta(O.rate, T)


def test_thresholds_of_collisional_rates():
    chk_thresholds(O.rate)


@pytest.mark.parametrize("T", T_COLION)
def test_collisional_ionisation_cooling_costs_the_ionisation_energy(T):
    chk_colion(O.rate, T)


@pytest.mark.parametrize("T", T_COLEXC)
def test_excitation_cooling_collision_strength(T):
    chk_colexc(O.rate, T)


def test_free_free_cooling_is_the_classical_emissivity():
    chk_free_free(O.rate)


# Plausible transcription mistakes, each planted in a compiled copy of the
# oracle's source: (what it is, the exact text in m1_oracle.c, its replacement).
PLANTED = [
    ("beta: lambda^-1.5 for lambda^-1.089", "pow(l, -1.089)", "pow(l, -1.5)"),
    ("beta: exp(-lambda) for exp(-lambda/2)", "exp(-0.5 * l) * pow(l, -1.089)", "exp(-l) * pow(l, -1.089)"),
    ("beta: outer exponent 1.01 for 1.101", "0.874), 1.101)", "0.874), 1.01)"),
    ("beta: 2.111 for 21.11", "21.11 * pow(T, -1.5)", "2.111 * pow(T, -1.5)"),
    ("recombination cooling: case A constant of case B", "1.778e-29 * T", "3.435e-30 * T"),
    ("recombination cooling: case B constant of case A", "3.435e-30 * T", "1.778e-29 * T"),
    ("recombination cooling A: T factor dropped", "1.778e-29 * T *", "1.778e-29 *"),
    ("recombination cooling A: lambda^1.695 for 1.965", "pow(l, 1.965)", "pow(l, 1.695)"),
    ("recombination cooling B: lambda^1.907 for 1.970", "pow(l, 1.970)", "pow(l, 1.907)"),
    ("recombination cooling B: 2.520 for 2.250", "pow(l / 2.250, 0.376), 3.720)",
     "pow(l / 2.520, 0.376), 3.720)"),
    ("recombination cooling B: outer exponent 3.270 for 3.720", "0.376), 3.720)", "0.376), 3.270)"),
    ("collisional-ionisation cooling: 3/4 of the energy", "ORC_KB * ORC_T_HI * orc_beta(T)",
     "0.75 * ORC_KB * ORC_T_HI * orc_beta(T)"),
    ("excitation cooling: the ionisation temperature", "exp(-118348.0 / T) / (1.0 + sqrt(T / 1.0e5))",
     "exp(-157807.0 / T) / (1.0 + sqrt(T / 1.0e5))"),
    ("excitation cooling: 7.5e-18 for 7.5e-19", "7.5e-19 * exp", "7.5e-18 * exp"),
    ("excitation cooling: 11834.8 for 118348", "exp(-118348.0 / T) / (1.0 + sqrt(T / 1.0e5))",
     "exp(-11834.8 / T) / (1.0 + sqrt(T / 1.0e5))"),
    ("free-free: T for sqrt(T)", "1.42e-27 * 1.3 * sqrt(T)", "1.42e-27 * 1.3 * T"),
    ("free-free: g_ff 1.1 for 1.3", "1.42e-27 * 1.3 * sqrt(T)", "1.42e-27 * 1.1 * sqrt(T)"),
    ("alpha_B: lambda^1.05 for 1.500", "2.753e-14 * pow(l, 1.500)", "2.753e-14 * pow(l, 1.050)"),
    ("alpha_A: 1.269e-12 for 1.269e-13", "1.269e-13 * pow", "1.269e-12 * pow"),
]


def _planted_rate_provider(tmpdir, old, new):
    import ctypes as C
    import subprocess
    src = open(O._build.SRC).read()
    assert src.count(old) == 1, old
    path = os.path.join(tmpdir, "planted.c")
    open(path, "w").write(src.replace(old, new))
    so = os.path.join(tmpdir, "planted.so")
    subprocess.run(["gcc", "-std=gnu99", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    so, path, "-lm"], check=True)
    L = C.CDLL(so)
    fns = {}
    for name in O.RATE_NAMES:
        f = getattr(L, "orc_" + name)
        f.restype, f.argtypes = C.c_double, [C.c_double]
        fns[name] = f
    return lambda name, T: fns[name](T)


def test_pins_hold_for_the_oracle_and_fail_for_planted_mistakes(tmp_path):
    """Every pin passes on the oracle; each planted mistake fails at least one."""
    pins = all_pins()
    for name, chk in pins:
        chk(O.rate)
    survivors = []
    for i, (what, old, new) in enumerate(PLANTED):
        d = tmp_path / f"p{i}"
        d.mkdir()
        rate = _planted_rate_provider(str(d), old, new)
        failed = []
        for name, chk in pins:
            try:
                chk(rate)
            except AssertionError:
                failed.append(name)
        if not failed:
            survivors.append(what)
    assert not survivors, survivors
