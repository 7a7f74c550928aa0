"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an invariant, a limiting case with a known answer, a textbook value, or an
independent brute-force evaluation on a tiny grid.  A plausible mistake in
the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I

C = I.C_LIGHT


def grey_params(G=1, sig=0.0, c=0.1 * C, **kw):
    return O.Params(sigN=[sig] * G, sigE=[sig] * G, Eavg=[20 * 1.602176634e-12] * G,
                    frac=[1.0 / G] * G, c=c, **kw)


# ---------------------------------------------------------------- closure
def levermore_chi(f):
    """Levermore (1984) M1 Eddington factor, textbook form."""
    return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * math.sqrt(4.0 - 3.0 * f * f))


def test_closure_limits():
    P, chi, a, g = O.closure([2.0, 0.0, 0.0, 0.0])
    assert chi == 1.0 / 3.0 and a == 1.0 / 3.0 and g == 0.75
    np.testing.assert_array_equal(P, [2 / 3, 0, 0, 2 / 3, 0, 2 / 3])
    for d in range(3):
        U = [3.0, 0.0, 0.0, 0.0]
        U[1 + d] = 3.0                      # |F| = cN: free streaming along d
        P, chi, a, g = O.closure(U)
        assert chi == 1.0 and a == 0.0 and g == 1.0
        M = np.zeros((3, 3))
        M[d, d] = 3.0                        # N n (x) n
        np.testing.assert_array_equal(P, M[np.triu_indices(3)])
    # N = 0: no pressure
    P, *_ = O.closure([0.0, 0.0, 0.0, 0.0])
    assert np.all(P == 0.0)


@pytest.mark.parametrize("beta", [0.0, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99])
def test_closure_lorentz_boosted_isotropic(beta):
    """Levermore's M1 closure is exact for radiation that is isotropic in a
    frame moving with speed beta c: f = 4b/(3+b^2), chi = (1+3b^2)/(3+b^2)."""
    f = 4 * beta / (3 + beta * beta)
    chi_exact = (1 + 3 * beta * beta) / (3 + beta * beta)
    n = np.array([0.48, -0.6, 0.64])
    n /= np.linalg.norm(n)
    N = 1.7
    P, chi, a, g = O.closure(np.r_[N, f * N * n])
    assert chi == pytest.approx(chi_exact, rel=1e-14, abs=1e-15)
    D = np.zeros((3, 3))
    D[np.triu_indices(3)] = P / N
    D = D + np.triu(D, 1).T
    # eigenvalue chi along n, (1 - chi)/2 across it, trace 1
    np.testing.assert_allclose(D @ n, chi_exact * n, rtol=1e-13, atol=1e-15)
    t = np.cross(n, [1.0, 0.0, 0.0])
    t /= np.linalg.norm(t)
    np.testing.assert_allclose(D @ t, 0.5 * (1 - chi_exact) * t, rtol=1e-13, atol=1e-15)
    assert np.trace(D) == pytest.approx(1.0, rel=1e-14, abs=0)


def test_closure_random_states_match_textbook_form():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        N = 10 ** rng.uniform(-30, 3)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        f = rng.uniform(0, 1)
        P, chi, a, g = O.closure(np.r_[N, f * N * n])
        chi_t = levermore_chi(f)
        D_t = 0.5 * (1 - chi_t) * np.eye(3) + 0.5 * (3 * chi_t - 1) * np.outer(n, n)
        np.testing.assert_allclose(P / N, D_t[np.triu_indices(3)], rtol=1e-12, atol=1e-14)
        assert chi == pytest.approx(chi_t, rel=1e-13, abs=0)


def test_closure_flux_limit_guard():
    """|F| > cN (a rounding excess) is read as free streaming along F."""
    P, chi, a, g = O.closure([1.0, 1.5, 0.0, 0.0])
    assert chi == 1.0
    np.testing.assert_array_equal(P, [1.0, 0, 0, 0, 0, 0])


# ---------------------------------------------------------------- GLF flux
def test_glf_consistent_with_physical_flux():
    rng = np.random.default_rng(2)
    for _ in range(200):
        U = I.random_realizable_state((1, 1, 1), 1, int(rng.integers(1 << 30)))[0, 0, 0, 0]
        P, *_ = O.closure(U)
        Pm = np.zeros((3, 3))
        Pm[np.triu_indices(3)] = P
        Pm = Pm + np.triu(Pm, 1).T
        for d in range(3):
            Phi = O.glf_flux(d, U, U)
            np.testing.assert_allclose(Phi, np.r_[U[1 + d], Pm[d]], rtol=1e-15, atol=0)


def test_glf_is_upwind_for_free_streaming():
    """At f = 1 the GLF flux is exactly the upwind flux at speed c."""
    rng = np.random.default_rng(3)
    for d in range(3):
        for _ in range(50):
            NL, NR = rng.uniform(0, 5, 2)
            e = np.zeros(3)
            e[d] = 1.0
            L, R = np.r_[NL, NL * e], np.r_[NR, NR * e]
            # exact up to the rounding of (NL + NR) - (NR - NL)
            ulp = 2.3e-16 * max(NL, NR)
            np.testing.assert_allclose(O.glf_flux(d, L, R), np.r_[NL, NL * e],
                                       rtol=0, atol=ulp)
            L, R = np.r_[NL, -NL * e], np.r_[NR, -NR * e]
            np.testing.assert_allclose(O.glf_flux(d, L, R), np.r_[-NR, NR * e],
                                       rtol=0, atol=ulp)


# ---------------------------------------------------------------- transport
def test_courant_number():
    p = grey_params()
    assert O.courant_number(p, 1e20) == pytest.approx(0.3, rel=1e-15, abs=0)
    assert O.timestep(p, 1e20) == pytest.approx(0.9 * 1e20 / (3 * p.c), rel=1e-15, abs=0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_transport_fourier_mode_closed_form(axis):
    """F = 0, N = A + B cos(k i): one GLF step gives
    N' = A + B cos(k i)(1 - lam(1 - cos k)),  F'_axis = (lam/3) B sin k sin(k i)."""
    p = grey_params()
    n, m = 16, 3
    k = 2 * np.pi * m / n
    shape = [4, 4, 4]
    shape[2 - axis] = n
    A, B = 1.0, 0.6
    i = np.arange(n)
    prof = A + B * np.cos(k * i)
    sh = [1, 1, 1]
    sh[2 - axis] = n
    U = np.zeros((1, *shape, 4))
    U[0, ..., 0] = prof.reshape(sh)
    lam = 0.3
    out = O.transport(p, U, lam)
    Nexp = A + B * np.cos(k * i) * (1 - lam * (1 - np.cos(k)))
    Fexp = lam / 3 * B * np.sin(k) * np.sin(k * i)
    np.testing.assert_allclose(out[0, ..., 0], np.broadcast_to(Nexp.reshape(sh), shape),
                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[0, ..., 1 + axis], np.broadcast_to(Fexp.reshape(sh), shape),
                               rtol=0, atol=1e-15)
    for d in range(3):
        if d != axis:
            assert np.all(out[0, ..., 1 + d] == 0.0)


def test_uniform_field_is_a_fixed_point():
    p = grey_params(G=2)
    U = np.empty((2, 5, 6, 7, 4))
    U[0, ..., :] = [1.3, 0.2, -0.5, 0.7]
    U[1, ..., :] = [0.4, 0.0, 0.0, 0.3]
    out = O.transport(p, U, 0.3)
    np.testing.assert_array_equal(out, U)


@pytest.mark.parametrize("axis,sign", [(0, 1), (0, -1), (1, 1), (2, -1)])
def test_free_streaming_beam(axis, sign):
    """A planar beam with F = cN in vacuum moves at exactly c: centroid
    advances by c dt per step, F stays equal to N, photons are conserved."""
    nlong = 64
    shape = [2, 2, 2]
    shape[2 - axis] = nlong
    bc = [I.BC_PERIODIC] * 6
    bc[2 * axis] = bc[2 * axis + 1] = I.BC_TRANSMISSIVE
    p = grey_params(bc=bc)
    U = np.zeros((1, *shape, 4))
    i = np.arange(nlong)
    prof = np.where((i >= 24) & (i < 40), 1.0, 0.0)
    sh = [1, 1, 1]
    sh[2 - axis] = nlong
    U[0, ..., 0] = prof.reshape(sh)
    U[0, ..., 1 + axis] = sign * U[0, ..., 0]
    lam = O.courant_number(p, 1e20)
    steps = 20

    def centroid(V):
        w = V[0, ..., 0].sum(axis=tuple(a for a in range(3) if a != 2 - axis))
        return (w * i).sum() / w.sum(), w.sum()

    c0, s0 = centroid(U)
    for _ in range(steps):
        U = O.transport(p, U, lam)
    c1, s1 = centroid(U)
    assert c1 - c0 == pytest.approx(sign * steps * lam, rel=1e-12, abs=0)
    assert s1 == pytest.approx(s0, rel=1e-14, abs=0)
    np.testing.assert_array_equal(U[0, ..., 1 + axis], sign * U[0, ..., 0])


def test_photon_and_flux_conservation_periodic():
    p = grey_params(G=1)
    U = I.random_realizable_state((5, 6, 8), 1, 7)
    s0 = U.reshape(-1, 4).sum(axis=0)
    for _ in range(1000):
        U = O.transport(p, U, 0.3)
    s1 = U.reshape(-1, 4).sum(axis=0)
    assert abs(s1[0] - s0[0]) <= 1e-12 * abs(s0[0])
    np.testing.assert_allclose(s1[1:], s0[1:], rtol=0, atol=1e-12 * abs(s0[0]))


@pytest.mark.parametrize("bc", [[0] * 6, [2, 1, 2, 1, 2, 1], [1] * 6])
def test_realizability_every_cell_every_step(bc):
    p = grey_params(G=1, bc=bc, isothermal=True, rates_const=True)
    U = I.random_realizable_state((6, 5, 7), 1, 13)
    xHI = np.full((6, 5, 7), 1.0)
    T = np.full((6, 5, 7), 1e4)
    n0 = np.full((6, 5, 7), 1e-3)
    r = O.run(p, U, xHI, T, n0, 1e20, 1.0, 200)
    assert r.nclamp == 0 and r.err == 0
    assert np.all(r.hist[:, 2] <= 1.0 + 1e-12)


def _permute(U, perm):
    """Permute spatial axes (x,y,z order perm) and the flux components."""
    # U[g, z, y, x, c]; perm maps new axis d -> old axis perm[d] (0=x)
    ax = [2 - perm[2], 2 - perm[1], 2 - perm[0]]
    V = np.transpose(U[..., :], (0, 1 + ax[0], 1 + ax[1], 1 + ax[2], 4)).copy()
    V[..., 1:] = V[..., [1 + perm[0], 1 + perm[1], 1 + perm[2]]]
    return V


def test_axis_permutation_symmetry():
    p = grey_params(G=1)
    U = I.random_realizable_state((4, 5, 6), 1, 21)
    out = O.transport(p, U, 0.3)
    for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)]:
        outp = O.transport(p, _permute(U, perm), 0.3)
        np.testing.assert_allclose(outp, _permute(out, perm), rtol=1e-13, atol=1e-15)


def test_reflection_symmetry_is_bitwise():
    p = grey_params(G=1)
    U = I.random_realizable_state((4, 5, 6), 1, 22)
    out = O.transport(p, U, 0.3)
    R = U[:, :, :, ::-1].copy()
    R[..., 1] = -R[..., 1]
    outR = O.transport(p, R, 0.3)
    E = out[:, :, :, ::-1].copy()
    E[..., 1] = -E[..., 1]
    np.testing.assert_array_equal(outR, E)


def _numpy_transport(U, lam, bc):
    """Independent brute force: pad with ghosts, textbook Levermore closure,
    GLF flux per face, unsplit sum (tiny grids only)."""
    G, nz, ny, nx, _ = U.shape
    out = np.empty_like(U)

    def Dmat(u):
        N = u[0]
        if N <= 0:
            return np.zeros((3, 3))
        fv = u[1:] / N
        f = min(np.linalg.norm(fv), 1.0)
        n = fv / np.linalg.norm(fv) if np.linalg.norm(fv) > 0 else np.zeros(3)
        chi = levermore_chi(f)
        return N * (0.5 * (1 - chi) * np.eye(3) + 0.5 * (3 * chi - 1) * np.outer(n, n))

    def flux(d, u):
        return np.r_[u[1 + d], Dmat(u)[d]]

    def cell(g, z, y, x, d, s):
        c = [x, y, z]
        n = [nx, ny, nz]
        c[d] += s
        if 0 <= c[d] < n[d]:
            return U[g, c[2], c[1], c[0]].copy()
        b = bc[2 * d + (1 if s > 0 else 0)]
        if b == 0:
            c[d] %= n[d]
            return U[g, c[2], c[1], c[0]].copy()
        u = U[g, z, y, x].copy()
        if b == 2:
            u[1 + d] = -u[1 + d]
        return u

    for g in range(G):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    u = U[g, z, y, x]
                    tot = np.zeros(4)
                    for d in range(3):
                        L, R = cell(g, z, y, x, d, -1), cell(g, z, y, x, d, +1)
                        Fp = 0.5 * (flux(d, u) + flux(d, R)) - 0.5 * (R - u)
                        Fm = 0.5 * (flux(d, L) + flux(d, u)) - 0.5 * (u - L)
                        tot += Fp - Fm
                    out[g, z, y, x] = u - lam * tot
    return out


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 3, 3), (4, 4, 4), (7, 5, 3)])
@pytest.mark.parametrize("bc", [[0] * 6, [2, 1, 2, 1, 2, 1], [1, 2, 0, 0, 2, 1]])
def test_bruteforce_tiny_grids(shape, bc):
    p = grey_params(G=2, bc=bc)
    U = I.random_realizable_state(shape, 2, hash((shape, tuple(bc))) & 0xFFFF)
    out = O.transport(p, U, 0.3)
    ref = _numpy_transport(U, 0.3, bc)
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- chemistry
def test_photoionisation_equilibrium_is_dtau_independent():
    """With constant sources, the fixed point of the semi-implicit update is
    the photo-ionisation equilibrium: per group c sig_i xHI n0 N_i = S_i and
    (alpha + beta) n0 x^2 - beta n0 x - nunit sum(S)/n0 = 0."""
    alpha, beta = 2.59e-13, 3e-15
    p = O.Params(sigN=[3e-18, 8e-19], sigE=[3e-18, 8e-19], Eavg=[3e-11, 5e-11],
                 frac=[0.7, 0.3], c=0.1 * C, isothermal=True, ots=True,
                 rates_const=True, alphaA=alpha, alphaB=alpha, beta=beta)
    n0, nunit = 2e-3, 1e-3
    S = np.array([3e-16, 1e-16])   # nunit per second; below the cell's recombination ceiling
    R = nunit * S.sum() / n0
    x_exp = (beta * n0 + math.sqrt((beta * n0) ** 2 + 4 * (alpha + beta) * n0 * R)) \
        / (2 * (alpha + beta) * n0)
    assert 0.0 < x_exp < 1.0
    for dt in [1e13, 1e14, 1e15, 1e16]:
        U = np.zeros((2, 4))
        xHI, T = 1.0 - 1.2e-3, 1e4
        for _ in range(20000):
            U, xHI, T, ncyc, err = O.chem_cell(p, dt, nunit, n0, S, U, xHI, T)
            assert err == 0 and ncyc == 1
        assert 1.0 - xHI == pytest.approx(x_exp, rel=1e-10, abs=0)
        Nexp = S / (p.c * np.array(p.sigN) * xHI * n0)
        np.testing.assert_allclose(U[:, 0], Nexp, rtol=1e-10)


def test_pure_recombination_converges_at_first_order():
    """N = 0, beta = 0, T fixed: dx/dt = -alpha n0 x^2, 1/x(t) = 1/x0 + alpha n0 t."""
    alpha, n0 = 4e-13, 1.0
    x0, t = 0.9, 2.0 / (alpha * n0)
    exact = 1.0 / (1.0 / x0 + alpha * n0 * t)
    errs = []
    for k in range(4, 10):
        p = grey_params(G=1, sig=1e-18, isothermal=True, rates_const=True,
                        alphaA=alpha, alphaB=alpha, beta=0.0, ots=True, nsub=2 ** k)
        U, xHI, T, ncyc, err = O.chem_cell(p, t, 1.0, n0, [0.0], np.zeros(4), 1 - x0, 1e4)
        assert ncyc == 2 ** k and err == 0
        errs.append(abs((1 - xHI) - exact))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.1), ratios
    assert errs[-1] < 2e-3 * exact


def _ode_reference(p, nunit, n0, S, U0, xHI0, T0, t):
    """The continuous thermochemistry ODEs of Sec. 2.2.4 (Eqs. e:therm1g,
    e:therm2g, e:therm3, e:therm4 with e:g2, e:g3), integrated by scipy at
    tight tolerance.  Rate coefficients are the oracle's fit functions (the
    library primitives of this check); everything else is written here."""
    from scipy.integrate import solve_ivp
    kB, eV = 1.380649e-16, 1.602176634e-12
    G = p.G
    sigN, sigE, Eavg = map(np.asarray, (p.sigN, p.sigE, p.Eavg))
    SigE = sigE * Eavg - sigN * 13.6 * eV

    def T_of(xHI, e):
        return e / (1.5 * (2.0 - xHI) * n0 * kB)

    def rhs(_, y):
        N = y[:G]
        F = y[G:4 * G].reshape(G, 3)
        xHI, e = y[4 * G], y[4 * G + 1]
        x = 1.0 - xHI
        T = T_of(xHI, e)
        aA, aB, be = O.rate("alphaA", T), O.rate("alphaB", T), O.rate("beta", T)
        alpha = aB if p.ots else aA
        kap = p.c * sigN * xHI * n0
        dN = S - kap * N
        if not p.ots:
            dN[0] += (aA - aB) * x * x * n0 * n0 / nunit
        dF = -kap[:, None] * F
        dxHI = alpha * x * x * n0 - be * x * xHI * n0 - xHI * np.sum(p.c * sigN * nunit * N)
        de = p.c * xHI * n0 * np.sum(SigE * nunit * N) - O.cooling(p, n0, xHI, T)
        return np.r_[dN, dF.ravel(), dxHI, de]

    e0 = 1.5 * (2.0 - xHI0) * n0 * kB * T0
    y0 = np.r_[U0[:, 0], U0[:, 1:].ravel(), xHI0, e0]
    sol = solve_ivp(rhs, [0, t], y0, method="Radau", rtol=1e-11, atol=1e-30)
    y = sol.y[:, -1]
    return y[:G], y[G:4 * G].reshape(G, 3), y[4 * G], T_of(y[4 * G], y[4 * G + 1])


def test_chemistry_converges_to_the_continuous_equations():
    """Strong photo-heating (T 8000 K -> 1.5e4 K) and photo-ionisation
    (xHI 0.6 -> 0.07) of a 2-group cell with sources and recombination
    photons: the sub-cycled update converges at first order to the solution
    of the continuous equations once the sub-steps are small enough that the
    10% rule no longer halves them."""
    gt = O.group_table(I.GROUPS_2, 5e4)
    p = O.Params(sigN=gt["sigN"], sigE=gt["sigE"], Eavg=gt["Eavg"], frac=gt["frac"],
                 c=0.1 * C, ots=False)
    n0, nunit = 3e-3, 1e-3
    S = np.array([1.5e-11, 4e-12])
    U0 = np.array([[2.0, 0.3, -0.2, 0.5], [1.0, 0.0, 0.4, 0.1]])
    xHI0, T0 = 0.6, 8000.0
    t = 1e11
    N_ref, F_ref, x_ref, T_ref = _ode_reference(p, nunit, n0, S, U0, xHI0, T0, t)
    assert T_ref > 1.8 * T0 and x_ref < 0.15 * xHI0
    errs = []
    for k in range(6, 10):
        p.nsub = 2 ** k
        U, xHI, T, ncyc, err = O.chem_cell(p, t, nunit, n0, S, U0, xHI0, T0)
        assert err == 0 and ncyc == 2 ** k
        e = max(abs(xHI - x_ref) / x_ref, abs(T - T_ref) / T_ref,
                np.max(np.abs(U[:, 0] - N_ref) / N_ref),
                np.max(np.abs(U[:, 1:] - F_ref)) / np.max(np.abs(F_ref)))
        errs.append(e)
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 1.9) & (ratios < 2.1)), (errs, ratios)
    assert errs[-1] < 1e-2


def test_adaptive_step_obeys_ten_percent_rule_and_tracks_ode():
    gt = O.group_table(I.GROUPS_1, 5e4)
    p = O.Params(sigN=gt["sigN"], sigE=gt["sigE"], Eavg=gt["Eavg"], frac=gt["frac"],
                 c=0.1 * C, ots=True)
    n0, nunit = 1e-3, 1e-3
    S = np.array([0.0])
    U0 = np.array([[5.0, 0.0, 0.0, 0.0]])
    xHI0, T0, t = 1.0 - 1.2e-3, 100.0, 6e10
    N_ref, F_ref, x_ref, T_ref = _ode_reference(p, nunit, n0, S, U0, xHI0, T0, t)
    U, xHI, T, ncyc, err = O.chem_cell(p, t, nunit, n0, S, U0, xHI0, T0)
    assert err == 0 and ncyc > 10
    # each accepted sub-step changes e by at most 10%, so T cannot have
    # grown faster than 1.1^ncyc, and the result follows the ODE closely
    assert T <= T0 * 1.1 ** ncyc * (2.0 - xHI0) / (2.0 - xHI)
    assert T == pytest.approx(T_ref, rel=0.1, abs=0)
    assert xHI == pytest.approx(x_ref, rel=0.3, abs=0)   # the 10% rule controls e, not x


def test_isothermal_keeps_temperature_bitwise():
    p = grey_params(G=1, sig=2e-18, isothermal=True)
    U, xHI, T, ncyc, err = O.chem_cell(p, 1e12, 1e-3, 1e-3, [1e-8], np.zeros(4), 0.9, 12345.678)
    assert T == 12345.678 and ncyc == 1


def test_photon_budget_with_sources_and_no_absorber():
    """sigma = 0, periodic box: total photons grow by exactly sum(Q) dt per step."""
    p = grey_params(G=2, sig=0.0, isothermal=True, rates_const=True)
    p.frac = [0.25, 0.75]
    shape = (6, 7, 5)
    U = I.random_realizable_state(shape, 2, 5) * 1e-3
    dx, nunit = 3e20, 2e-6
    cells = np.array([0, 17, 17, 100], dtype=np.int64)
    Q = np.array([1e48, 2e49, 3e47, 5e48])
    S = O.source_field(p, shape, cells, Q, dx, nunit)
    r = O.run(p, U, np.ones(shape), np.full(shape, 1e4), np.full(shape, 1e-3), dx, nunit,
              50, S)
    dt = O.timestep(p, dx)
    ph0 = U[..., 0].sum() * nunit * dx ** 3
    expected = ph0 + Q.sum() * dt * np.arange(1, 51)
    np.testing.assert_allclose(r.hist[:, 1], expected, rtol=1e-12)


# ---------------------------------------------------------------- rates, groups
# Osterbrock & Ferland (2006), "Astrophysics of Gaseous Nebulae and Active
# Galactic Nuclei", 2nd ed., Table 2.1: H I recombination coefficients, cm^3/s.
OSTERBROCK_T = [5000.0, 10000.0, 20000.0]
OSTERBROCK_ALPHA_A = [6.82e-13, 4.18e-13, 2.51e-13]
OSTERBROCK_ALPHA_B = [4.54e-13, 2.59e-13, 1.43e-13]


def test_recombination_rates_against_textbook():
    for T, aA, aB in zip(OSTERBROCK_T, OSTERBROCK_ALPHA_A, OSTERBROCK_ALPHA_B):
        assert O.rate("alphaB", T) == pytest.approx(aB, rel=0.01, abs=0)
        assert O.rate("alphaA", T) == pytest.approx(aA, rel=0.04, abs=0)
        assert O.rate("alphaA", T) > O.rate("alphaB", T)


def test_rates_physical_shape():
    Ts = np.logspace(2, 8, 61)
    aB = np.array([O.rate("alphaB", T) for T in Ts])
    be = np.array([O.rate("beta", T) for T in Ts[Ts < 1e6]])
    assert np.all(np.diff(aB) < 0)                   # recombination slows when hot
    assert np.all(np.diff(be[be > 0]) > 0)           # collisional ionisation grows
    assert O.rate("beta", 1e4) < 1e-2 * O.rate("alphaB", 1e4)
    for name in O.RATE_NAMES:
        v = np.array([O.rate(name, T) for T in Ts])
        assert np.all(np.isfinite(v)) and np.all(v >= 0)


def test_hydrogenic_cross_section():
    assert O.sigma_HI(13.6) == 6.30e-18
    assert O.sigma_HI(13.5) == 0.0
    E = np.logspace(np.log10(13.6 * (1 + 1e-9)), 5, 400)
    s = np.array([O.sigma_HI(e) for e in E])
    assert np.all(np.diff(s) < 0)
    slope = math.log(O.sigma_HI(2e9) / O.sigma_HI(1e9)) / math.log(2.0)
    assert slope == pytest.approx(-3.5, abs=0.01)    # 1s photo-ionisation ~ E^-7/2


def _bose_tail(xa):
    """int_xa^inf x^2/(e^x - 1) dx by its convergent series."""
    k = np.arange(1, 400)
    return np.sum(np.exp(-k * xa) * (xa * xa / k + 2 * xa / k ** 2 + 2 / k ** 3))


def test_group_quadrature_against_closed_forms():
    kT = 1.380649e-16 * 5e4 / 1.602176634e-12
    zeta3 = 1.2020569031595942
    # whole spectrum, sigma = 1: <E> = pi^4/(30 zeta(3)) kT
    t = O.group_table([1e-4 * kT, 80 * kT], 5e4, use_sigma=False)
    assert t["Eavg"][0] / 1.602176634e-12 == pytest.approx(math.pi ** 4 / (30 * zeta3) * kT, rel=1e-7, abs=0)
    assert t["sigN"][0] == pytest.approx(1.0, rel=1e-14, abs=0)
    # photon fraction split at a and b
    edges = [13.6, 24.6, 54.4, 1000.0]
    t = O.group_table(edges, 5e4, use_sigma=False)
    tails = [_bose_tail(e / kT) for e in edges]
    fr = np.array([tails[i] - tails[i + 1] for i in range(3)])
    np.testing.assert_allclose(t["frac"], fr / fr.sum(), rtol=1e-11)


def test_group_table_structure():
    for Tbb, edges in [(1e5, I.GROUPS_1), (5e4, I.GROUPS_3), (5e4, I.GROUPS_2)]:
        t = O.group_table(edges, Tbb)
        assert t["frac"].sum() == pytest.approx(1.0, rel=1e-15, abs=0)
        assert np.all(np.diff(t["sigN"]) < 0)        # harder groups absorb less
        for i in range(len(edges) - 1):
            lo, hi = edges[i] * 1.602176634e-12, edges[i + 1] * 1.602176634e-12
            assert lo < t["Eavg"][i] < hi
            assert O.sigma_HI(edges[i + 1]) < t["sigN"][i] < O.sigma_HI(edges[i])
            assert t["sigE"][i] < t["sigN"][i]       # sigma falls with energy


def test_step_cells_is_the_full_step_on_those_cells():
    """The sampled-cell step used by the large-grid GPU checks reproduces the
    oracle's full step bit for bit on the cells it evaluates."""
    w = I.reion(n=20, steps=5, nsrc=6)
    t = O.group_table(w.edges_eV, w.T_bb)
    t = {k: I.f32(v) for k, v in t.items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 bc=[2, 1, 0, 0, 1, 1])
    box = w.boxes[0]
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, x, T = box.initial_state(3)
    r = O.run(p, U, x, T, box.n0, box.dx, nunit, 4, S)
    full = O.run(p, r.U, r.xHI, r.T, box.n0, box.dx, nunit, 1, S)
    cells = np.array([0, 19, 380, 399, 7999, 4210, int(box.src_cells[0])], dtype=np.int64)
    Uo, xo, To, err = O.step_cells(p, r.U, r.xHI, r.T, box.n0, box.dx, nunit, cells, S)
    assert err == 0
    np.testing.assert_array_equal(Uo, full.U.reshape(3, -1, 4)[:, cells, :].transpose(1, 0, 2))
    np.testing.assert_array_equal(xo, full.xHI.reshape(-1)[cells])
    np.testing.assert_array_equal(To, full.T.reshape(-1)[cells])


def test_box_parallel_oracle_runs_are_the_same_bits():
    """The test harness may run an ensemble's boxes side by side (one
    single-threaded oracle call per core); the results must be the bits of
    the sequential multi-threaded runs."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from _harness import run_oracle
    w = I.ensemble(nboxes=4, steps=3, sides=(8, 12), seed=5)
    a = run_oracle(w, 3, threads=3)
    b = run_oracle(w, 3, box_parallel=True)
    for x, y in zip(a, b):
        for u, v in zip(x[:4], y[:4]):
            np.testing.assert_array_equal(u, v)
        assert x[4:] == y[4:]
