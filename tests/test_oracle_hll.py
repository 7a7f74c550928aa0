"""Pins of the oracle's HLL flux (the less diffusive flux the paper plans,
Sec. 2.2.3): Harten-Lax-van Leer with the extreme eigenvalues of the M1 flux
Jacobian, tabulated in (z = sqrt(1 - f), mu) and interpolated bilinearly.

* the speed table against closed forms: the isotropic limit f = 0 (the
  Jacobian of (F, N/3) has eigenvalues +-1/sqrt(3)), the flux parallel to
  the face normal (the 1-D M1 system's eigenvalues and the transverse
  speed), free streaming f = 1 (every speed equals mu);
* the speed table against eigenvalues of a finite-difference Jacobian;
* the flux: consistency Phi(U, U) = G(U), exact upwinding of a beam,
  reflection symmetry;
* the transport: uniform fixed point, conservation, a beam moving at c,
  realizability, and less lateral spreading than GLF (the paper's reason
  for wanting it: sharper shadows).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I

C = I.C_LIGHT


def params(G=1, flux=O.FLUX_HLL, **kw):
    return O.Params(sigN=[0.0] * G, sigE=[0.0] * G, Eavg=[20 * 1.602176634e-12] * G,
                    frac=[1.0 / G] * G, c=0.1 * C, flux=flux, **kw)


def chi(f):
    return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * math.sqrt(4.0 - 3.0 * f * f))


def test_isotropic_row_is_one_over_sqrt3():
    t = O.hll_speed_table(64, 64)
    np.testing.assert_allclose(t[64, :], 1.0 / math.sqrt(3.0), rtol=1e-12)


def test_free_streaming_row_is_mu():
    t = O.hll_speed_table(64, 64)
    np.testing.assert_array_equal(t[0, :], -1.0 + 2.0 * np.arange(65) / 64)
    # and the eigenvalues of f -> 1 do converge there (splitting ~ sqrt(1 - f))
    for mu in (-0.6, 0.2, 0.9):
        ev = np.linalg.eigvals(O.flux_jacobian_fmu(1.0 - 1e-8, mu)).real
        assert np.max(np.abs(ev - mu)) < 1e-3


@pytest.mark.parametrize("i", [1, 5, 16, 40, 63])
def test_normal_flux_column_matches_the_1d_system(i):
    """F along the normal: the (N, F_n) block is the 1-D M1 system with
    P = chi(f) N, eigenvalues (chi' +- sqrt(chi'^2 + 4 (chi - f chi')))/2;
    the two transverse modes move at g f with g = (3 chi - 1)/(2 f^2)."""
    t = O.hll_speed_table(64, 64)
    f = 1.0 - (i / 64) ** 2
    h = 1e-6
    dchi = (chi(f + h) - chi(f - h)) / (2 * h) if f + h <= 1 else (chi(f) - chi(f - 2 * h)) / (2 * h)
    disc = math.sqrt(dchi * dchi + 4.0 * (chi(f) - f * dchi))
    lp, lm = (dchi + disc) / 2, (dchi - disc) / 2
    gt = (3.0 * chi(f) - 1.0) / (2.0 * f)
    assert t[i, 64] == pytest.approx(max(lp, gt), rel=1e-7, abs=0)           # mu = +1
    assert t[i, 0] == pytest.approx(-min(lm, gt), rel=1e-7, abs=0)           # mu = -1


def test_speed_table_against_finite_difference_jacobians():
    t = O.hll_speed_table(64, 64)
    rng = np.random.default_rng(3)
    for _ in range(40):
        i, j = rng.integers(1, 64), rng.integers(0, 65)
        f, mu = 1.0 - (i / 64) ** 2, -1.0 + 2.0 * j / 64
        U = np.array([1.0, f * mu, f * math.sqrt(max(0.0, 1 - mu * mu)), 0.0])
        J = np.zeros((4, 4))
        for m in range(4):
            h = 1e-6
            up, um = U.copy(), U.copy()
            up[m] += h
            um[m] -= h
            J[:, m] = (O.glf_flux(0, up, up) - O.glf_flux(0, um, um)) / (2 * h)
        assert np.max(np.linalg.eigvals(J).real) == pytest.approx(t[i, j], abs=1e-6)


def test_flux_consistency_and_beam_upwinding():
    p = params()
    rng = np.random.default_rng(5)
    for _ in range(50):
        N = rng.uniform(0.1, 3)
        F = rng.standard_normal(3)
        F *= N * rng.uniform(0, 0.99) / np.linalg.norm(F)
        U = np.r_[N, F]
        for d in range(3):
            np.testing.assert_allclose(O.face_flux(p, d, U, U), O.glf_flux(d, U, U), rtol=1e-13,
                                       atol=1e-15 * N)
    # a beam F = N along +x entering vacuum: the flux is the beam's own state
    for N in (1.0, 1e-20, 3.5e10):
        L = np.array([N, N, 0.0, 0.0])
        np.testing.assert_allclose(O.face_flux(p, 0, L, np.zeros(4)), L, rtol=1e-15)
        np.testing.assert_allclose(O.face_flux(p, 0, L, 0.5 * L), L, rtol=1e-15)


def test_flux_reflection_symmetry():
    p = params()
    rng = np.random.default_rng(6)
    flip = np.array([1, -1, 1, 1])
    for _ in range(30):
        L, R = [np.r_[n, rng.uniform(-0.5, 0.5, 3) * n] for n in rng.uniform(0.1, 2, 2)]
        a = O.face_flux(p, 0, L, R)
        b = O.face_flux(p, 0, R * flip, L * flip)
        np.testing.assert_allclose(a, -b * flip, rtol=1e-12, atol=1e-15)


def test_uniform_field_is_a_fixed_point():
    p = params(G=2)
    U = np.empty((2, 5, 6, 7, 4))
    U[0, ..., :] = [1.3, 0.2, -0.5, 0.7]
    U[1, ..., :] = [0.4, 0.0, 0.0, 0.3]
    np.testing.assert_array_equal(O.transport(p, U, 0.3), U)


def test_conservation_periodic():
    p = params()
    U = I.random_realizable_state((5, 6, 8), 1, 7)
    s0 = U.reshape(-1, 4).sum(axis=0)
    for _ in range(1000):
        U = O.transport(p, U, 0.3)
    s1 = U.reshape(-1, 4).sum(axis=0)
    assert abs(s1[0] - s0[0]) <= 1e-12 * abs(s0[0])
    np.testing.assert_allclose(s1[1:], s0[1:], rtol=0, atol=1e-12 * abs(s0[0]))


@pytest.mark.parametrize("sign", [1, -1])
def test_beam_moves_at_c(sign):
    nlong = 64
    p = params(bc=[I.BC_TRANSMISSIVE, I.BC_TRANSMISSIVE] + [I.BC_PERIODIC] * 4)
    U = np.zeros((1, 2, 2, nlong, 4))
    i = np.arange(nlong)
    U[0, ..., 0] = np.where((i >= 24) & (i < 40), 1.0, 0.0)
    U[0, ..., 1] = sign * U[0, ..., 0]
    lam = O.courant_number(p, 1e20)
    w0 = U[0, ..., 0].sum(axis=(0, 1))
    c0 = (w0 * i).sum() / w0.sum()
    for _ in range(20):
        U = O.transport(p, U, lam)
    w1 = U[0, ..., 0].sum(axis=(0, 1))
    assert (w1 * i).sum() / w1.sum() - c0 == pytest.approx(sign * 20 * lam, rel=1e-12, abs=0)
    assert w1.sum() == pytest.approx(w0.sum(), rel=1e-14, abs=0)
    np.testing.assert_allclose(U[0, ..., 1], sign * U[0, ..., 0], rtol=1e-15, atol=0)


@pytest.mark.parametrize("bc", [[0] * 6, [2, 1, 2, 1, 2, 1], [1] * 6])
def test_realizability(bc):
    p = params(bc=bc, isothermal=True, rates_const=True)
    shape = (6, 5, 7)
    U = I.random_realizable_state(shape, 1, 13)
    r = O.run(p, U, np.ones(shape), np.full(shape, 1e4), np.full(shape, 1e-3), 1e20, 1.0, 200)
    assert r.nclamp == 0 and r.err == 0


def test_narrow_beam_spreads_less_than_with_glf():
    """A beam one cell wide in y (F = N along +x) crossing vacuum: the
    transverse second moment after 60 steps, HLL well below GLF."""
    shape = (1, 33, 96)
    bc = [I.BC_TRANSMISSIVE, I.BC_TRANSMISSIVE, I.BC_PERIODIC, I.BC_PERIODIC,
          I.BC_PERIODIC, I.BC_PERIODIC]
    out = {}
    for flux in (O.FLUX_GLF, O.FLUX_HLL):
        p = params(flux=flux, bc=bc)
        U = np.zeros((1, *shape, 4))
        U[0, 0, 16, 4:20, 0] = 1.0
        U[0, 0, 16, 4:20, 1] = 1.0
        lam = O.courant_number(p, 1e20)
        for _ in range(60):
            U = O.transport(p, U, lam)
        w = U[0, 0, :, :, 0].sum(axis=1)
        y = np.arange(shape[1]) - 16
        out[flux] = (w * y * y).sum() / w.sum()
    assert out[O.FLUX_HLL] < 0.5 * out[O.FLUX_GLF], out


def test_library_table_matches_the_oracle():
    """The library's wave-speed table (its own Jacobian by forward-mode
    differentiation, the decoupled transverse mode taken out, Newton on the
    remaining cubic) against the oracle's (its Jacobian, numpy eigenvalues):
    two independent computations of the same numbers (no GPU needed)."""
    from paper_1508_07888_b300 import binding as B
    np.testing.assert_allclose(B.rt_hll_speeds(64, 64), O.hll_speed_table(64, 64), rtol=0,
                               atol=2e-12)


def test_beam_stays_realizable_under_rounding_noise():
    """Rounding leaves beam cells with |F| slightly above cN; with the speeds
    mu of f = 1 the HLL update would amplify that excess step after step.
    With the limiter a beam entering an absorbing clump stays realizable
    when every step's state is perturbed at the 1e-13 level."""
    w = I.shadow(n=12, steps=60)
    box = w.boxes[0]
    t = {k: I.f32(v) for k, v in O.group_table(w.edges_eV, w.T_bb).items()}
    nunit = w.nunit(box)
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 bc=list(w.bc), flux=O.FLUX_HLL,
                 inflow=[O.inflow_density(w.inflow[f], t["frac"], w.c_red, nunit)
                         for f in range(6)])
    U, x, T = box.initial_state(3)
    rng = np.random.default_rng(1)
    for _ in range(60):
        r = O.run(p, U, x, T, box.n0, box.dx, nunit, 1, None)
        assert r.err == 0
        U = r.U * (1 + 1e-13 * rng.standard_normal(r.U.shape))
        x, T = r.xHI, r.T
        N, F = U[..., 0], np.linalg.norm(U[..., 1:], axis=-1)
        assert np.all(F <= N * (1 + 1e-12) + 1e-300)
