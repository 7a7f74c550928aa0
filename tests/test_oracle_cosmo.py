"""Pins of the oracle's supercomoving run (Sec. 3: N~ = a^3 N r_s^3,
F~ = a^4 r_s^2 t_s F, dt~ = dt/(a^2 t_s); the state is the comoving N^, F^
and T~ = a^2 T, the chemistry runs in physical units at each step's a):

* no expansion at a = 1 is the static run, bit for bit;
* no expansion at a != 1 is the static run of the physical box
  (density n0/a^3, cell a dx, unit nunit/a^3, temperature T~/a^2);
* Einstein-de Sitter expansion follows a = (a0^1.5 + 1.5 H0 t)^(2/3);
* a free-streaming beam keeps its comoving photon number and its reduced
  flux f decays as a0/a (F~ / c~ with c~ ~ a);
* gas at rest with no radiation cools adiabatically, T ~ a^-2 (T~ constant).
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I

H0 = 2.2e-18          # s^-1 (about 68 km/s/Mpc)
H_FAST = 2.2e-15      # a toy rate, so that a few hundred steps expand the box severalfold


def _setup(n=10, nsrc=2):
    w = I.reion(n=n, steps=20, nsrc=nsrc, seed=51, lum_seed=52)
    box = w.boxes[0]
    t = {k: I.f32(v) for k, v in O.group_table(w.edges_eV, w.T_bb).items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 cfl=w.cfl, bc=list(w.bc))
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    return w, box, p, nunit, S


def test_no_expansion_at_a1_is_the_static_run():
    w, box, p, nunit, S = _setup()
    U, x, T = box.initial_state(w.ngroups)
    a = O.run(p, U, x, T, box.n0, box.dx, nunit, 20, S)
    b = O.run_cosmo(p, U, x, T, box.n0, box.dx, nunit, 20, S, 0.0, 0.3, 0.7, 1.0)
    assert b.a == 1.0
    for u, v in ((a.U, b.run.U), (a.xHI, b.run.xHI), (a.T, b.run.T)):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("a0", [0.5, 0.125])
def test_no_expansion_at_a_is_the_physical_box(a0):
    w, box, p, nunit, S = _setup()
    U, x, T = box.initial_state(w.ngroups)
    T_sc = T * a0 ** 2
    c = O.run_cosmo(p, U, x, T_sc, box.n0, box.dx, nunit, 20, S, 0.0, 0.3, 0.7, a0)
    # the physical box: the same stored numbers in the unit nunit/a^3
    ph = O.run(p, U, x, T, box.n0 / a0 ** 3, box.dx * a0, nunit / a0 ** 3, 20, S)
    np.testing.assert_allclose(c.run.U, ph.U, rtol=1e-11, atol=1e-14 * np.abs(ph.U).max())
    np.testing.assert_allclose(c.run.xHI, ph.xHI, rtol=1e-11)
    np.testing.assert_allclose(c.run.T / a0 ** 2, ph.T, rtol=1e-11)
    assert np.min(ph.xHI) < 0.9


def test_einstein_de_sitter_expansion():
    a, t = 0.1, 0.0
    for k in range(2000):
        dt = a * 3e12
        a = O.advance_a(a, dt, H_FAST, 1.0, 0.0)
        t += dt
    exact = (0.1 ** 1.5 + 1.5 * H_FAST * t) ** (2.0 / 3.0)
    assert a == pytest.approx(exact, rel=1e-10, abs=0)
    assert a > 0.3


def test_beam_in_expanding_space():
    p = O.Params(sigN=[0.0], sigE=[0.0], Eavg=[3.2e-11], frac=[1.0], c=0.1 * I.C_LIGHT,
                 isothermal=True, rates_const=True)
    shape = (2, 3, 4)
    U = np.zeros((1, *shape, 4))
    U[0, ..., 0] = 2.0
    U[0, ..., 1] = 2.0                        # f = 1 along x, uniform (periodic)
    x = np.ones(shape)
    T = np.full(shape, 1e4)
    dx = 3e22                                 # a large comoving cell: a long dt per step
    r = O.run_cosmo(p, U, x, T, np.full(shape, 1e-3), dx, 1.0, 300, None, H_FAST, 0.3, 0.7, 0.2)
    assert r.a > 0.3
    np.testing.assert_allclose(r.run.U[0, ..., 0], 2.0, rtol=1e-14)
    np.testing.assert_allclose(r.run.U[0, ..., 1], 2.0 * 0.2 / r.a, rtol=1e-12)


def test_adiabatic_cooling_of_gas_at_rest():
    p = O.Params(sigN=[6e-18], sigE=[3e-18], Eavg=[3.2e-11], frac=[1.0], c=0.1 * I.C_LIGHT)
    shape = (2, 2, 2)
    U = np.zeros((1, *shape, 4))
    x = np.full(shape, 1.0 - 1e-4)
    a0 = 0.1
    T_sc = np.full(shape, 500.0) * a0 ** 2             # physical 500 K at a0
    r = O.run_cosmo(p, U, x, T_sc, np.full(shape, 1e-7), 3e22, 1.0, 400, None, H_FAST, 1.0, 0.0, a0)
    assert r.a > 1.5 * a0 and r.run.err == 0
    # T~ is nearly constant (radiative cooling of 1e-7 cm^-3 gas is slow), so
    # the physical temperature fell as a^-2
    np.testing.assert_allclose(r.run.T, T_sc, rtol=1e-3)
    assert np.all(r.run.T / r.a ** 2 < 500.0 * (a0 / r.a) ** 2 * 1.001)
