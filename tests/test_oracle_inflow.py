"""Pins of the oracle's inflow boundary (the clump test of Sec. 6.5 feeds a
photon flux through the x = 0 face; the ghost cell holds a beam F = cN along
the inward normal):

* photon accounting: into an empty box, exactly N_in c dt per face cell and
  step enters, for GLF and HLL alike, until the beam reaches the far face;
* the steady state of an empty box is the uniform beam N = N_in, F = c N_in;
* the incoming flux per group follows the source spectrum's fractions.
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I

C = I.C_LIGHT


def params(G=2, flux=O.FLUX_GLF, inflow=None, bc=None):
    frac = [0.7, 0.3][:G]
    p = O.Params(sigN=[0.0] * G, sigE=[0.0] * G, Eavg=[20 * 1.602176634e-12] * G, frac=frac,
                 c=0.1 * C, flux=flux,
                 bc=bc or [I.BC_INFLOW, I.BC_TRANSMISSIVE] + [I.BC_PERIODIC] * 4)
    if inflow is not None:
        p.inflow = inflow
    return p


@pytest.mark.parametrize("flux", [O.FLUX_GLF, O.FLUX_HLL])
def test_photons_enter_at_the_given_rate(flux):
    nunit = 2.0
    rho = O.inflow_density(3.0e6, [0.7, 0.3], 0.1 * C, nunit)
    p = params(flux=flux, inflow=[rho, [0, 0], [0, 0], [0, 0], [0, 0], [0, 0]])
    shape = (3, 4, 80)
    U = np.zeros((2, *shape, 4))
    lam = 0.3
    for k in range(1, 101):
        U = O.transport(p, U, lam)
        if k % 25 == 0:
            tot = U[..., 0].sum(axis=(1, 2, 3))
            np.testing.assert_allclose(tot, rho * lam * k * shape[0] * shape[1], rtol=1e-12)
    # photon number flux of the incoming beam: c N nunit = 3e6 /cm^2/s in total
    assert rho.sum() * 0.1 * C * nunit == pytest.approx(3.0e6, rel=1e-15, abs=0)
    np.testing.assert_allclose(rho / rho.sum(), [0.7, 0.3], rtol=1e-15)


def test_empty_box_fills_with_the_uniform_beam():
    rho = np.array([1.5, 0.25])
    p = params(inflow=[rho, [0, 0], [0, 0], [0, 0], [0, 0], [0, 0]])
    shape = (2, 3, 12)
    U = np.zeros((2, *shape, 4))
    for _ in range(400):
        U = O.transport(p, U, 0.3)
    for g in range(2):
        np.testing.assert_allclose(U[g, ..., 0], rho[g], rtol=1e-12)
        np.testing.assert_allclose(U[g, ..., 1], rho[g], rtol=1e-12)
        assert np.max(np.abs(U[g, ..., 2:])) <= 1e-14 * rho[g]


def test_inflow_on_the_far_face_points_inward():
    rho = np.array([2.0])
    p = params(G=1, inflow=[[0], rho, [0], [0], [0], [0]],
               bc=[I.BC_TRANSMISSIVE, I.BC_INFLOW] + [I.BC_PERIODIC] * 4)
    U = np.zeros((1, 2, 2, 30, 4))
    for _ in range(10):
        U = O.transport(p, U, 0.3)
    assert U[0, ..., -1, 0].min() > 0 and U[0, ..., 0, 0].max() == 0.0
    assert np.all(U[0, ..., 1] <= 0.0)
