"""Pins of the oracle's hand-written adjoint (reverse mode of the step, with
the branch decisions of the forward pass frozen) against central finite
differences of the oracle's own forward functions.

Each check is a dot-product identity <w, J v> = <J^T w, v> with random v, w:
J v comes from differencing the forward map, J^T w from the adjoint, so a
wrong sign, a dropped term or a transposed index in the adjoint fails it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I

C = I.C_LIGHT


def params(G=2, **kw):
    t = O.group_table((13.6, 24.6, 54.4, 1000.0)[: G + 1] if G < 3 else I.GROUPS_3, 5e4)
    base = dict(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=0.1 * C)
    base.update(kw)
    return O.Params(**base)


def test_flux_jacobian_against_differences():
    rng = np.random.default_rng(1)
    for trial in range(60):
        N = 10 ** rng.uniform(-3, 1)
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        f = rng.uniform(0.0, 0.98) if trial < 50 else rng.uniform(1.05, 1.3)   # clamp branch
        U = np.r_[N, f * N * n]
        for d in range(3):
            J = O.flux_jacobian(d, U)
            Jfd = np.zeros((4, 4))
            for m in range(4):
                h = 1e-6 * N
                up, um = U.copy(), U.copy()
                up[m] += h
                um[m] -= h
                Jfd[:, m] = (O.glf_flux(d, up, up) - O.glf_flux(d, um, um)) / (2 * h)
            np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-7)


def _cell_case(rng, p, iso=False):
    G = p.G
    U = np.zeros((G, 4))
    U[:, 0] = rng.uniform(0.5, 3.0, G)
    d = rng.standard_normal((G, 3))
    U[:, 1:] = d / np.linalg.norm(d, axis=1, keepdims=True) * (U[:, :1] * rng.uniform(0.1, 0.9, (G, 1)))
    return dict(U=U, xHI=rng.uniform(0.3, 0.9), T=1e4 if iso else rng.uniform(3e3, 2e4),
                n0=rng.uniform(1e-3, 4e-3), S=rng.uniform(0.0, 1e-11, G))


@pytest.mark.parametrize("kw", [dict(nsub=4), dict(nsub=4, ots=True), dict(nsub=2, G=1),
                                dict(nsub=3, G=3), dict(nsub=1, isothermal=True),
                                dict(nsub=1, isothermal=True, rates_const=True, alphaA=4e-13,
                                     alphaB=2.6e-13, beta=1e-15)])
def test_chemistry_adjoint_dot_product(kw):
    G = kw.pop("G", 2)
    p = params(G, **kw)
    rng = np.random.default_rng(len(kw) * 11 + G)
    dt, nunit = 3e10, 1e-3
    for _ in range(5):
        c = _cell_case(rng, p, iso=p.isothermal)
        w = dict(U=rng.standard_normal((G, 4)), xHI=rng.standard_normal(),
                 T=rng.standard_normal() * 1e-4)
        v = dict(U=rng.standard_normal((G, 4)), xHI=rng.standard_normal() * 1e-2,
                 T=0.0 if p.isothermal else rng.standard_normal() * 10.0,
                 n0=rng.standard_normal() * 1e-4, S=rng.standard_normal(G) * 1e-12)

        def fwd(eps):
            U1, x1, T1, ncyc, err = O.chem_cell(p, dt, nunit, c["n0"] + eps * v["n0"],
                                                c["S"] + eps * v["S"], c["U"] + eps * v["U"],
                                                c["xHI"] + eps * v["xHI"], c["T"] + eps * v["T"])
            assert err == 0
            return np.sum(w["U"] * U1) + w["xHI"] * x1 + w["T"] * T1

        h = 1e-6
        lhs = (fwd(h) - fwd(-h)) / (2 * h)
        bU, bx, bT, dn0, dS, n = O.chem_cell_adj(p, dt, nunit, c["n0"], c["S"], c["U"], c["xHI"],
                                                 c["T"], w["U"], w["xHI"], w["T"])
        rhs = (np.sum(bU * v["U"]) + bx * v["xHI"] + bT * v["T"] + dn0 * v["n0"]
               + np.sum(dS * v["S"]))
        assert rhs == pytest.approx(lhs, rel=2e-6, abs=1e-12 * (abs(lhs) + 1)), (lhs, rhs, n)


def test_transport_adjoint_dot_product():
    p = params(2)
    shape = (5, 6, 7)
    U = I.random_realizable_state(shape, 2, 3) * 0.9 + 0.05
    U[..., 1:] *= 0.8
    rng = np.random.default_rng(4)
    v = rng.standard_normal(U.shape)
    w = rng.standard_normal(U.shape)
    lam = 0.3
    h = 1e-6
    lhs = np.sum(w * (O.transport(p, U + h * v, lam) - O.transport(p, U - h * v, lam))) / (2 * h)
    rhs = np.sum(O.transport_adj(p, U, w, lam) * v)
    assert rhs == pytest.approx(lhs, rel=1e-7, abs=0)


def test_full_adjoint_against_run_differences():
    """Gradient of L = sum_t w_t X(t) with respect to the luminosities and the
    density, over a few steps of a small periodic box with sources."""
    p = params(2, nsub=2)
    shape = (6, 8, 10)
    rng = np.random.default_rng(7)
    n0 = I.f32(1e-3 * np.exp(0.5 * rng.standard_normal(shape)))
    dx = I.DX_REF
    nunit = 1e49 / (p.c * dx * dx)
    cells = np.array([5, 77, 300, 479], dtype=np.int64)
    Q = np.array([3e48, 1e49, 5e48, 2e48])
    U0 = np.zeros((2, *shape, 4))
    x0 = np.full(shape, 1 - 1.2e-3)
    T0 = np.full(shape, 100.0)
    steps = 6
    wts = rng.uniform(0.5, 1.5, steps)

    def loss(Qv, n0v):
        S = O.source_field(p, shape, cells, Qv, dx, nunit)
        r = O.run(p, U0, x0, T0, n0v, dx, nunit, steps, S)
        assert r.err == 0
        return float(np.dot(wts, r.hist[:, 0]))

    S = O.source_field(p, shape, cells, Q, dx, nunit)
    dS, dn0 = O.adjoint(p, U0, x0, T0, n0, dx, nunit, steps, wts, S)
    vol = dx ** 3
    dQ = np.array([sum(p.frac[i] * dS[i, c] for i in range(2)) for c in cells]) / (vol * nunit)
    for k in range(len(cells)):
        h = 1e-5 * Q[k]
        Qp, Qm = Q.copy(), Q.copy()
        Qp[k] += h
        Qm[k] -= h
        fd = (loss(Qp, n0) - loss(Qm, n0)) / (2 * h)
        assert dQ[k] == pytest.approx(fd, rel=1e-5, abs=0), (k, dQ[k], fd)
    for seed in range(2):
        v = np.random.default_rng(100 + seed).standard_normal(shape) * n0
        h = 1e-6
        fd = (loss(Q, n0 + h * v) - loss(Q, n0 - h * v)) / (2 * h)
        assert np.sum(dn0 * v.reshape(-1)) == pytest.approx(fd, rel=1e-5, abs=0)
