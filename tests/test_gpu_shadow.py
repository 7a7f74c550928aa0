"""GPU inflow boundary and the static-gas clump (shadow) test of Sec. 6.5.

* parity of the small clump box against the oracle, GLF and HLL, every form
  (FP64 and strict <= 1e-9, split x_HI and T <= 1e-3);
* an empty box with inflow fills with the uniform beam;
* the 64^3 clump box: the plane I-front sweeps the background, the dense
  clump traps it and casts a shadow behind it, sharper with HLL than with
  GLF (the paper's remark on GLF's weak shadows)."""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import field_errors, linf_rel, make_solver, run_gpu, run_oracle, tables

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "strict", "split"])
def test_small_clump_parity(flux, prec):
    """150 steps of the 24^3 clump box.  GLF: every field element-wise as
    elsewhere.  HLL amplifies rounding-sized differences in the faint cells
    ahead of the front (the oracle against itself, 1e-15 perturbation: ~1e-3
    there after 90 steps, the gas state 1e-9), so its runs are compared
    normwise and its steps element-wise in test_clump_hll_one_step_parity."""
    w = I.shadow(n=24, steps=150)
    ora = run_oracle(w, 150, flux=flux)[0]
    assert ora[4] == 0
    (gpu,), st = run_gpu(w, 150, prec, flux=flux)
    assert gpu[4] == B.RT_OK
    if prec == "split":
        ex, eT = linf_rel(gpu[1], ora[1]), linf_rel(gpu[2], ora[2])
        print("split clump errors", flux, ex, eT)
        # HLL carries the FP32 transport's 1e-7 through its amplification
        tol_x, tol_T = (1e-3, 1e-3) if flux == 0 else (1e-3, 1e-2)
        assert ex <= tol_x and eT <= tol_T, (ex, eT)
        if flux == 0:
            # the FP32 transport's radiation, element-wise (floored relative)
            err = field_errors(gpu, ora, 3)
            assert max(err[k] for k in err if k[0] in "NF") <= 1e-4, err
        else:
            # HLL, normwise: the flux amplifies the FP32 transport's rounding
            # in the faint cells ahead of the front (the oracle against itself
            # takes a 1e-15 perturbation to ~1e-3 there), so over 150 steps
            # the radiation bar is the conditioning's, not 1e-4 (measured
            # 3.7e-4 in group 1, 2.1e-3 in group 2); its one-step error is
            # held to 1e-4 element-wise in test_clump_hll_one_step_parity
            for g in range(3):
                scale = np.max(np.abs(ora[0][g, ..., 0]))
                eN = np.max(np.abs(gpu[0][g] - ora[0][g])) / scale
                assert eN <= 1e-2, (g, eN)
    elif flux == 0:
        err = field_errors(gpu, ora, 3)
        assert max(err.values()) <= 1e-9, err
    else:
        for g in range(3):
            scale = np.max(np.abs(ora[0][g, ..., 0]))
            eN = np.max(np.abs(gpu[0][g] - ora[0][g])) / scale
            assert eN <= 1e-5, (g, eN)
        ex, eT = linf_rel(gpu[1], ora[1]), linf_rel(gpu[2], ora[2])
        assert ex <= 1e-6 and eT <= 1e-6, (ex, eT)
    assert np.min(ora[1]) < 0.5                     # the front entered


@pytest.mark.parametrize("prec", ["fp64", "strict", "split"])
def test_clump_hll_one_step_parity(prec):
    """HLL, one step from the same state (the oracle's after 100 steps): every
    element against the oracle."""
    w = I.shadow(n=24, steps=100)
    box = w.boxes[0]
    ora = run_oracle(w, 100, flux=1)[0]
    st = [(ora[0], ora[1], ora[2])]
    one = run_oracle(w, 1, None, st, flux=1)[0]
    (gpu,), _ = run_gpu(w, 1, prec, None, st, flux=1)
    assert gpu[4] == B.RT_OK
    err = field_errors(gpu, one, 3)
    assert max(err.values()) <= (1e-4 if prec == "split" else 1e-12), err


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_empty_box_fills_with_the_inflow_beam(prec):
    n = 16
    box = I.Box(n0=np.full((n, n, n), 1e-3), src_cells=np.zeros(0, dtype=np.int64),
                src_Q=np.zeros(0), T0=1e4)
    w = I.Workload(name="beam", boxes=[box], edges_eV=I.GROUPS_2, T_bb=1e5, c_frac=0.1,
                   steps=400, isothermal=True, rates_const=True,
                   bc=[I.BC_INFLOW, I.BC_TRANSMISSIVE] + [I.BC_PERIODIC] * 4,
                   inflow=[2e6, 0, 0, 0, 0, 0])
    to, tp = tables(w)
    (gpu,), _ = run_gpu(w, 400, prec, tp, sigN=[0.0, 0.0])
    rho = O.inflow_density(2e6, tp["frac"], w.c_red, w.nunit(box))
    tol = 1e-5 if prec == "split" else 1e-12
    for g in range(2):
        np.testing.assert_allclose(gpu[0][g, ..., 0], rho[g], rtol=tol)
        np.testing.assert_allclose(gpu[0][g, ..., 1], rho[g], rtol=tol)


def test_clump_casts_a_sharper_shadow_with_hll():
    w = I.shadow(n=64)
    res = {}
    for flux in (0, 1):
        (gpu,), st = run_gpu(w, 3000, "split", flux=flux)
        assert gpu[4] == B.RT_OK
        res[flux] = gpu[1]                               # xHI [z, y, x]
    n = 64
    c = np.arange(n) + 0.5
    Z, Y = np.meshgrid(c, c, indexing="ij")
    r_yz = np.hypot(Y - 32.0, Z - 32.0)
    behind = (r_yz < 5.0)                                # the clump's shadow (radius 7.8 cells)
    aside = (r_yz > 14.0)
    out = {}
    for flux, xHI in res.items():
        far = xHI[:, :, 61:].mean(axis=2)                # planes behind the clump (x > 6.3 kpc)
        assert np.median(far[aside]) < 0.05, flux        # the front swept past the clump
        clump_core = xHI[29:35, 29:35, 50:55]
        assert clump_core.min() > 0.5, flux              # the dense clump holds the front
        out[flux] = float(np.mean(far[behind]))
    print("mean neutral fraction in the shadow: GLF", out[0], "HLL", out[1])
    assert out[1] > 0.5                                  # HLL keeps the shadow neutral
    assert out[1] > out[0] + 0.1                         # GLF's shadow is weaker
