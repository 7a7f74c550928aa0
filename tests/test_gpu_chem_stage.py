"""The chemistry stage alone (Sec. 2.2.4; rows a5-a8) from identical inputs.

A spatially uniform radiation field with periodic faces is a fixed point of
the transport: every face of the GLF update sees the same state on both
sides, so the flux differences vanish (exactly in the FP64 forms, to FP32
rounding in the split form's convex form).  One step from such a field is
then the sub-cycled chemistry of every cell on the same N, F, x_HI, T and n0
as the oracle's.  The cells span cold gas (below the 155 K cut of the rate
tables) to 1e5 K and neutral to ionised, on a lognormal density with
sources, in a box whose cell count leaves a ragged last work item.

* FP64 and strict forms: every field within 1e-9 of the oracle, the
  stage-wise bound of the FP64 chemistry.
* Split form: the photon update runs in FP32, the precision N and F are
  stored in, and x_HI, T, the rates and the sums in FP64; its fields are
  held to the FP32 rounding those inputs carry."""
import numpy as np
import pytest

from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import field_errors, run_gpu, run_oracle, tables

SHAPE = (10, 12, 14)                     # 1680 cells: 52 full 32-cell items and a ragged one


def _stage_workload(seed=11):
    n0 = I.f32(I.lognormal_field(SHAPE, 1.0, 2.0, seed))
    cells = I.densest_cells(n0, 4)
    Q = I.loguniform_lum(4, seed + 100)
    box = I.Box(n0=n0, src_cells=cells, src_Q=Q)
    w = I.Workload(name="chem_stage", boxes=[box], edges_eV=I.GROUPS_3, T_bb=5e4, c_frac=0.1,
                   steps=1)
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    G = w.ngroups
    U = np.zeros((G,) + SHAPE + (4,))
    for g, Ng in enumerate((0.3, 0.1, 0.02)):
        U[g, ..., 0] = Ng
        U[g, ..., 1:] = Ng * np.array([0.2, -0.1, 0.05])
    U = I.f32(U)
    xHI = np.where(rng.uniform(size=SHAPE) < 1.0 / 3.0, 1.0 - 1.2e-3,
                   10.0 ** rng.uniform(-6.0, 0.0, SHAPE))
    T = 10.0 ** rng.uniform(np.log10(50.0), 5.0, SHAPE)
    return w, [(U, xHI, T)]


def test_stage_inputs_cover_the_rate_regimes():
    w, st = _stage_workload()
    T = st[0][2]
    assert (T < 155.0).mean() > 0.1 and (T > 1e4).mean() > 0.2
    assert w.boxes[0].ncell % 32 != 0


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "strict", "split"])
def test_chemistry_stage_against_the_oracle(prec):
    w, st = _stage_workload()
    to, tp = tables(w)
    (ora,) = run_oracle(w, 1, to, st)
    assert ora[4] == 0
    (gpu,), stats = run_gpu(w, 1, prec, tp, st)
    assert gpu[4] == B.RT_OK
    err = field_errors(gpu, ora, w.ngroups)
    print("chemistry stage", prec, err)
    if prec == "split":
        # measured: N 2.0e-6, F 3.5e-7, x_HI 2.4e-6, T 2.6e-7 (floored relative)
        for g in range(w.ngroups):
            assert err[f"N{g}"] <= 1e-5 and err[f"F{g}"] <= 1e-5, err
        assert err["xHI"] <= 1e-5 and err["T"] <= 1e-5, err
    else:
        assert max(err.values()) <= 1e-9, err
    # the step's diagnostics: ionised fraction, photons, n(x_HI < 0.5), sub-cycles
    tol = 1e-9 if prec != "split" else 1e-5
    np.testing.assert_allclose(gpu[3][0, [0, 1, 4]], ora[3][0, [0, 1, 4]], rtol=tol)
    assert gpu[3][0, 3] == ora[3][0, 3]
