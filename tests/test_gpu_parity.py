"""GPU parity: the C-ABI library against the FP64 CPU oracle on the same
seeded inputs, element by element.

Tolerances (L-inf relative with a floor of 1e-6 of the field's maximum):
  RT_PREC_FP64_STRICT, constant rates  -> bit-identical
  RT_PREC_FP64 and strict with rate fits -> <= 1e-9 (chemistry), transport 1e-12
  RT_PREC_SPLIT (FP32 transport)       -> radiation fields <= 1e-4 after 100 steps
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import field_errors, linf_rel, make_solver, report, run_gpu, run_oracle, tables

pytestmark = pytest.mark.gpu


def _empty_workload(shape, G, bc, seed, c_frac=0.1):
    nz, ny, nx = shape
    box = I.Box(n0=np.full(shape, 1e-3), src_cells=np.zeros(0, dtype=np.int64),
                src_Q=np.zeros(0), T0=1e4)
    edges = (I.GROUPS_3 + (2000.0,))[:G + 1] if G <= 3 else (13.6, 24.6, 54.4, 200.0, 1000.0)
    w = I.Workload(name="transport", boxes=[box], edges_eV=edges, T_bb=5e4, c_frac=c_frac,
                   steps=3, isothermal=True, rates_const=True, bc=list(bc))
    U = I.f32(I.random_realizable_state(shape, G, seed))
    return w, [(U, np.full(shape, 1.0), np.full(shape, 1e4))]


SHAPES = [(1, 1, 1), (2, 3, 5), (7, 5, 3), (9, 33, 17), (8, 16, 64), (33, 9, 40)]
BCS = [[0] * 6, [2, 1, 2, 1, 2, 1], [1, 1, 0, 0, 2, 2]]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("G", [1, 3])
def test_transport_parity_ragged(shape, bc, G):
    """sigma = 0 and no sources: the chemistry leaves the radiation untouched,
    so three steps are three pure GLF transport steps."""
    w, st = _empty_workload(shape, G, bc, seed=sum(shape) * 7 + G)
    to, tp = tables(w)
    zero = [0.0] * G
    ora = run_oracle(w, 3, to, st, sigN=zero)[0]
    for prec in ("strict", "fp64", "split"):
        gpu = run_gpu(w, 3, prec, tp, st, sigN=zero)[0][0]
        assert gpu[4] == B.RT_OK
        if prec == "strict":
            np.testing.assert_array_equal(gpu[0], ora[0])
        elif prec == "fp64":
            # fused multiply-adds move results by ulps of the neighbours
            assert linf_rel(gpu[0], ora[0], floor_frac=1.0) <= 1e-14
        else:
            # random states put tiny N next to N ~ 1: FP32 cancellation is
            # bounded relative to the field's scale, not to each tiny cell
            e = linf_rel(gpu[0], ora[0], floor_frac=1.0)
            assert e <= 3e-6, e
        np.testing.assert_array_equal(gpu[1], ora[1])


def test_stromgren_config1_strict_is_bit_identical():
    w = I.stromgren(32, steps=100)
    ora = run_oracle(w, 100)[0]
    gpu = run_gpu(w, 100, "strict")[0][0]
    assert gpu[4] == B.RT_OK
    np.testing.assert_array_equal(gpu[0], ora[0])
    np.testing.assert_array_equal(gpu[1], ora[1])
    np.testing.assert_array_equal(gpu[2], ora[2])
    n_gpu, n_ora = np.count_nonzero(gpu[1] < 0.5), np.count_nonzero(ora[1] < 0.5)
    assert n_gpu == n_ora > 0
    np.testing.assert_array_equal(gpu[3][:, 3], ora[3][:, 3])      # ionised-cell history
    np.testing.assert_allclose(gpu[3][:, [0, 1, 2]], ora[3][:, [0, 1, 2]], rtol=1e-12)


def test_stromgren_config1_fp64_and_split():
    w = I.stromgren(32, steps=100)
    ora = run_oracle(w, 100)[0]
    gpu = run_gpu(w, 100, "fp64")[0][0]
    err = field_errors(gpu, ora, 1)
    report("Stromgren 32^3", "fp64", 100, err)
    assert max(err.values()) <= 1e-12, err
    assert np.count_nonzero(gpu[1] < 0.5) == np.count_nonzero(ora[1] < 0.5)
    spl = run_gpu(w, 100, "split")[0][0]
    err = field_errors(spl, ora, 1)
    report("Stromgren 32^3", "split", 100, err)
    print("split config-1 errors", err)
    assert err["N0"] <= 1e-4 and err["F0"] <= 1e-4, err
    assert err["xHI"] <= 1e-4, err


def _small_reion(n=24, nsrc=8, **kw):
    w = I.reion(n=n, steps=30, nsrc=nsrc)
    for k, v in kw.items():
        setattr(w, k, v)
    return w


@pytest.mark.parametrize("prec", ["fp64", "strict"])
def test_reion_small_fp64_parity(prec):
    w = _small_reion()
    ora = run_oracle(w, 30)[0]
    (gpu,), st = run_gpu(w, 30, prec)
    assert gpu[4] == B.RT_OK
    err = field_errors(gpu, ora, 3)
    assert max(err.values()) <= 1e-9, err
    assert st.realizability_clamps == 0
    np.testing.assert_allclose(gpu[3][:, [0, 1, 2, 4]], ora[3][:, [0, 1, 2, 4]], rtol=1e-9)
    np.testing.assert_array_equal(gpu[3][:, 3], ora[3][:, 3])


def test_reion_small_split_errors_reported():
    w = _small_reion()
    ora = run_oracle(w, 30)[0]
    (gpu,), st = run_gpu(w, 30, "split")
    assert gpu[4] == B.RT_OK
    err = field_errors(gpu, ora, 3)
    print("split reion errors", err)
    for g in range(3):
        assert err[f"N{g}"] <= 1e-4 and err[f"F{g}"] <= 1e-4, err
    assert err["xHI"] <= 1e-3 and err["T"] <= 1e-3, err


def test_fixed_subcycles_parity():
    """Eight fixed chemistry intervals per step at c/20 (the 256^3 workload's
    settings) on a small box."""
    w = _small_reion(n=20, nsrc=6, nsub=8, c_frac=0.05)
    ora = run_oracle(w, 20)[0]
    (gpu,), _ = run_gpu(w, 20, "fp64")
    err = field_errors(gpu, ora, 3)
    assert max(err.values()) <= 1e-9, err
    np.testing.assert_array_equal(gpu[3][:, 4], ora[3][:, 4])       # sub-cycle counts


def test_ensemble_of_uneven_boxes_parity():
    w = I.ensemble(nboxes=5, steps=20, sides=(8, 12, 16, 20), seed=9)
    ora = run_oracle(w, 20)
    for prec, tol in (("fp64", 1e-9), ("split", None)):
        gpu, st = run_gpu(w, 20, prec)
        for b in range(5):
            err = field_errors(gpu[b], ora[b], 2)
            if tol is not None:
                assert max(err.values()) <= tol, (b, err)
            else:
                assert max(err[k] for k in err if k[0] in "NF") <= 1e-4, (b, err)


def test_duplicate_sources_and_history():
    w = I.stromgren(16, steps=40)
    box = w.boxes[0]
    box.src_cells = np.array([0, 5, 0, 300, 5], dtype=np.int64)
    box.src_Q = np.array([3e47, 1e47, 2e47, 5e46, 4e47])
    ora = run_oracle(w, 40)[0]
    gpu = run_gpu(w, 40, "strict")[0][0]
    np.testing.assert_array_equal(gpu[0], ora[0])
    np.testing.assert_array_equal(gpu[1], ora[1])


def test_subcycle_cap_is_reported_not_faulted():
    w = _small_reion(n=12, nsrc=4)
    s = make_solver(w, "fp64", max_halvings=0)
    codes = [s.step(1) for _ in range(30)]
    st = s.stats()
    s.close()
    assert B.RT_ERR_SUBCYCLE in codes
    assert st.error_bits & 4


def test_upload_download_and_argument_errors():
    w = _small_reion(n=10, nsrc=2)
    s = make_solver(w, "split")
    U, xHI, T = w.boxes[0].initial_state(3)
    U = np.ascontiguousarray(I.random_realizable_state(w.boxes[0].shape, 3, 1), dtype=np.float32)
    xHI = xHI * 0.5
    B.rt_upload(s.h, 0, U=U, xHI=xHI, T=T)
    U2 = np.zeros_like(U)
    x2, T2 = np.zeros_like(xHI), np.zeros_like(T)
    B.rt_download(s.h, 0, U=U2, xHI=x2, T=T2)
    np.testing.assert_array_equal(U2, U)
    np.testing.assert_array_equal(x2, xHI)
    assert s.step(0) == B.RT_OK
    with pytest.raises(B.RTError):
        B.rt_step(s.h, -1)
    host_hist = np.zeros(10)
    assert B.lib().rt_step(s.h, 1, host_hist.ctypes.data) == B.RT_ERR_ARG
    with pytest.raises(B.RTError):
        B.rt_set_sources(s.h, 0, [10 ** 9], [1e48])
    with pytest.raises(B.RTError):
        B.rt_set_sources(s.h, 1, [0], [1e48])
    s.close()


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("shape,bc", [((33, 9, 40), [1, 1, 0, 0, 2, 2]), ((9, 33, 17), [0] * 6),
                                      ((16, 48, 48), [2, 1, 2, 1, 2, 1]),
                                      ((12, 20, 37), [3, 1, 0, 0, 2, 2])])
def test_transport_launch_shapes_are_bitwise_equal(shape, bc, flux):
    """Every launch shape of the FP32 transport, GLF and HLL (tile x grid,
    rt_params.tune = 2 + k) gives the same bits as the default; the tuner
    (tune = 1) picks one of them and reports it.  The last case has an
    inflow face (its ghost beam written into the halo by both kernels)."""
    G = 3
    w, st = _empty_workload(shape, G, bc, seed=sum(shape) + 5)
    if bc[0] == I.BC_INFLOW:
        w.inflow = [2e6, 0, 0, 0, 0, 0]
    ref = run_gpu(w, 3, "split", None, st, flux=flux)[0][0]
    assert ref[4] == B.RT_OK
    shapes = set()
    k = 0
    while True:
        try:
            (out,), stats = run_gpu(w, 3, "split", None, st, tune=2 + k, flux=flux)
        except B.RTError as e:
            assert e.code == B.RT_ERR_ARG and k >= 3, (k, e)
            break
        shapes.add((stats.tile_x, stats.tile_y, stats.transport_grid, stats.transport_zchunk,
                    stats.transport_lockstep, stats.transport_tma, stats.transport_gpb))
        for a, b in zip(out[:3], ref[:3]):
            np.testing.assert_array_equal(a, b)
        k += 1
    assert len({s[:2] for s in shapes}) == 3            # three tile shapes were run
    assert len({s[3] for s in shapes}) >= 2              # whole columns and z-chunks
    (out,), stats = run_gpu(w, 3, "split", None, st, tune=1, flux=flux)
    assert (stats.tile_x, stats.tile_y, stats.transport_grid, stats.transport_zchunk,
            stats.transport_lockstep, stats.transport_tma, stats.transport_gpb) in shapes
    if flux == 0:       # GLF: lockstep rows, TMA and two groups per block (3 = 2 + 1) were run
        assert any(s[4] > 0 for s in shapes) and any(s[5] for s in shapes)
        assert any(s[6] == 2 for s in shapes) and any(s[6] == 2 and s[4] > 0 for s in shapes)
    for a, b in zip(out[:3], ref[:3]):
        np.testing.assert_array_equal(a, b)


def test_tuned_full_step_matches_default():
    """Transport and chemistry with sources: the tuned launch shape changes
    no bit of the state or the history."""
    w = _small_reion()
    (ref,), _ = run_gpu(w, 10, "split")
    (out,), st = run_gpu(w, 10, "split", tune=1)
    for a, b in zip(out[:4], ref[:4]):
        np.testing.assert_array_equal(a, b)
    assert st.tile_x * st.tile_y == 256 and st.chem_grid > 0
    (_,), st = run_gpu(w, 2, "split", tune=2 + 31)       # 16x16 tiles, planes by TMA
    assert st.transport_tma == 1
    (_,), st64 = run_gpu(w, 2, "fp64")
    assert st64.transport_tma == 0


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_chemistry_launch_shapes_are_bitwise_equal(prec):
    """Every chemistry launch shape (rt_params.chem_tune = 2 + k: 1 or 2
    resident blocks per SM x 1, 2 or 4 work items per draw) gives the same
    bits, state and diagnostics history, as the default on uneven boxes with
    sources; the tuner (chem_tune = 1) picks one of them and reports it."""
    w = I.ensemble(nboxes=5, steps=6, sides=(8, 12, 16, 20), seed=11)
    ref, st0 = run_gpu(w, 6, prec)
    assert st0.chem_grab == 1
    seen = set()
    for k in range(6):
        out, st = run_gpu(w, 6, prec, chem_tune=2 + k)
        seen.add((st.chem_grid, st.chem_grab))
        for b in range(len(w.boxes)):
            for x, y in zip(out[b][:4], ref[b][:4]):
                np.testing.assert_array_equal(x, y)
    assert {g for _, g in seen} == {1, 2, 4}
    out, st = run_gpu(w, 6, prec, chem_tune=1)
    assert (st.chem_grid, st.chem_grab) in seen
    for b in range(len(w.boxes)):
        for x, y in zip(out[b][:4], ref[b][:4]):
            np.testing.assert_array_equal(x, y)


def test_ensemble_launch_shapes_are_bitwise_equal():
    """Uneven boxes in one launch: every transport launch shape, the
    column-aligned grids, the z-chunked orders and two groups per block
    included (their runs then straddle boxes of other depths), gives the same
    bits, state and history, as the default."""
    w = I.ensemble(nboxes=5, steps=6, sides=(8, 12, 16, 20), seed=11)
    ref, _ = run_gpu(w, 6, "split")
    for k in (0, 5, 7, 9, 12, 14, 15, 18, 19, 23, 26, 27, 31, 33, 35, 36):
        out, _ = run_gpu(w, 6, "split", tune=2 + k)
        for b in range(5):
            for x, y in zip(out[b][:4], ref[b][:4]):
                np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("shape", [(7, 5, 3), (9, 33, 17), (33, 9, 40)])
@pytest.mark.parametrize("bc", BCS)
def test_hll_transport_parity(shape, bc):
    """The HLL flux (rt_params.flux = 1): three pure transport steps against
    the oracle's HLL transport.  The two sides build their wave-speed tables
    independently (agreeing to ~1e-12), which bounds the FP64 agreement."""
    G = 3
    w, st = _empty_workload(shape, G, bc, seed=sum(shape) * 3 + 1)
    to, tp = tables(w)
    zero = [0.0] * G
    ora = run_oracle(w, 3, to, st, sigN=zero, flux=O.FLUX_HLL)[0]
    for prec in ("strict", "fp64", "split"):
        gpu = run_gpu(w, 3, prec, tp, st, sigN=zero, flux=1)[0][0]
        assert gpu[4] == B.RT_OK
        U, Uo = gpu[0], ora[0]
        scale = np.max(np.abs(Uo[..., 0]))
        err = np.max(np.abs(U - Uo)) / scale
        assert err <= (2e-6 if prec == "split" else 1e-10), (prec, err)


def test_hll_full_step_parity_and_sharper_than_glf():
    """Sources, absorption and chemistry with the HLL flux: FP64 against the
    oracle <= 1e-9; the run differs from the GLF run."""
    w = _small_reion()
    ora = run_oracle(w, 30, flux=O.FLUX_HLL)[0]
    (gpu,), st = run_gpu(w, 30, "fp64", flux=1)
    assert gpu[4] == B.RT_OK
    err = field_errors(gpu, ora, 3)
    assert max(err.values()) <= 1e-9, err
    assert st.realizability_clamps == 0
    (glf,), _ = run_gpu(w, 30, "fp64")
    assert np.max(np.abs(glf[1] - gpu[1])) > 1e-3


def test_hll_rejected_where_unsupported():
    import torch
    w = _small_reion(n=8, nsrc=1)
    s = make_solver(w, "fp64", flux=1)
    st = s.states[0]
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(w.boxes[0].ncell, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RTError) as e:
        B.rt_adjoint(s.h, st.U.data_ptr(), st.xHI.data_ptr(), st.T.data_ptr(), 1, 1,
                     z.data_ptr(), len(w.boxes[0].src_Q), d.data_ptr())
    assert e.value.code == B.RT_ERR_ARG and "GLF" in str(e.value)
    s.close()
