"""Multi-step parity at the full sizes of the workloads: every output field of
every cell after the run, element-wise against the oracle run over the same
steps (not one step at a time from the GPU's own state, so that error that
accumulates over the run is measured at the shapes the benchmark runs).

Tolerances (L-inf relative with a floor of 1e-6 of the field's maximum; F in
units of the local N):
  * all-FP64 form: every field <= 1e-9;
  * split form (FP32 transport): the radiation N and F <= 1e-4; x_HI and T
    carry the FP32 radiation's error into the chemistry and are reported,
    with a sanity bound of 1e-2.

Workloads: the 128^3 reionisation box over 100 steps, the 64-box ensemble
over 100 steps, and the 256^3 box with 8 fixed chemistry intervals over 20
steps.  The oracle runs on every host core (the ensemble's boxes side by
side).  When RT_PARITY_REPORT names a file, each test appends its measured
errors to it as one JSON line.
"""
import numpy as np
import pytest

from paper_1508_07888_b300 import binding as B

from _harness import field_errors, report, run_gpu

pytestmark = pytest.mark.gpu


def check(prec, errs, name):
    if prec == "fp64":
        assert max(errs.values()) <= 1e-9, (name, errs)
    else:
        assert max(v for k, v in errs.items() if k[0] in "NF") <= 1e-4, (name, errs)
        assert errs["xHI"] <= 1e-2 and errs["T"] <= 1e-2, (name, errs)


def merge(per_box):
    """Worst error per field over boxes."""
    out = {}
    for e in per_box:
        for k, v in e.items():
            out[k] = max(out.get(k, 0.0), v)
    return out


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_reion128_100_steps_every_field(prec, reion128_oracle):
    w, _, tp, ora = reion128_oracle
    assert ora[4] == 0
    (gpu,), st = run_gpu(w, 100, prec, tp)
    assert gpu[4] == B.RT_OK and st.error_bits == 0
    errs = field_errors(gpu, ora, w.ngroups)
    report("reion 128^3", prec, 100, errs)
    check(prec, errs, "reion128")
    # diagnostics history: ionised fraction, photons, max f, mean sub-cycles
    rtol = 1e-9 if prec == "fp64" else 1e-3
    np.testing.assert_allclose(gpu[3][:, [0, 1, 2, 4]], ora[3][:, [0, 1, 2, 4]], rtol=rtol)
    if prec == "fp64":
        np.testing.assert_array_equal(gpu[3][:, 3], ora[3][:, 3])   # count(x_HI < 0.5)


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_ensemble64_100_steps_every_field(prec, ensemble64_oracle):
    w, _, tp, ora = ensemble64_oracle
    assert all(o[4] == 0 for o in ora)
    gpu, st = run_gpu(w, 100, prec, tp)
    assert st.error_bits == 0
    per_box = []
    for b in range(len(w.boxes)):
        assert gpu[b][4] == B.RT_OK
        per_box.append(field_errors(gpu[b], ora[b], w.ngroups))
    errs = merge(per_box)
    report("ensemble 64 boxes", prec, 100, errs)
    check(prec, errs, "ensemble")


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_reion256_nsub8_20_steps_every_field(prec, reion256_oracle):
    w, _, tp, ora = reion256_oracle
    assert ora[4] == 0
    (gpu,), st = run_gpu(w, 20, prec, tp)
    assert gpu[4] == B.RT_OK and st.error_bits == 0
    errs = field_errors(gpu, ora, w.ngroups)
    del gpu
    report("reion 256^3 nsub 8", prec, 20, errs)
    check(prec, errs, "reion256")
