"""GPU supercomoving units (rt_params.cosmo, Sec. 3) against the oracle's
run_cosmo: the comoving state, T~ = a^2 T, the chemistry at each step's a(t),
and a(t) itself.  Tolerances as for the static runs (FP64 and strict
<= 1e-9, split x_HI and T <= 1e-3).  A toy expansion rate makes a 60-step
run expand the box by a few per cent."""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import field_errors, linf_rel, make_solver, oracle_params, run_gpu, tables

pytestmark = pytest.mark.gpu

COSMO = (2.0e-14, 0.3, 0.7, 0.2)          # H0 [1/s], omega_m, omega_l, a0


def _oracle(w, steps, cosmo):
    box = w.boxes[0]
    to, _ = tables(w)
    p = oracle_params(w, to)
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, x, T = box.initial_state(w.ngroups)
    H0, Om, OL, a0 = cosmo
    return O.run_cosmo(p, U, x, T * a0 ** 2, box.n0, box.dx, nunit, steps, S, H0, Om, OL, a0)


def _gpu(w, steps, prec, cosmo, calls=(None,)):
    box = w.boxes[0]
    U, x, T = box.initial_state(w.ngroups)
    s = make_solver(w, prec, None, [(U, x, T * cosmo[3] ** 2)], cosmo=cosmo)
    done = 0
    for n in calls:
        n = steps - done if n is None else n
        assert s.step(n) == B.RT_OK
        done += n
    U, x, T = s.numpy_state(0)
    a = s.stats().a
    s.close()
    return U, x, T, a


@pytest.mark.parametrize("prec", ["fp64", "strict", "split"])
def test_cosmo_parity(prec):
    w = I.reion(n=12, steps=60, nsrc=3, seed=61, lum_seed=62)
    r = _oracle(w, 60, COSMO)
    assert r.run.err == 0 and r.a > 1.02 * COSMO[3]
    U, x, T, a = _gpu(w, 60, prec, COSMO)
    assert a == pytest.approx(r.a, rel=1e-14, abs=0)
    if prec == "split":
        ex, eT = linf_rel(x, r.run.xHI), linf_rel(T, r.run.T)
        assert ex <= 1e-3 and eT <= 1e-3, (ex, eT)
        err = field_errors((U, x, T), (r.run.U, r.run.xHI, r.run.T), 3)
        assert max(err[k] for k in err if k[0] in "NF") <= 1e-4, err
    else:
        err = field_errors((U, x, T), (r.run.U, r.run.xHI, r.run.T), 3)
        assert max(err.values()) <= 1e-9, err
    assert np.min(r.run.xHI) < 0.5


def test_chunked_calls_agree_bitwise():
    w = I.reion(n=8, steps=5000, nsrc=1, seed=63, lum_seed=64)
    cosmo = (2.0e-16, 0.3, 0.7, 0.1)
    one = _gpu(w, 5000, "fp64", cosmo)                    # 4096 + 904 inside the library
    two = _gpu(w, 5000, "fp64", cosmo, calls=(2500, 2500))
    for u, v in zip(one[:3], two[:3]):
        np.testing.assert_array_equal(u, v)
    assert one[3] == two[3] > 0.1
    a = 0.1
    dt = O.timestep(oracle_params(w, tables(w)[0]), w.boxes[0].dx)
    for _ in range(5000):
        a = O.advance_a(a, a * dt, *cosmo[:3])
    assert one[3] == pytest.approx(a, rel=1e-13, abs=0)


def test_no_expansion_is_the_static_run():
    w = I.reion(n=12, steps=30, nsrc=3, seed=61, lum_seed=62)
    static = run_gpu(w, 30, "fp64")[0][0]
    U, x, T, a = _gpu(w, 30, "fp64", (0.0, 0.3, 0.7, 1.0))
    assert a == 1.0
    for u, v in zip((U, x, T), static[:3]):
        np.testing.assert_array_equal(u, v)
