"""GPU CRTA fine level (rt_set_fine) against the oracle's run_crta: refined
cells run the chemistry with their parent's post-transport radiation and
source injected.

Tolerances as for the coarse chemistry: FP64 and strict forms <= 1e-9
(L-inf relative); the split form's FP32 radiation bounds its x_HI and T by
1e-3.  The bitwise checks compare the library with itself (a refined copy of
a coarse cell, the coarse run with and without the fine level)."""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import linf_rel, make_solver, oracle_params, tables

pytestmark = pytest.mark.gpu


def _workload(n=16, nsrc=4, steps=20):
    return I.reion(n=n, steps=steps, nsrc=nsrc, seed=41, lum_seed=42)


def _gpu_crta(w, prec, fine, steps, table=None, states=None):
    s = make_solver(w, prec, table, states)
    xf, Tf = s.set_fine(0, fine.parent, fine.n0, fine.xHI, fine.T)
    code, hist = s.run(steps)
    U, xHI, T = s.numpy_state(0)
    out = (U, xHI, T, hist[:, 0, :], code, xf.cpu().numpy(), Tf.cpu().numpy())
    st = s.stats()
    s.close()
    return out, st


@pytest.mark.parametrize("prec", ["fp64", "strict", "split"])
def test_fine_level_parity(prec):
    w = _workload()
    box = w.boxes[0]
    to, tp = tables(w)
    fine = I.refine_densest(box, frac=0.15, seed=5)
    p = oracle_params(w, to)
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, xHI, T = box.initial_state(w.ngroups)
    r = O.run_crta(p, U, xHI, T, box.n0, box.dx, nunit, 20, S, fine.parent, fine.n0, fine.xHI,
                   fine.T)
    assert r.coarse.err == 0
    g, st = _gpu_crta(w, prec, fine, 20, tp)
    assert g[4] == B.RT_OK
    tol = 1e-3 if prec == "split" else 1e-9
    ex, eT = linf_rel(g[5], r.xHI_fine), linf_rel(g[6], r.T_fine)
    print(prec, "fine errors", ex, eT)
    assert ex <= tol and eT <= tol, (ex, eT)
    assert linf_rel(g[1], r.coarse.xHI) <= tol
    assert np.min(r.xHI_fine) < 0.5                    # some refined cells were ionised
    assert st.kernel_launches[2] == 0                   # profiling off: nothing timed


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_copy_children_follow_their_parents_bitwise(prec):
    w = _workload()
    box = w.boxes[0]
    U, xHI, T = box.initial_state(w.ngroups)
    parents = np.array(list(box.src_cells) + [0, 100, box.ncell - 1], dtype=np.int64)
    fine = I.FineLevel(parent=parents, n0=box.n0.reshape(-1)[parents],
                       xHI=xHI.reshape(-1)[parents], T=T.reshape(-1)[parents])
    g, _ = _gpu_crta(w, prec, fine, 15)
    np.testing.assert_array_equal(g[5], g[1].reshape(-1)[parents])
    np.testing.assert_array_equal(g[6], g[2].reshape(-1)[parents])


def test_fine_level_leaves_the_coarse_run_unchanged_and_is_timed():
    w = _workload()
    box = w.boxes[0]
    fine = I.refine_densest(box, frac=0.2, seed=6)
    s0 = make_solver(w, "split")
    c0, h0 = s0.run(12)
    a = s0.numpy_state(0)
    s0.close()
    s = make_solver(w, "split")
    s.set_fine(0, fine.parent, fine.n0, fine.xHI, fine.T)
    B.rt_set_profiling(s.h, 1)
    c1, h1 = s.run(12)
    b = s.numpy_state(0)
    st = s.stats()
    s.close()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(h0, h1)
    assert st.kernel_launches[2] == 12 and st.kernel_ms[2] > 0


def test_set_fine_arguments():
    import torch
    w = _workload(n=8, nsrc=1)
    s = make_solver(w, "fp64")
    n = 5
    good = torch.zeros(n, dtype=torch.int64, device="cuda")
    bad = torch.full((n,), w.boxes[0].ncell, dtype=torch.int64, device="cuda")
    d = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.RTError) as e:
        B.rt_set_fine(s.h, 0, n, bad.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr())
    assert e.value.code == B.RT_ERR_ARG
    with pytest.raises(B.RTError):
        B.rt_set_fine(s.h, 1, n, good.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr())
    host = np.zeros(n, dtype=np.int64)
    with pytest.raises(B.RTError):
        B.rt_set_fine(s.h, 0, n, host.ctypes.data, d.data_ptr(), d.data_ptr(), d.data_ptr())
    B.rt_set_fine(s.h, 0, 0, 0, 0, 0, 0)                # removing an absent level is fine
    s.close()


def test_reion_128_fine_level_sampled_step(reion128_oracle):
    """The 128^3 workload with its densest eighth refined into 8 children
    (2,097,152 refined cells), refined after the oracle's 100 steps: each child
    starts in its parent's state at that time.  One GPU step from that
    oracle-made state, against the oracle's chemistry of sampled refined
    cells from the oracle's own transport of the same coarse state."""
    import torch
    w, to, tp, ora = reion128_oracle
    box = w.boxes[0]
    U, xHI, T = ora[:3]
    fine = I.refine_densest(box, frac=0.125, seed=7)
    x0 = xHI.reshape(-1)[fine.parent].copy()
    T0 = T.reshape(-1)[fine.parent].copy()
    s = make_solver(w, "fp64", tp, [(U, xHI, T)])
    xf, Tf = s.set_fine(0, fine.parent, fine.n0, x0, T0)
    assert s.step(1) == B.RT_OK
    x1, T1 = xf.cpu().numpy(), Tf.cpu().numpy()
    s.close()
    p = oracle_params(w, to)
    nunit = w.nunit(box)
    dt = O.timestep(p, box.dx)
    Us = O.transport(p, U, O.courant_number(p, box.dx))
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    rng = np.random.default_rng(128)
    near_src = np.flatnonzero(np.isin(fine.parent, box.src_cells))
    front = np.flatnonzero((x0 > 0.02) & (x0 < 0.98))
    if front.size > 2000:
        front = rng.choice(front, 2000, replace=False)
    idx = np.unique(np.concatenate([rng.choice(fine.parent.size, 3000, replace=False), near_src,
                                    front]))
    G = w.ngroups
    Usf = Us.reshape(G, -1, 4)
    worst = 0.0
    for f in idx:
        c = fine.parent[f]
        _, xo, To_, _, err = O.chem_cell(p, dt, nunit, float(fine.n0[f]), S[:, c], Usf[:, c, :],
                                          float(x0[f]), float(T0[f]))
        assert err == 0
        worst = max(worst, abs(x1[f] - xo) / max(abs(xo), 1e-6), abs(T1[f] - To_) / To_)
    assert worst <= 1e-11, worst
