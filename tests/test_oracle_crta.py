"""Pins of the oracle's CRTA fine level (Sec. 5: transport on the coarse grid
only; refined cells run the thermochemistry with the coarse radiation field
injected unchanged).

* a refined cell that copies its parent (same density and state) follows the
  parent bit for bit, step after step -- so it reads the right parent's
  post-transport radiation and source, over the right dt;
* the fine level does not change the coarse run;
* after one step, a refined cell equals the coarse cell of a run in which
  the parent's density is replaced by the child's (the post-transport field
  of the first step does not depend on the density), so the child's own
  density is the one used.
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import inputs as I


def _setup(n=12, nsrc=3, steps=20):
    w = I.reion(n=n, steps=steps, nsrc=nsrc, seed=31, lum_seed=32)
    box = w.boxes[0]
    t = {k: I.f32(v) for k, v in O.group_table(w.edges_eV, w.T_bb).items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 cfl=w.cfl, bc=list(w.bc))
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    return w, box, p, nunit, S


def test_copy_children_follow_their_parents_bitwise():
    w, box, p, nunit, S = _setup()
    U, xHI, T = box.initial_state(w.ngroups)
    parents = np.array([0, 5, 77, 1000, box.ncell - 1] + list(box.src_cells), dtype=np.int64)
    n0 = box.n0.reshape(-1)
    r = O.run_crta(p, U, xHI, T, box.n0, box.dx, nunit, 20, S, parents, n0[parents],
                   xHI.reshape(-1)[parents], T.reshape(-1)[parents])
    assert r.coarse.err == 0
    np.testing.assert_array_equal(r.xHI_fine, r.coarse.xHI.reshape(-1)[parents])
    np.testing.assert_array_equal(r.T_fine, r.coarse.T.reshape(-1)[parents])
    assert np.any(r.xHI_fine < 0.9)                  # the sources' cells did evolve


def test_fine_level_leaves_the_coarse_run_unchanged():
    w, box, p, nunit, S = _setup()
    U, xHI, T = box.initial_state(w.ngroups)
    fine = I.refine_densest(box, frac=0.1, seed=3)
    a = O.run(p, U, xHI, T, box.n0, box.dx, nunit, 10, S)
    b = O.run_crta(p, U, xHI, T, box.n0, box.dx, nunit, 10, S, fine.parent, fine.n0,
                   fine.xHI, fine.T).coarse
    for x, y in ((a.U, b.U), (a.xHI, b.xHI), (a.T, b.T), (a.hist, b.hist)):
        np.testing.assert_array_equal(x, y)


def test_child_after_one_step_equals_a_coarse_cell_with_its_density():
    w, box, p, nunit, S = _setup()
    U, xHI, T = box.initial_state(w.ngroups)
    rng = np.random.default_rng(8)
    # a radiation field already present, so the first step's chemistry sees photons
    U = I.f32(I.random_realizable_state(box.shape, w.ngroups, 9, nmax=50.0))
    parents = rng.choice(box.ncell, size=6, replace=False).astype(np.int64)
    n0f = I.f32(box.n0.reshape(-1)[parents] * rng.uniform(0.2, 5.0, 6))
    r = O.run_crta(p, U, xHI, T, box.n0, box.dx, nunit, 1, S, parents, n0f,
                   xHI.reshape(-1)[parents], T.reshape(-1)[parents])
    for k, c in enumerate(parents):
        n0 = box.n0.copy().reshape(-1)
        n0[c] = n0f[k]
        ref = O.run(p, U, xHI, T, n0.reshape(box.shape), box.dx, nunit, 1, S)
        assert r.xHI_fine[k] == ref.xHI.reshape(-1)[c]
        assert r.T_fine[k] == ref.T.reshape(-1)[c]
        assert r.xHI_fine[k] != r.coarse.xHI.reshape(-1)[c]     # the density mattered


def test_refine_densest_keeps_the_parent_mass():
    w, box, p, nunit, S = _setup()
    fine = I.refine_densest(box, frac=0.125, seed=4)
    par = fine.parent.reshape(-1, 8)
    assert np.all(par == par[:, :1])
    mean = fine.n0.reshape(-1, 8).mean(axis=1)
    np.testing.assert_allclose(mean, box.n0.reshape(-1)[par[:, 0]], rtol=1e-6)
    assert len(np.unique(par[:, 0])) == round(0.125 * box.ncell)
