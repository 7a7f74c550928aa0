"""GPU adjoint (rt_adjoint and the torch autograd wrapper):
  * against the oracle's FP64 adjoint (same algorithm) on a small periodic
    box, <= 1e-9;
  * against central finite differences of the forward run on the 64^3,
    200-step adjoint workload (16 sources, 1 group, 4 fixed chemistry
    intervals, checkpoints every 20 steps), <= 1e-3.
The loss is L = mean_t (X(t) - X*(t))^2 with X the volume-weighted ionised
fraction after each step and X* the history of the same run with every
luminosity multiplied by exp(0.1 z), z ~ N(0, 1) (seed 5)."""
import numpy as np
import pytest

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

from _harness import gpu_params, oracle_params, report, tables

pytestmark = pytest.mark.gpu


def _state(w, box, fp64=True):
    import torch
    U, xHI, T = box.initial_state(w.ngroups)
    return B.BoxState(U=torch.as_tensor(U, dtype=torch.float64, device="cuda"),
                      xHI=torch.as_tensor(xHI, dtype=torch.float64, device="cuda"),
                      T=torch.as_tensor(T, dtype=torch.float64, device="cuda"),
                      n0=torch.as_tensor(box.n0, dtype=torch.float64, device="cuda"),
                      dx=box.dx, nunit=w.nunit(box))


@pytest.mark.parametrize("prec", ["fp64", "strict"])
def test_adjoint_matches_oracle_adjoint(prec):
    import torch
    from paper_1508_07888_b300.autograd import HistoryRun
    w = I.reion(n=12, steps=15, nsrc=3, seed=21, lum_seed=22)
    w.nsub = 4
    w.edges_eV = I.GROUPS_2
    box = w.boxes[0]
    box.n0 = I.lognormal_field((14, 10, 12), 1.0, 2.0, 23)
    cells = np.array([box.n0.argmax(), 77, 77], dtype=np.int64)
    box.src_cells = cells
    box.src_Q = np.array([2e49, 5e48, 1e48])
    to, tp = tables(w)
    steps = 15
    wts = np.random.default_rng(3).uniform(0.5, 1.5, steps)
    # oracle
    p = oracle_params(w, to)
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, xHI, T = box.initial_state(2)
    dS, dn0 = O.adjoint(p, U, xHI, T, box.n0, box.dx, nunit, steps, wts, S)
    vol = box.dx ** 3
    dQo = np.array([sum(p.frac[i] * dS[i, c] for i in range(2)) for c in cells]) / (vol * nunit)
    # GPU
    run = HistoryRun(gpu_params(w, tp, prec), _state(w, box), cells, steps, ckpt_every=4)
    Q = torch.tensor(box.src_Q, dtype=torch.float64)
    n0 = torch.as_tensor(box.n0, dtype=torch.float64, device="cuda")
    X = run.forward(Q, n0)
    dQg, dn0g = run.backward(torch.as_tensor(wts, device="cuda"))
    run.close()
    d = dn0g.cpu().numpy().reshape(-1)
    report("adjoint 14x10x12 (vs the oracle's adjoint)", prec, steps,
           {"dL_dQ": np.max(np.abs(dQg.numpy() - dQo) / np.abs(dQo)),
            "dL_dn0": np.max(np.abs(d - dn0)) / np.max(np.abs(dn0))})
    np.testing.assert_allclose(dQg.numpy(), dQo, rtol=1e-9)
    assert np.max(np.abs(d - dn0)) <= 1e-9 * np.max(np.abs(dn0))
    assert np.abs(dQo).min() > 0


def _config5():
    import torch
    from paper_1508_07888_b300.autograd import HistoryRun, ionisation_history
    w = I.adjoint_box()
    box = w.boxes[0]
    _, tp = tables(w)
    run = HistoryRun(gpu_params(w, tp, "fp64"), _state(w, box), box.src_cells, w.steps,
                     ckpt_every=20)
    Q0 = torch.tensor(box.src_Q, dtype=torch.float64)
    n00 = torch.as_tensor(box.n0, dtype=torch.float64, device="cuda")
    with torch.no_grad():
        Xt = ionisation_history(Q0 * torch.as_tensor(I.target_perturbation(len(box.src_Q))),
                                n00, run)

    def loss(Q, n0):
        X = ionisation_history(Q, n0, run)
        return ((X - Xt) ** 2).mean()

    return run, Q0, n00, loss


def test_config5_gradients_match_finite_differences():
    import torch
    run, Q0, n00, loss = _config5()
    Q = Q0.clone().requires_grad_(True)
    n0 = n00.clone().requires_grad_(True)
    L = loss(Q, n0)
    L.backward()
    gQ = Q.grad.numpy()
    gn = n0.grad.detach()
    assert L.item() > 0
    h = 1e-4
    worst = {"dL_dQ": 0.0, "dL_dn0_directional": 0.0, "dL_dn0_cells": 0.0}
    with torch.no_grad():
        for k in range(len(Q0)):
            Qp, Qm = Q0.clone(), Q0.clone()
            Qp[k] *= 1 + h
            Qm[k] *= 1 - h
            fd = (loss(Qp, n00) - loss(Qm, n00)).item() / (2 * h * Q0[k].item())
            worst["dL_dQ"] = max(worst["dL_dQ"], abs(gQ[k] - fd) / max(abs(fd), 1e-3 * np.abs(gQ).max()))
            assert gQ[k] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(gQ).max()), (k, gQ[k], fd)
        rng = np.random.default_rng(55)
        for _ in range(4):                       # directional derivatives
            v = torch.as_tensor(rng.standard_normal(n00.shape), device="cuda") * n00
            fd = (loss(Q0, n00 + h * v) - loss(Q0, n00 - h * v)).item() / (2 * h)
            ad = torch.sum(gn * v).item()
            worst["dL_dn0_directional"] = max(worst["dL_dn0_directional"], abs(ad - fd) / abs(fd))
            assert ad == pytest.approx(fd, rel=1e-3, abs=0), (ad, fd)
        flat = gn.reshape(-1).cpu().numpy()
        top = np.argsort(-np.abs(flat))[:2000]
        for c in rng.choice(top, size=32, replace=False):
            e = torch.zeros(flat.size, dtype=torch.float64, device="cuda")
            e[int(c)] = n00.reshape(-1)[int(c)]
            e = e.reshape(n00.shape)
            fd = (loss(Q0, n00 + h * e) - loss(Q0, n00 - h * e)).item() / (2 * h * e.reshape(-1)[int(c)].item())
            worst["dL_dn0_cells"] = max(worst["dL_dn0_cells"],
                                        abs(flat[c] - fd) / max(abs(fd), 1e-3 * np.abs(flat).max()))
            assert flat[c] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(flat).max()), (c, flat[c], fd)
    report("adjoint 64^3 (gradient vs central differences)", "fp64", 200, worst)
    run.close()
