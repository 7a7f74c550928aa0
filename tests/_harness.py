"""Shared helpers of the parity tests: run one workload through the CPU
oracle and through the C-ABI library on the same seeded inputs."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle as O
from paper_1508_07888_b300 import binding as B
from paper_1508_07888_b300 import inputs as I

PREC = {"split": B.RT_PREC_SPLIT, "fp64": B.RT_PREC_FP64, "strict": B.RT_PREC_FP64_STRICT}


def f32_table(t: dict) -> dict:
    return {k: I.f32(v) for k, v in t.items()}


def tables(w: I.Workload):
    """Each side's own group table, rounded to float32-representable values;
    the two quadratures must agree after rounding."""
    to = f32_table(O.group_table(w.edges_eV, w.T_bb))
    tp = f32_table(B.rt_group_table(w.edges_eV, w.T_bb))
    for k in to:
        assert np.array_equal(to[k], tp[k]), k
    return to, tp


def oracle_params(w: I.Workload, table: dict, box=None, **over) -> O.Params:
    kw = dict(sigN=table["sigN"], sigE=table["sigE"], Eavg=table["Eavg"], frac=table["frac"],
              c=w.c_red, cfl=w.cfl, ots=w.ots, isothermal=w.isothermal, nsub=w.nsub,
              rates_const=w.rates_const, alphaA=w.alphaA, alphaB=w.alphaB, beta=w.beta,
              bc=list(w.bc))
    if any(w.inflow):
        box = box if box is not None else w.boxes[0]
        kw["inflow"] = [O.inflow_density(w.inflow[f], table["frac"], w.c_red, w.nunit(box))
                        for f in range(6)]
    kw.update(over)
    return O.Params(**kw)


def gpu_params(w: I.Workload, table: dict, precision: str, **over) -> B.rt_params:
    kw = dict(cfl=w.cfl, ots=w.ots, isothermal=w.isothermal, nsub=w.nsub,
              rates_const=w.rates_const, alphaA=w.alphaA, alphaB=w.alphaB, beta=w.beta,
              bc=w.bc, precision=PREC[precision], inflow=w.inflow)
    for k in ("sigN", "sigE", "Eavg", "frac"):
        if k in over:
            table = dict(table, **{k: over.pop(k)})
    if "c" in over:
        over["c_red"] = over.pop("c")
    c_red = over.pop("c_red", w.c_red)
    kw.update(over)
    return B.make_params(w.ngroups, table, c_red, **kw)


def run_oracle(w: I.Workload, steps: int, table=None, states=None, threads=None,
               box_parallel=False, **over):
    """Returns per box: (U, xHI, T, hist, err, nclamp).

    box_parallel: run the boxes side by side, one single-threaded oracle call
    per host core (the calls release the GIL and share no state; the results
    are the same bits as one after the other).  Otherwise each box runs on
    `threads` OpenMP threads (default: the host's cores, at most 8)."""
    table = table if table is not None else tables(w)[0]
    if threads is None:
        threads = min(8, os.cpu_count() or 1)

    def one(bi):
        box = w.boxes[bi]
        p = oracle_params(w, table, box=box, **over)
        nunit = w.nunit(box)
        U, xHI, T = states[bi] if states is not None else box.initial_state(w.ngroups)
        S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
        r = O.run(p, U, xHI, T, box.n0, box.dx, nunit, steps, S)
        return (r.U, r.xHI, r.T, r.hist, r.err, r.nclamp)

    if box_parallel:
        from concurrent.futures import ThreadPoolExecutor
        O.set_threads(1)
        order = sorted(range(len(w.boxes)), key=lambda b: -w.boxes[b].ncell)   # largest first
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            res = dict(zip(order, ex.map(one, order)))
        return [res[b] for b in range(len(w.boxes))]
    O.set_threads(threads)
    out = [one(bi) for bi in range(len(w.boxes))]
    O.set_threads(1)
    return out


def make_solver(w: I.Workload, precision: str, table=None, states=None, **over) -> B.Solver:
    table = table if table is not None else tables(w)[1]
    p = gpu_params(w, table, precision, **over)
    boxes = []
    for bi, box in enumerate(w.boxes):
        U, xHI, T = states[bi] if states is not None else box.initial_state(w.ngroups)
        boxes.append((U, xHI, T, box.n0, box.dx, w.nunit(box)))
    s = B.Solver.from_numpy(p, boxes)
    for bi, box in enumerate(w.boxes):
        s.set_sources(bi, box.src_cells, box.src_Q)
    return s


def run_gpu(w: I.Workload, steps: int, precision: str, table=None, states=None, **over):
    s = make_solver(w, precision, table, states, **over)
    code, hist = s.run(steps)
    out = []
    for bi in range(len(w.boxes)):
        U, xHI, T = s.numpy_state(bi)
        out.append((U, xHI, T, hist[:, bi, :], code))
    st = s.stats()
    s.close()
    return out, st


def linf_rel(a, b, floor_frac=1e-6):
    """max |a - b| / max(|b|, floor_frac * max|b|) over all elements."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b))
    if scale == 0.0:
        return float(np.max(np.abs(a - b)))
    den = np.maximum(np.abs(b), floor_frac * scale)
    return float(np.max(np.abs(a - b) / den))


def flux_rel(Fa, Fb, Nb, floor_frac=1e-6):
    """max |Fa - Fb| / max(N, floor_frac max N): the flux error in units of
    the local photon density (|Fhat| <= Nhat, so N is the flux's own scale;
    a per-component relative error is undefined where a component crosses 0)."""
    d = np.linalg.norm(np.asarray(Fa, np.float64) - np.asarray(Fb, np.float64), axis=-1)
    Nb = np.asarray(Nb, np.float64)
    scale = np.max(np.abs(Nb))
    if scale == 0.0:
        return float(np.max(d))
    return float(np.max(d / np.maximum(np.abs(Nb), floor_frac * scale)))


def field_errors(gpu_box, ora_box, G):
    """L-inf relative error per output field (N and F per group, xHI, T)."""
    Ug, xg, Tg = gpu_box[:3]
    Uo, xo, To = ora_box[:3]
    err = {}
    for g in range(G):
        err[f"N{g}"] = linf_rel(Ug[g, ..., 0], Uo[g, ..., 0])
        err[f"F{g}"] = flux_rel(Ug[g, ..., 1:], Uo[g, ..., 1:], Uo[g, ..., 0])
    err["xHI"] = linf_rel(xg, xo)
    err["T"] = linf_rel(Tg, To)
    return err


def report(name: str, form: str, steps: int, errs: dict) -> None:
    """Append a test's measured errors as one JSON line to the file that
    RT_PARITY_REPORT names (nothing when it is unset)."""
    path = os.environ.get("RT_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"workload": name, "form": form, "steps": steps,
                                "linf": {k: float(v) for k, v in errs.items()}}) + "\n")
