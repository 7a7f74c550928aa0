#!/usr/bin/env python
"""Benchmark of the M1 radiative-transfer step on B300.

Workload (one bench step = one full run of it, restarted from its initial
state): the 128^3 lognormal reionisation box -- ln(n0/1e-3) ~ N(0, 1) with
P(k) ~ k^-2, 64 sources at the densest cells with log-uniform luminosities in
[1e48, 1e50] photons/s, 3 photon groups of a 5e4 K black body, T evolving
with cooling, c/10, adaptive chemistry steps -- advanced by 500 radiative
steps (transport + chemistry + diagnostics each).  Metric: cell-updates/s =
cells x 500 / time of the run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line.  The timed form is the FP32-transport + FP64
chemistry split; the all-FP64 form is timed beside it.  Under torchrun every
rank runs an independent replica of the workload on its own GPU (the step has
no cross-box exchange), value = total cell-updates of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M1 RT cell-updates/s (transport+chem) vs all-FP64 GPU form; % HBM roofline"
UNIT = "cell-updates/s"
RT_STEPS = 500


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rt-steps", type=int, default=RT_STEPS,
                    help="radiative steps per bench step (the workload runs 500)")
    ap.add_argument("--no-fp64-form", action="store_true", help="skip the all-FP64 comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=3,
                    help="oracle steps timed at each of the CPU baseline's sample points")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-crta", action="store_true")
    ap.add_argument("--no-hll", action="store_true")
    ap.add_argument("--no-cosmo", action="store_true")
    ap.add_argument("--no-256", action="store_true", help="skip the 256^3 workload's row")
    ap.add_argument("--config-table", action="store_true",
                    help="instead of the bench line: one JSON line per workload x form")
    ap.add_argument("--only", choices=["reion256", "ensemble", "hll"], default=None,
                    help="run that row alone and print it (profiling commands)")
    ap.add_argument("--chem-tune", type=int, default=1,
                    help="chemistry launch shape: 1 = tuned at create, 2 + k = shape k, 0 = default")
    ap.add_argument("--tune", type=int, default=1,
                    help="rt_params.tune of the split form: 1 = time the transport's launch "
                         "shapes at create, 2 + k = shape k (profiling runs fix the shape)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ws, units_local: float, sec_local: float):
    """Whole-job throughput of ws replicas that each processed units_local in
    sec_local: all ranks' units over the slowest rank's time.  Returns
    (value, max seconds); every rank gets the same numbers."""
    sec = max_over_ranks(ws, sec_local)
    return units_local * ws / sec, sec


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]),
                                 util=float(f[4]), hw=f[6], hwt=f[7], swt=f[8], swp=f[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------- workload
def workload():
    from paper_1508_07888_b300 import inputs as I
    return I.reion(n=128, steps=RT_STEPS)


def group_table(w):
    from paper_1508_07888_b300 import binding as B
    from paper_1508_07888_b300 import inputs as I
    t = B.rt_group_table(w.edges_eV, w.T_bb)
    return {k: I.f32(v) for k, v in t.items()}


TUNE = 1
CHEM_TUNE = 1


def make_params(w, precision, tune=None, chem_tune=None):
    """tune = 1 / chem_tune = 1: the library times the transport's and the
    chemistry's launch shapes at create (outside every timed region) and keeps
    the fastest."""
    tune = TUNE if tune is None else tune
    chem_tune = CHEM_TUNE if chem_tune is None else chem_tune
    from paper_1508_07888_b300 import binding as B
    return B.make_params(w.ngroups, group_table(w), w.c_red, cfl=w.cfl, ots=w.ots,
                         isothermal=w.isothermal, nsub=w.nsub, bc=w.bc, precision=precision,
                         tune=tune, chem_tune=chem_tune, rates_const=w.rates_const, alphaA=w.alphaA,
                         alphaB=w.alphaB, beta=w.beta)


class DeviceRun:
    """The workload resident in HBM (all its boxes in one handle); reset()
    restores the initial state."""

    def __init__(self, w, precision, flux=0):
        import torch
        from paper_1508_07888_b300 import binding as B
        self.torch, self.B, self.w = torch, B, w
        self.p = make_params(w, precision)
        self.p.flux = flux
        fp = torch.float64 if precision != B.RT_PREC_SPLIT else torch.float32
        self.init, states = [], []
        for box in w.boxes:
            U, xHI, T = box.initial_state(w.ngroups)
            U0 = torch.as_tensor(U, dtype=fp, device="cuda")
            x0 = torch.as_tensor(xHI, dtype=torch.float64, device="cuda")
            T0 = torch.as_tensor(T, dtype=torch.float64, device="cuda")
            self.init.append((U0, x0, T0))
            states.append(B.BoxState(U=U0.clone(), xHI=x0.clone(), T=T0.clone(),
                                     n0=torch.as_tensor(box.n0, dtype=fp, device="cuda"),
                                     dx=box.dx, nunit=w.nunit(box)))
        self.states = states
        self.state = states[0]
        self.solver = B.Solver(self.p, states)
        for i, box in enumerate(w.boxes):
            self.solver.set_sources(i, box.src_cells, box.src_Q)
        self.state_bytes = sum(t.numel() * t.element_size()
                               for st in states for t in (st.U, st.xHI, st.T, st.n0))

    def reset(self):
        for st, (U0, x0, T0) in zip(self.states, self.init):
            st.U.copy_(U0)
            st.xHI.copy_(x0)
            st.T.copy_(T0)

    def run(self, nsteps, hist=None):
        code = self.solver.step(nsteps, hist)
        if code != self.B.RT_OK:
            raise RuntimeError(f"rt_step status {code}: {self.B.rt_last_error(self.solver.h)}")

    def close(self):
        self.solver.close()


def time_device(w, precision, K, W, nsteps, ws, profile):
    """K timed bench steps (reset + nsteps radiative steps) after W warm-ups.
    The diagnostics history of every step is written to a device buffer."""
    import torch
    from paper_1508_07888_b300 import binding as B
    r = DeviceRun(w, precision)
    hist = torch.zeros((nsteps, len(w.boxes), B.RT_NDIAG), dtype=torch.float64, device="cuda")
    for _ in range(W):
        r.reset()
        r.run(nsteps, hist)
    B.rt_set_profiling(r.solver.h, profile)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(nsteps, hist)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    st = B.rt_query(r.solver.h)
    kern = {name: {"ms_total": st.kernel_ms[j], "launches": int(st.kernel_launches[j])}
            for j, name in enumerate(B.KERNELS) if st.kernel_launches[j] > 0}
    diag = list(st.last_diag)
    h = hist.cpu().numpy()
    cells = np.array([b.ncell for b in w.boxes], dtype=np.float64)
    mean_sub = float(np.sum(h[:, :, 4] * cells) / (nsteps * cells.sum()))
    nbytes = r.state_bytes
    launch = {"transport_tile": [st.tile_x, st.tile_y], "transport_grid": st.transport_grid,
              "transport_zchunk": st.transport_zchunk, "transport_tma": bool(st.transport_tma),
              "transport_lockstep": st.transport_lockstep,
              "transport_gpb": st.transport_gpb,
              "chemistry_grid": st.chem_grid, "chemistry_grab": st.chem_grab,
              "tuned": bool(r.p.tune), "chemistry_tuned": bool(r.p.chem_tune)}
    r.close()
    return ms, kern, diag, nbytes, mean_sub, launch


def e2e_host(w, precision, K, W, nsteps):
    """Same metric through the C ABI with host buffers: every bench step
    uploads the inputs from pinned host memory, sets the sources, runs, and
    downloads the final state (copies inside the timed region)."""
    import numpy as np
    import torch
    from paper_1508_07888_b300 import binding as B
    box = w.boxes[0]
    fpn = np.float64 if precision != B.RT_PREC_SPLIT else np.float32
    U, xHI, T = box.initial_state(w.ngroups)

    def pinned(a, dt):
        t = torch.empty(a.shape, dtype=torch.from_numpy(np.zeros(1, dt)).dtype, pin_memory=True)
        t.numpy()[...] = a
        return t

    hU, hx, hT, hn = pinned(U, fpn), pinned(xHI, np.float64), pinned(T, np.float64), pinned(box.n0, fpn)
    oU, ox, oT = pinned(U, fpn), pinned(xHI, np.float64), pinned(T, np.float64)
    r = DeviceRun(w, precision)
    h = r.solver.h

    def one():
        B.rt_upload(h, 0, U=hU.numpy(), xHI=hx.numpy(), T=hT.numpy(), n0=hn.numpy())
        B.rt_set_sources(h, 0, box.src_cells, box.src_Q)
        code = B.rt_step(h, nsteps)
        if code != B.RT_OK:
            raise RuntimeError(f"rt_step status {code}")
        B.rt_download(h, 0, U=oU.numpy(), xHI=ox.numpy(), T=oT.numpy())

    for _ in range(W):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        one()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    h2d = sum(a.numel() * a.element_size() for a in (hU, hx, hT, hn)) + box.src_cells.nbytes * 2
    d2h = sum(a.numel() * a.element_size() for a in (oU, ox, oT))
    r.close()
    return sec, h2d, d2h


def cpu_baseline(w, steps, points=(0, 100, 250)):
    """The FP64 oracle, single-threaded, timed on `steps` radiative steps at
    each of `points` (step indices spread over the run, so that the sample
    carries the later steps' chemistry work too); between the points the
    oracle advances its own state on every host core, untimed."""
    import oracle as O
    box = w.boxes[0]
    t = O.group_table(w.edges_eV, w.T_bb)
    from paper_1508_07888_b300 import inputs as I
    t = {k: I.f32(v) for k, v in t.items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 cfl=w.cfl, ots=w.ots, isothermal=w.isothermal, nsub=w.nsub, bc=list(w.bc))
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, xHI, T = box.initial_state(w.ngroups)
    at, sec, timed = 0, 0.0, 0
    for k in points:
        if k > at:
            O.set_threads(os.cpu_count() or 1)
            r = O.run(p, U, xHI, T, box.n0, box.dx, nunit, k - at, S)
            U, xHI, T, at = r.U, r.xHI, r.T, k
        O.set_threads(1)
        t0 = time.perf_counter()
        r = O.run(p, U, xHI, T, box.n0, box.dx, nunit, steps, S)
        sec += time.perf_counter() - t0
        U, xHI, T, at = r.U, r.xHI, r.T, at + steps
        timed += steps
    O.set_threads(1)
    where = ", ".join(f"{k + 1}-{k + steps}" for k in points)
    return {"value": box.ncell * timed / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"radiative steps {where} of the same 128^3 3-group workload "
                      f"({sec:.1f} s timed, FP64 C oracle, 1 thread; the oracle advances its "
                      f"own state between the sampled steps on all host cores, untimed)",
            "cpu": cpu_model(), "host_cpu_count": os.cpu_count()}


def reion256_run(B, ws, K=3, nsteps=20):
    """The 256^3 workload (sigma = 1.5, P ~ k^-2.5, 1024 sources with
    Q ~ n0^1.5, 3 groups, c/20, 8 fixed chemistry intervals per step), split
    form, 20 radiative steps per run (of its 200): its state (805 MB of FP32
    radiation) is far beyond the 126 MB L2, so the transport's HBM rate is
    clean of cache reuse.  Per-kernel times by CUDA events."""
    import torch
    from paper_1508_07888_b300 import inputs as I
    w = I.reion_large()
    r = DeviceRun(w, B.RT_PREC_SPLIT)
    r.reset()
    r.run(nsteps)
    B.rt_set_profiling(r.solver.h, 1)
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(nsteps)
    e1.record()
    torch.cuda.synchronize()
    val, sec = replica_value(ws, w.cells * nsteps * K, e0.elapsed_time(e1) / 1e3)
    st = B.rt_query(r.solver.h)
    r.close()
    t_ms = st.kernel_ms[0] / max(st.kernel_launches[0], 1)
    c_ms = st.kernel_ms[1] / max(st.kernel_launches[1], 1)
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6400.0
    gbs = 32.0 * w.ngroups * w.cells / (t_ms * 1e-3) / 1e9
    return {"workload": w.name + " (sigma=1.5, P~k^-2.5, 1024 sources, 3 groups, c/20, nsub=8)",
            "value": val, "unit": UNIT, "cells": w.cells, "rt_steps_per_run": nsteps,
            "ms_per_run": sec * 1e3 / K,
            "transport_ms_per_launch": t_ms, "transport_gbs": gbs,
            "transport_frac": gbs / hbm,
            "transport_traffic": profiled_traffic().get(
                "transport_256_lockstep" if st.transport_lockstep else "transport_256_columns"),
            "launch": {"transport_tile": [st.tile_x, st.tile_y], "transport_grid": st.transport_grid,
                       "transport_zchunk": st.transport_zchunk, "transport_lockstep": st.transport_lockstep,
                       "transport_tma": bool(st.transport_tma), "transport_gpb": st.transport_gpb,
                       "chemistry_grid": st.chem_grid, "chemistry_grab": st.chem_grab},
            "chemistry_ms_per_launch": c_ms,
            "peak_note": "of measured" if pk else "of fallback"}


def ensemble_run(B, ws, K=3):
    """The batched workload: 64 periodic boxes of side 32-96 (2 groups, 1-16
    sources each) in one handle, 100 radiative steps per run, each step one
    launch per kernel over all boxes, replayed from the captured graph."""
    import torch
    from paper_1508_07888_b300 import inputs as I
    w = I.ensemble()
    r = DeviceRun(w, B.RT_PREC_SPLIT)
    r.reset()
    r.run(w.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(w.steps)
    e1.record()
    torch.cuda.synchronize()
    val, sec = replica_value(ws, w.cells * w.steps * K, e0.elapsed_time(e1) / 1e3)
    ms = sec * 1e3
    r.close()
    return {"value": val, "unit": UNIT,
            "ms_per_run": ms / K, "boxes": len(w.boxes), "cells": w.cells,
            "rt_steps_per_run": w.steps, "launches_per_step": 2, "graph": True}


def crta_run(K=3, nsteps=100):
    """CRTA fine level (Sec. 5): the 128^3 workload with its densest eighth
    refined into 8 children each (2,097,152 refined cells, densities
    lognormal around the parent's), 100 steps per run; the fine chemistry
    runs after the coarse chemistry of every step, timed by CUDA events."""
    import torch
    from paper_1508_07888_b300 import binding as B
    from paper_1508_07888_b300 import inputs as I
    w = workload()
    fine = I.refine_densest(w.boxes[0], frac=0.125, seed=7)
    r = DeviceRun(w, B.RT_PREC_SPLIT)
    x0 = torch.as_tensor(fine.xHI, device="cuda")
    T0 = torch.as_tensor(fine.T, device="cuda")
    xf, Tf = r.solver.set_fine(0, fine.parent, fine.n0, fine.xHI, fine.T)
    def reset():
        r.reset()
        xf.copy_(x0)
        Tf.copy_(T0)
    reset()
    r.run(nsteps)
    B.rt_set_profiling(r.solver.h, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        reset()
        r.run(nsteps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = B.rt_query(r.solver.h)
    r.close()
    nf = fine.parent.size
    fine_ms = st.kernel_ms[2] / max(st.kernel_launches[2], 1)
    return {"workload": "reion_128^3_g3 + densest 1/8 refined x8", "fine_cells": int(nf),
            "rt_steps_per_run": nsteps, "ms_per_run": ms / K,
            "fine_ms_per_step": fine_ms,
            "fine_cell_updates_per_s": nf / (fine_ms * 1e-3),
            "all_cell_updates_per_s": (w.cells + nf) * nsteps * K / (ms * 1e-3)}


def hll_run(K=3, nsteps=None):
    """The HLL flux (the less diffusive flux the paper plans) on the same
    128^3 workload, split form, 500 steps per run: whole-step throughput and
    the transport kernel's time and HBM rate (algorithmic 32 B per
    cell-group)."""
    import torch
    from paper_1508_07888_b300 import binding as B
    w = workload()
    nsteps = nsteps or w.steps
    r = DeviceRun(w, B.RT_PREC_SPLIT, flux=1)
    r.reset()
    r.run(nsteps)
    B.rt_set_profiling(r.solver.h, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(nsteps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = B.rt_query(r.solver.h)
    r.close()
    t_ms = st.kernel_ms[0] / max(st.kernel_launches[0], 1)
    return {"value": w.cells * nsteps * K / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms / K,
            "transport_ms_per_launch": t_ms,
            "transport_gbs": 32.0 * w.ngroups * w.cells / (t_ms * 1e-3) / 1e9,
            "transport_traffic": profiled_traffic().get("transport_hll"),
            "chemistry_ms_per_launch": st.kernel_ms[1] / max(st.kernel_launches[1], 1)}


def cosmo_run(K=3):
    """The 128^3 workload in supercomoving units (Sec. 3): a0 = 0.1,
    H0 = 67.7 km/s/Mpc, omega_m = 0.31, omega_l = 0.69, split form, 500
    steps per run; throughput against the static run shows the cost of the
    per-step scalings."""
    import torch
    from paper_1508_07888_b300 import binding as B
    w = workload()
    r = DeviceRun(w, B.RT_PREC_SPLIT)
    r.p.cosmo, r.p.H0, r.p.omega_m, r.p.omega_l, r.p.a0 = 1, 2.194e-18, 0.31, 0.69, 0.1
    r.solver.close()
    r.solver = B.Solver(r.p, r.states)
    for i, box in enumerate(w.boxes):
        r.solver.set_sources(i, box.src_cells, box.src_Q)
    r.reset()
    r.run(w.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(w.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    a = B.rt_query(r.solver.h).a
    r.close()
    return {"value": w.cells * w.steps * K / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms / K,
            "a_after_all_runs": a, "a0": 0.1}


def adjoint_run():
    """The adjoint workload (64^3, 16 sources, 1 group, 4 fixed chemistry
    intervals, 200 steps, checkpoints every 20): forward and reverse time of
    one gradient of an ionised-fraction-history loss."""
    import torch
    from paper_1508_07888_b300 import binding as B
    from paper_1508_07888_b300 import inputs as I
    from paper_1508_07888_b300.autograd import HistoryRun, ionisation_history
    w = I.adjoint_box()
    box = w.boxes[0]
    t = B.rt_group_table(w.edges_eV, w.T_bb)
    t = {k: I.f32(v) for k, v in t.items()}
    p = B.make_params(1, t, w.c_red, nsub=w.nsub, precision=B.RT_PREC_FP64)
    U, xHI, T = box.initial_state(1)
    st = B.BoxState(U=torch.as_tensor(U, device="cuda"), xHI=torch.as_tensor(xHI, device="cuda"),
                    T=torch.as_tensor(T, device="cuda"),
                    n0=torch.as_tensor(box.n0, dtype=torch.float64, device="cuda"),
                    dx=box.dx, nunit=w.nunit(box))
    run = HistoryRun(p, st, box.src_cells, w.steps, ckpt_every=20)
    Q = torch.tensor(box.src_Q, dtype=torch.float64, requires_grad=True)
    n0 = torch.as_tensor(box.n0, dtype=torch.float64, device="cuda").requires_grad_(True)
    with torch.no_grad():
        Xt = ionisation_history(Q * torch.as_tensor(I.target_perturbation(len(box.src_Q))), n0, run)
    X = ionisation_history(Q, n0, run)                    # warm-up
    ((X - Xt) ** 2).mean().backward()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = ionisation_history(Q, n0, run)
    L = ((X - Xt) ** 2).mean()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    run.close()
    fwd = box.ncell * w.steps / (t1 - t0)
    return {"workload": w.name, "forward_ms": 1e3 * (t1 - t0), "backward_ms": 1e3 * (t2 - t1),
            "forward_cell_updates_per_s": fwd, "backward_over_forward": (t2 - t1) / (t1 - t0),
            "form": "FP64", "checkpoint_every": 20}


def profiled_traffic():
    """DRAM bytes per launch of each kernel from the committed ncu summary,
    kept only while the kernel source still has the hash it was captured at."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1508_07888_b300", "csrc", "rt_kernels.cuh")
    out = {}
    try:
        digest = hashlib.sha1(open(src, "rb").read()).hexdigest()
        for line in open(path):
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[3] == digest:
                out[f[0]] = float(f[2])
    except OSError:
        pass
    return out


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def chem_flops_per_subcycle(G: int, ots: bool, split: bool = True, adaptive: bool = True) -> float:
    """Algorithmic FP64 flops of one accepted chemistry sub-cycle (a5-a8 and
    the rate fits), counted from the formulas as written.  The split form
    runs the photon update of each group (1 + c sigma x_HI n0 dtau: 4, (N + S
    dtau)/den: 3, F/den: 3) in FP32, 10 G flops that are not FP64 work, and
    the recombination photons of group 1 ((alpha_A - alpha_B) x^2 n0^2 /
    nunit: 7 flops, absent with OTS) too.  OTS also drops the alpha_A fit (7).
    The dtau estimate |e / (H - Lambda)| (4 G + 19) belongs to adaptive
    sub-cycling only: with a fixed number of sub-cycles there is none."""
    base = 111.0 - (14.0 if ots else (7.0 if split else 0.0))
    if not adaptive:
        base -= 19.0 + 4.0 * G
    return (12.0 if split else 22.0) * G + base


# FP64 flops of one GLF transport cell-group, counted from the formulas as
# written (+ - x / sqrt each 1): closure 42 (F/N 3, f^2 5, s 3, a 6, g 4,
# P 21), three faces of 16 (each face shared by two cells), update 28
TRANSPORT_FP64_FLOPS = 118.0


def fp64_peak_tflops():
    """FP64 pipe: 148 SMs x 2 DFMA/clock x 2 flop x 2032 MHz (a DFMA loop
    measured 1.97 DFMA/clock/SM at the clock it ran at)."""
    return 148 * 2 * 2 * 2032e6 / 1e12


def oracle_sample(w, steps, boxes=None):
    """1-thread oracle rate (cell-updates/s) on the first `steps` steps of
    the given boxes (all by default): a bounded sample of the workload."""
    import oracle as O
    from paper_1508_07888_b300 import inputs as I
    t = O.group_table(w.edges_eV, w.T_bb)
    t = {k: I.f32(v) for k, v in t.items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 cfl=w.cfl, ots=w.ots, isothermal=w.isothermal, nsub=w.nsub, bc=list(w.bc),
                 rates_const=w.rates_const, alphaA=w.alphaA, alphaB=w.alphaB, beta=w.beta)
    O.set_threads(1)
    cells, sec = 0, 0.0
    for b in (boxes if boxes is not None else range(len(w.boxes))):
        box = w.boxes[b]
        nunit = w.nunit(box)
        S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
        U, xHI, T = box.initial_state(w.ngroups)
        t0 = time.perf_counter()
        O.run(p, U, xHI, T, box.n0, box.dx, nunit, steps, S)
        sec += time.perf_counter() - t0
        cells += box.ncell * steps
    return cells / sec, sec


def config_table():
    """One JSON line per workload x precision form: throughput, per-kernel
    times, the transport's HBM fraction (split: 32 G B, FP64: 64 G B per
    cell; or FP64 flops for the FP64 form's transport) and the chemistry's
    FP64 fraction, and a bounded 1-thread oracle sample of the same
    workload.  Not part of the default run."""
    import torch
    from paper_1508_07888_b300 import binding as B
    from paper_1508_07888_b300 import inputs as I
    torch.cuda.set_device(0)
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6400.0
    f64 = fp64_peak_tflops()
    cfgs = [("1: Stromgren 32^3, 1 group, FP64 constant rates", I.stromgren(32), 100, 20, None),
            ("2: reionisation 128^3, 3 groups, adaptive chemistry", I.reion(), 500, 3, None),
            ("3: reionisation 256^3, 3 groups, c/20, nsub 8 (20 of its 200 steps)",
             I.reion_large(), 20, 1, None),
            ("4: ensemble of 64 boxes 32-96^3, 2 groups", I.ensemble(), 100, 2, [0, 1, 2, 3])]
    for name, w, nsteps, osteps, oboxes in cfgs:
        orate, osec = oracle_sample(w, osteps, oboxes)
        for prec, pname in ((B.RT_PREC_SPLIT, "split"), (B.RT_PREC_FP64, "fp64")):
            ms, kern, diag, nbytes, mean_sub, launch = time_device(w, prec, 2, 1, nsteps, 1,
                                                                   profile=True)
            cells = w.cells
            per = {k: v["ms_total"] / max(v["launches"], 1) for k, v in kern.items()}
            G = w.ngroups
            row = {"config": name, "form": pname, "value": cells * nsteps * 2 / (ms * 1e-3),
                   "unit": UNIT, "rt_steps": nsteps, "kernels_ms_per_launch": per,
                   "mean_subcycles": mean_sub,
                   "oracle_1thread": {"value": orate, "sample": f"{osteps} steps, "
                                      + (f"boxes {oboxes}" if oboxes else "whole workload"),
                                      "seconds": osec}}
            t = per.get("transport")
            if t:
                if prec == B.RT_PREC_SPLIT:
                    gbs = 32.0 * G * cells / (t * 1e-3) / 1e9
                    row["transport_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": hbm,
                                                 "unit": "GB/s", "frac": gbs / hbm}
                else:
                    tf = TRANSPORT_FP64_FLOPS * G * cells / (t * 1e-3) / 1e12
                    gbs = 64.0 * G * cells / (t * 1e-3) / 1e9
                    row["transport_roofline"] = {"bound": "alu", "achieved": tf, "peak": f64,
                                                 "unit": "TFLOP/s", "frac": tf / f64,
                                                 "hbm_frac": gbs / hbm}
            c = per.get("chemistry")
            if c and not w.rates_const:
                fl = chem_flops_per_subcycle(G, w.ots, prec == B.RT_PREC_SPLIT,
                                             adaptive=w.nsub == 0) * cells * mean_sub
                tf = fl / (c * 1e-3) / 1e12
                row["chemistry_roofline"] = {"bound": "alu", "achieved": tf, "peak": f64,
                                             "unit": "TFLOP/s", "frac": tf / f64}
            print(json.dumps(row), flush=True)
    print(json.dumps({"config": "5: adjoint 64^3, 1 group, 200 steps", "form": "fp64",
                      **adjoint_run()}), flush=True)


def main():
    global TUNE, CHEM_TUNE
    args = parse()
    TUNE = args.tune
    CHEM_TUNE = args.chem_tune
    if args.config_table:
        config_table()
        return
    if args.only:
        import torch
        from paper_1508_07888_b300 import binding as B
        torch.cuda.set_device(0)
        row = {"reion256": lambda: reion256_run(B, 1, K=args.steps, nsteps=args.rt_steps),
               "ensemble": lambda: ensemble_run(B, 1, K=args.steps),
               "hll": lambda: hll_run(K=args.steps, nsteps=args.rt_steps)}[args.only]()
        print(json.dumps({"only": args.only, **row}), flush=True)
        return
    ws, rank, local = dist_setup(args)
    w = workload()
    box = w.boxes[0]
    nsteps = args.rt_steps
    units_per_step = box.ncell * nsteps

    if args.impl == "reference":
        if rank != 0:
            return
        # the reference arm: the CPU oracle as it stands, each bench step a
        # bounded sample (2 radiative steps) of the workload
        import oracle as O
        t = O.group_table(w.edges_eV, w.T_bb)
        from paper_1508_07888_b300 import inputs as I
        t = {k: I.f32(v) for k, v in t.items()}
        p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"],
                     c=w.c_red, cfl=w.cfl, bc=list(w.bc))
        nunit = w.nunit(box)
        S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
        O.set_threads(1)
        per = 2
        U, xHI, T = box.initial_state(w.ngroups)
        for _ in range(args.warmup):
            O.run(p, U, xHI, T, box.n0, box.dx, nunit, 1, S)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            O.run(p, U, xHI, T, box.n0, box.dx, nunit, per, S)
        sec = time.perf_counter() - t0
        val = box.ncell * per * args.steps / sec
        sample = (f"{per} radiative steps of the 128^3 3-group workload per bench step "
                  f"(FP64 C oracle, 1 thread)")
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": box.ncell, "rt_steps_per_bench_step": per},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    import torch
    from paper_1508_07888_b300 import binding as B
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    B.lib()

    clocks = Clocks(local)
    clocks.start()
    ms, kern, diag, state_bytes, mean_sub, launch = time_device(w, B.RT_PREC_SPLIT, args.steps,
                                                                args.warmup, nsteps, ws, profile=True)
    clk = clocks.stop()
    value, sec = replica_value(ws, units_per_step * args.steps, ms / 1e3)
    ms = sec * 1e3
    ms_step = ms / args.steps

    fp64 = None
    if not args.no_fp64_form:
        ms64, kern64, _, _, _, _ = time_device(w, B.RT_PREC_FP64, args.steps, args.warmup, nsteps,
                                            ws, profile=True)
        v64, sec64 = replica_value(ws, units_per_step * args.steps, ms64 / 1e3)
        ms64 = sec64 * 1e3
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.steps,
                "split_over_fp64": value / v64,
                "kernels_ms_per_launch": {k: v["ms_total"] / max(v["launches"], 1)
                                          for k, v in kern64.items()}}

    e2e = None
    if not args.no_e2e:
        sec, h2d, d2h = e2e_host(w, B.RT_PREC_SPLIT, args.steps, min(args.warmup, 1), nsteps)
        v_e2e, sec = replica_value(ws, units_per_step * args.steps, sec)
        e2e = {"value": v_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # per-kernel shares and the rooflines (algorithmic units per launch over
    # the CUDA-event launch time measured above)
    tot = sum(v["ms_total"] for v in kern.values())
    per_launch = {k: v["ms_total"] / max(v["launches"], 1) for k, v in kern.items()}
    shares = {k: v["ms_total"] / tot for k, v in kern.items()} if tot > 0 else {}
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6400.0
    peak_note = "of measured" if pk else "of fallback"
    traffic = profiled_traffic()
    G = w.ngroups
    t_bytes = 32.0 * G * box.ncell                  # read + write of (N, F) in FP32, per launch
    t_ach = t_bytes / (per_launch["transport"] * 1e-3) / 1e9
    roof_t = {"kernel": "transport", "bound": "hbm", "achieved": t_ach, "peak": hbm_peak,
              "unit": "GB/s", "frac": t_ach / hbm_peak,
              "traffic": traffic.get("transport"),
              "algorithmic_bytes_per_launch": t_bytes, "peak_note": peak_note}
    # chemistry: FP64 flops of one accepted sub-cycle, counted from the
    # formulas as written (+ - x / each 1; pow, exp, sqrt 1): the rate fits 45
    # (lambda 1, alpha_A 7, alpha_B 7, recombination + free-free cooling 11,
    # beta 11, excitation cooling 6, k_C 2; OTS needs no alpha_A), the dtau
    # estimate 4 G + 19, the trial 18 G + 47 (7 of them the recombination
    # photons of group 1 without OTS) -> 22 G + 111; the split form's photon
    # update (10 G of the trial's flops) and the recombination photons (7)
    # run in FP32 -> 12 G + 104 FP64 flops, against the FP64 pipe peak: 148
    # SMs x 2 DFMA/clock x 2 flop x 2032 MHz
    fp64_peak = fp64_peak_tflops()
    c_flops = chem_flops_per_subcycle(G, w.ots) * box.ncell * mean_sub
    c_ach = c_flops / (per_launch["chemistry"] * 1e-3) / 1e12
    roof_c = {"kernel": "chemistry", "bound": "alu", "achieved": c_ach, "peak": fp64_peak,
              "unit": "TFLOP/s", "frac": c_ach / fp64_peak,
              "traffic": traffic.get("chemistry"),
              "algorithmic_flops_per_launch": c_flops, "mean_subcycles": mean_sub,
              "peak_note": "FP64 pipe, derived from ncu's 2 DFMA/clock/SM and the 2032 MHz "
                           "maximum clock (a DFMA-loop kernel measured 1.97 DFMA/clock/SM at "
                           "the clock it ran at)"}
    dominant = max(shares, key=shares.get) if shares else "transport"
    roofline = roof_c if dominant == "chemistry" else roof_t

    ens = None if args.no_ensemble else ensemble_run(B, ws)
    adj = None if args.no_adjoint else adjoint_run()
    crta = None if args.no_crta else crta_run()
    hll = None if args.no_hll else hll_run()
    cosmo = None if args.no_cosmo else cosmo_run()
    r256 = None if args.no_256 else reion256_run(B, ws)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_sample_steps)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": w.name + " (lognormal sigma=1, P~k^-2, 64 sources, 3 groups "
                                            "5e4 K BB, c/10, T evolving, adaptive chemistry)",
                       "cells": box.ncell, "rt_steps_per_bench_step": nsteps,
                       "form": "split: FP32 transport + FP64 chemistry (x_HI, T, rates, sums; photon update in FP32)",
                       "l2": f"inputs larger than L2 (resident state {state_bytes / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "roofline_transport": roof_t,
            "kernels": {k: {"ms_per_launch": per_launch[k], "share": shares.get(k),
                            "launches": kern[k]["launches"]} for k in kern},
            "launch": launch,
            "fp64_form": fp64, "e2e": e2e, "cpu_baseline": cpu,
            "ensemble": ens, "adjoint": adj, "crta": crta, "hll": hll, "cosmo": cosmo,
            "reion256": r256,
            # the profiled transport and chemistry launches, plus the one launch per
            # rt_step call (one per bench step) that forms the chemistry's per-cell constants
            "gpu_launches": int(sum(v["launches"] for v in kern.values())) + args.steps,
            "clocks": clk, "final_diag": dict(zip(B.DIAG_NAMES, diag)),
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
