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
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

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
    ap.add_argument("--cpu-sample-steps", type=int, default=5)
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


def make_params(w, precision):
    from paper_1508_07888_b300 import binding as B
    return B.make_params(w.ngroups, group_table(w), w.c_red, cfl=w.cfl, ots=w.ots,
                         isothermal=w.isothermal, nsub=w.nsub, bc=w.bc, precision=precision)


class DeviceRun:
    """The workload resident in HBM; reset() restores the initial state."""

    def __init__(self, w, precision):
        import torch
        from paper_1508_07888_b300 import binding as B
        self.torch, self.B, self.w = torch, B, w
        box = w.boxes[0]
        self.p = make_params(w, precision)
        fp = torch.float64 if precision != B.RT_PREC_SPLIT else torch.float32
        U, xHI, T = box.initial_state(w.ngroups)
        dev = "cuda"
        self.U0 = torch.as_tensor(U, dtype=fp, device=dev)
        self.x0 = torch.as_tensor(xHI, dtype=torch.float64, device=dev)
        self.T0 = torch.as_tensor(T, dtype=torch.float64, device=dev)
        st = B.BoxState(U=self.U0.clone(), xHI=self.x0.clone(), T=self.T0.clone(),
                        n0=torch.as_tensor(box.n0, dtype=fp, device=dev), dx=box.dx,
                        nunit=w.nunit(box))
        self.state = st
        self.solver = B.Solver(self.p, [st])
        self.solver.set_sources(0, box.src_cells, box.src_Q)
        self.state_bytes = sum(t.numel() * t.element_size() for t in (st.U, st.xHI, st.T, st.n0))

    def reset(self):
        self.state.U.copy_(self.U0)
        self.state.xHI.copy_(self.x0)
        self.state.T.copy_(self.T0)

    def run(self, nsteps):
        code = self.solver.step(nsteps)
        if code != self.B.RT_OK:
            raise RuntimeError(f"rt_step status {code}: {self.B.rt_last_error(self.solver.h)}")

    def close(self):
        self.solver.close()


def time_device(w, precision, K, W, nsteps, ws, profile):
    """K timed bench steps (reset + nsteps radiative steps) after W warm-ups."""
    import torch
    from paper_1508_07888_b300 import binding as B
    r = DeviceRun(w, precision)
    for _ in range(W):
        r.reset()
        r.run(nsteps)
    B.rt_set_profiling(r.solver.h, profile)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        r.reset()
        r.run(nsteps)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    st = B.rt_query(r.solver.h)
    kern = {name: {"ms_total": st.kernel_ms[j], "launches": int(st.kernel_launches[j])}
            for j, name in enumerate(B.KERNELS) if st.kernel_launches[j] > 0}
    diag = list(st.last_diag)
    nbytes = r.state_bytes
    r.close()
    return ms, kern, diag, nbytes


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


def cpu_baseline(w, steps):
    """The FP64 oracle, single-threaded, on the first `steps` radiative steps
    of the same workload."""
    import oracle as O
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    box = w.boxes[0]
    t = O.group_table(w.edges_eV, w.T_bb)
    from paper_1508_07888_b300 import inputs as I
    t = {k: I.f32(v) for k, v in t.items()}
    p = O.Params(sigN=t["sigN"], sigE=t["sigE"], Eavg=t["Eavg"], frac=t["frac"], c=w.c_red,
                 cfl=w.cfl, ots=w.ots, isothermal=w.isothermal, nsub=w.nsub, bc=list(w.bc))
    nunit = w.nunit(box)
    S = O.source_field(p, box.shape, box.src_cells, box.src_Q, box.dx, nunit)
    U, xHI, T = box.initial_state(w.ngroups)
    O.set_threads(1)
    t0 = time.perf_counter()
    O.run(p, U, xHI, T, box.n0, box.dx, nunit, steps, S)
    sec = time.perf_counter() - t0
    return {"value": box.ncell * steps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"radiative steps 1-{steps} of the same 128^3 3-group workload "
                      f"({sec:.1f} s, FP64 C oracle, 1 thread; early steps carry fewer "
                      f"chemistry sub-cycles than the 500-step average)",
            "cpu": cpu_model(), "host_cpu_count": os.cpu_count()}


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


def main():
    args = parse()
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
    ms, kern, diag, state_bytes = time_device(w, B.RT_PREC_SPLIT, args.steps, args.warmup,
                                              nsteps, ws, profile=True)
    clk = clocks.stop()
    ms = max_over_ranks(ws, ms)
    value = units_per_step * args.steps * ws / (ms / 1e3)
    ms_step = ms / args.steps

    fp64 = None
    if not args.no_fp64_form:
        ms64, kern64, _, _ = time_device(w, B.RT_PREC_FP64, args.steps, args.warmup, nsteps, ws,
                                         profile=True)
        ms64 = max_over_ranks(ws, ms64)
        v64 = units_per_step * args.steps * ws / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.steps,
                "split_over_fp64": value / v64,
                "kernels_ms_per_launch": {k: v["ms_total"] / max(v["launches"], 1)
                                          for k, v in kern64.items()}}

    e2e = None
    if not args.no_e2e:
        sec, h2d, d2h = e2e_host(w, B.RT_PREC_SPLIT, args.steps, min(args.warmup, 1), nsteps)
        sec = max_over_ranks(ws, sec)
        e2e = {"value": units_per_step * args.steps * ws / sec, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # per-kernel shares and the roofline of the dominant kernel
    tot = sum(v["ms_total"] for v in kern.values())
    per_launch = {k: v["ms_total"] / max(v["launches"], 1) for k, v in kern.items()}
    shares = {k: v["ms_total"] / tot for k, v in kern.items()} if tot > 0 else {}
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6400.0
    peak_note = "of measured" if pk else "of fallback"
    G = w.ngroups
    t_bytes = 32.0 * G * box.ncell                  # read + write of (N, F) in FP32, per launch
    t_ach = t_bytes / (per_launch["transport"] * 1e-3) / 1e9
    roof_t = {"kernel": "transport", "bound": "hbm", "achieved": t_ach, "peak": hbm_peak,
              "unit": "GB/s", "frac": t_ach / hbm_peak, "traffic": None,
              "algorithmic_bytes_per_launch": t_bytes, "peak_note": peak_note}
    dominant = max(shares, key=shares.get) if shares else "transport"
    c_bytes = (32.0 * G + 36.0) * box.ncell        # chemistry: read U*, xHI, T, n0; write U, xHI, T
    c_ach = c_bytes / (per_launch["chemistry"] * 1e-3) / 1e9
    roof_c = {"kernel": "chemistry", "bound": "alu", "achieved": c_ach, "peak": hbm_peak,
              "unit": "GB/s", "frac": c_ach / hbm_peak, "traffic": None,
              "algorithmic_bytes_per_launch": c_bytes,
              "note": "FP64-pipe bound; bytes/launch over time shown against HBM peak"}
    roofline = roof_c if dominant == "chemistry" else roof_t

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
                       "form": "split: FP32 transport + FP64 chemistry",
                       "l2": f"inputs larger than L2 (resident state {state_bytes / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "roofline_transport": roof_t,
            "kernels": {k: {"ms_per_launch": per_launch[k], "share": shares.get(k),
                            "launches": kern[k]["launches"]} for k in kern},
            "fp64_form": fp64, "e2e": e2e, "cpu_baseline": cpu,
            "gpu_launches": int(sum(v["launches"] for v in kern.values())),
            "clocks": clk, "final_diag": dict(zip(B.DIAG_NAMES, diag)),
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
