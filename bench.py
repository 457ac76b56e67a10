"""Throughput of the thermocapillary two-phase step on GB300.

Workload: the 256^3 melt-pool surrogate (liquid rho 7900 under gas rho 1,
dsigma/dT = -4.3e-4 N/(m K), moving Gaussian surface heat flux, seeded 1 %
temperature perturbation), mixed-precision step (float transport, double
projection refinement to ||r|| <= 1e-10 ||b||), dt from the stability limits.
A step is one full SSP-RK3 step: three stages, three projections.

Metric: cell-updates per second = cells / step time (whole job: summed over
ranks; with more than one GPU each rank runs an independent replica).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line is printed by rank 0.  ``--impl reference`` times the CPU
oracle on the host cores (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per full step at 256^3 (FP64 vs mixed) & HBM roofline %"
UNIT = "cell-updates/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM = 6800.0
# FP64 flops per cell of one launch of an FP64-bound class: the mixed-form
# residual takes per coupled face a difference and an FMA (2 flops + 1, 6
# faces), then b - w*acc and the r^2 accumulation (2 + 2)
FP64_FLOPS_PER_CELL = {"residual64": 22}


def alg_bytes_per_cell(cls: str, mixed: bool) -> float | None:
    """Algorithmic bytes per cell of one launch, counted the way the
    measurement plan counts them: one smoothing sweep (both colours) touches
    p (read and write), b and alpha, 4 accesses, so one colour launch is 2
    accesses; the residual restriction p, b, alpha and 1/8 of a coarse
    value; the prolongation 1/8 coarse and p read and written; the stage
    kernels every field they must read or write once.  s = 4 (mixed) or
    8 (FP64); the double projection fields (b, p) are 8 in both forms."""
    s = 4 if mixed else 8
    table = {
        "gs_fine": 2 * s,                        # one colour: half of (p r+w, b, alpha)
        "gs_fused_pre": 4 * s,                   # fused sweeps: p r+w, b, alpha once per launch
        "gs_fused_post": 4 * s + s / 8,          # ... and the coarse correction (1/8)
        "restrict_fine": 3 * s + s / 8,
        "prolong_fine": 2 * s + s / 8,
        "momentum": 9 * s + 3 * s,               # u,v,w,alpha,T,kappa,M0..2 in; u*,v*,w* out
        "scalars": 7 * s + 2 * s,                # u,v,w,alpha,T,Sn alpha,Sn T in; alpha,T out
        "interface": 2 * s + 4 * s,              # alpha, T in; kappa, M out
        "smooth": 2 * s,
        "div_rhs": 3 * s + 8,
        "correct": 6 * s + 8 + s + 3 * s,        # u*, Sn u, p, alpha in; u out
        "residual64": 8 + 8 + 4 + 4 + 4,         # p, b, alpha in; float r and the first sweep's e out
        "add_correction": 8 + 4 + 8,
        "beta": s + 3 * s,
    }
    return table.get(cls)


def compulsory_bytes_per_cell(cls: str, mixed: bool) -> float | None:
    """Bytes per cell each launch must move with the data layout of the
    library (three stored face-coefficient arrays beta instead of alpha,
    colour-strided sweeps that stream every cache line of x and b)."""
    s = 4 if mixed else 8
    table = {
        "gs_fine": 2 * s + s + 3 * s,            # x read+write, b, three betas
        "gs_fused_pre": 2 * s + s + 3 * s,
        "gs_fused_post": 2 * s + s + 3 * s + s / 8,
        "restrict_fine": 2 * s + s + 3 * s + 2 * s / 8,
        "prolong_fine": 2 * s + s / 8,
        "residual64": 8 + 8 + 3 * 4 + 4 + 4,     # p, b, float beta in; float r, e out
        "correct": 6 * s + 8 + 3 * s + 3 * s,    # u*, Sn u, p, beta in; u out
        "beta": s + 3 * s,
    }
    return table.get(cls, alg_bytes_per_cell(cls, mixed))


def whole_step_alg_bytes(mixed: bool, nbar_v: float, n_outer: float) -> float:
    """Algorithmic bytes per cell of one full step (three stages) with
    nbar_v V-cycles and n_outer double refinements per stage: mixed
    3 (120 + 100 nbar_v + 40 n_outer), FP64 3 (208 + 195 nbar_v)."""
    if mixed:
        return 3.0 * (120.0 + 100.0 * nbar_v + 40.0 * n_outer)
    return 3.0 * (208.0 + 195.0 * nbar_v)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per axis (default 256)")
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="grid of the melt-pool surrogate (overrides --n), e.g. 512 512 256")
    ap.add_argument("--mg-pre", type=int, default=None, help="pre-smoothing sweeps (default 2)")
    ap.add_argument("--mg-post", type=int, default=None, help="post-smoothing sweeps (default 2)")
    ap.add_argument("--mg-coarse", type=int, default=None,
                    help="sweeps before and after the correction on the coarse levels (default 3)")
    ap.add_argument("--mg-levels", type=int, default=None,
                    help="cap on the multigrid hierarchy depth (default: the workload's)")
    ap.add_argument("--f64-steps", type=int, default=3, help="steps of the FP64 side measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--copy-streams", type=int, default=6, help="copy streams of the host-buffer measurement")
    ap.add_argument("--copy-chunks", type=int, default=1, help="chunks per field of the host-buffer measurement")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the mixed-against-FP64 error report at 64^3")
    ap.add_argument("--channel-steps", type=int, default=20,
                    help="steps of the thermocapillary-channel side measurement (0: skip)")
    ap.add_argument("--mx-inner", type=int, default=None,
                    help="float V-cycles per double refinement of the mixed solve (default: the "
                         "workload's, 2)")
    ap.add_argument("--adjoint", action="store_true",
                    help="instead: the FP64 adjoint workload (gradient of the interface-height "
                         "objective through a checkpointed rollout, and the adjoint step's cost)")
    ap.add_argument("--adj-n", type=int, default=192, help="adjoint workload: cells per axis")
    ap.add_argument("--adj-steps", type=int, default=200, help="adjoint workload: rollout steps")
    ap.add_argument("--adj-every", type=int, default=20, help="adjoint workload: checkpoint interval")
    ap.add_argument("--droplet", action="store_true",
                    help="instead: the migrating droplet of the paper's Sec. V-A at 100 x 100, FP64 "
                         "(validation run, one JSON line)")
    ap.add_argument("--droplet-steps", type=int, default=2000,
                    help="droplet: steps to run (the paper's t = 0.12 s is about 28000)")
    ap.add_argument("--c5", action="store_true",
                    help="instead: the 512x512x256 melt-pool surrogate by multigrid depth, FP64 "
                         "and mixed, with the adjoint step timed beside it (one JSON line)")
    ap.add_argument("--droplet-coarse-rtol", type=float, default=None,
                    help="droplet: stopping tolerance of the coarsest-level CG (default 1e-12)")
    ap.add_argument("--fd", action="store_true",
                    help="adjoint workload: also central differences in theta (4 more rollouts)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# the sources of the forward kernels (the adjoint's files do not change them)
FORWARD_SOURCES = ("fvm_device.cuh", "fvm_internal.h", "fvm_mg.cu", "fvm_stage.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2209_09671_gb300", "csrc")
    for name in FORWARD_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(cls: str, mixed: bool, ncells: int):
    """DRAM bytes per launch from the committed ncu summary, scaled from the
    captured grid to ncells cells (the traffic of these kernels grows in
    proportion to the cells), or None when the kernels changed since it was
    taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    key = f"{cls}/{'mixed' if mixed else 'f64'}"
    v = d.get("per_launch_bytes", {}).get(key)
    if v is None:
        return None
    return float(v) * ncells / float(d.get("cells", 256 ** 3))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[0]) for s in self.samples if len(s) >= 8 and s[0].replace(".", "").isdigit()]
        smax = [float(s[1]) for s in self.samples if len(s) >= 8 and s[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for s in self.samples:
            if len(s) < 8:
                continue
            for k, name in enumerate(names):
                if s[4 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def cpu_oracle_sample(target_s: float = 12.0, threads: int | None = None):
    """The FP64 oracle on the host cores: melt-pool recipe (same h, physics and
    seed) at 48^3, as many steps as fit in about target_s seconds (1 to 24),
    with `threads` torch threads (None: all the host's cores)."""
    import torch

    import cases
    from oracle import fvm_oracle as O
    n = 48
    before = torch.get_num_threads()
    nthreads = threads if threads else (os.cpu_count() or before)
    torch.set_num_threads(nthreads)
    p, s = cases.melt_pool(n, n, n, precision=cases.F64)
    t0 = time.perf_counter()
    st = s
    steps = 0
    while True:
        st, _ = O.step(st, p, steps, 0.0)
        steps += 1
        if time.perf_counter() - t0 >= target_s or steps >= 24:
            break
    el = time.perf_counter() - t0
    used = torch.get_num_threads()
    torch.set_num_threads(before)
    return {"value": n ** 3 * steps / el, "unit": UNIT, "cores": used,
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle, melt-pool recipe at {n}^3 (h, physics, seed of the 256^3 "
                      f"workload), {steps} full steps in {el:.1f} s on {used} thread(s)"}


def cpu_baselines():
    """The oracle sample at the host's core count (the reported baseline) and
    at one thread beside it."""
    full = cpu_oracle_sample(12.0, None)
    one = cpu_oracle_sample(8.0, 1)
    full["single_thread"] = {k: one[k] for k in ("value", "cores", "sample")}
    return full


def run_reference(args, rank, world):
    if rank != 0:
        return
    cb = cpu_oracle_sample(target_s=20.0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": None, "warmup": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "melt-pool surrogate (CPU oracle sample, 48^3 of the "
                                   "256^3 recipe)", "grid": [48, 48, 48]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def adjoint_workload(n):
    """The thermocapillary channel (equal unit properties, Dirichlet
    dT cos(2 pi x/L) bottom wall with dT = 10, an interface at mid-height
    carrying a seeded ripple of 0.6 cells) at n x n x n with a stationary
    Gaussian surface source of power 20 at the centre of the interface, FP64,
    projections to 1e-11.  The objective is the squared deviation of the
    column interface heights from the heights the same rollout reaches
    without thermocapillary driving (dsigma/dT = 0 and no source):
    J = sum (H - H_ref)^2 h^2.  J is then the square of the thermocapillary
    deformation alone (dJ/dtheta theta / J = 2 and 1), so central
    differences keep their digits."""
    import cases
    p, s = cases.adjoint_channel(nx=n, ny=n, nz=n, dT=10.0, q_power=20.0, ripple=0.6)
    p = p.replace(precision=cases.F64, mg_rtol=1e-11, mg_max_cycles=200, adjoint=1)
    return p, s


def run_adjoint(args, rank, world, local_rank):
    """One JSON line: cost of fvm_step_adjoint against fvm_step at the same
    size, and the gradient dJ/dtheta of the interface-height objective after
    --adj-steps steps (checkpoint every --adj-every), optionally checked
    against central differences of the forward rollout."""
    import torch

    import paper_2209_09671_gb300 as P
    from paper_2209_09671_gb300 import adjoint as ADJ
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p, s0 = adjoint_workload(args.adj_n)
    N = p.nx * p.ny * p.nz
    stream = torch.cuda.Stream(device=dev)

    def J_of(alpha):
        H = alpha.sum(dim=0) * p.h
        return ((H - target) ** 2).sum() * p.h * p.h

    with torch.cuda.stream(stream):
        solver = P.Solver(p, device=dev, stream=stream)
        state = P.to_device(s0, False, dev)
        info = solver.fvm_step({k: v.clone() for k, v in state.items()}, 0, 0.0)
        dt = info["dt"]
        dts = [dt] * args.adj_steps
        # the reference heights: the same rollout without thermocapillary driving
        ref_solver = P.Solver(p.replace(adjoint=0, dsigma_dT=0.0, q_power=0.0), device=dev,
                              stream=stream)
        ref_state = {k: v.clone() for k, v in state.items()}
        ADJ.rollout(ref_solver, ref_state, 0, dts)
        target = ref_state["alpha"].sum(dim=0) * p.h
        ref_solver.close()
        del ref_state
        # forward step and adjoint step, timed with events on the solver's stream
        work = {k: v.clone() for k, v in state.items()}
        for q in range(2):
            solver.fvm_step(work, q, dt, info=False)
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for q in range(reps):
            solver.fvm_step(work, 2 + q, dt, info=False)
        e1.record(stream)
        stream.synchronize()
        fwd_ms = e0.elapsed_time(e1) / reps
        gen = torch.Generator(device=dev)
        gen.manual_seed(20220919)
        lam = {k: torch.rand(work[k].shape, generator=gen, dtype=torch.float64, device=dev) - 0.5
               for k in P.fvm.FIELDS5}
        lam_out = {k: torch.empty_like(work[k]) for k in P.fvm.FIELDS5}
        solver.fvm_step_adjoint(work, 5, dt, lam, lam_out)
        solver.fvm_launch_count(reset=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for q in range(reps):
            solver.fvm_step_adjoint(work, 5, dt, lam, lam_out)
        e1.record(stream)
        stream.synchronize()
        adj_ms = e0.elapsed_time(e1) / reps
        adj_launches = solver.fvm_launch_count() / reps
        solver.fvm_profile(True)
        solver.fvm_step_adjoint(work, 5, dt, lam, lam_out)
        prof = solver.fvm_profile_read()
        solver.fvm_profile(False)
        del work, lam, lam_out
        # the gradient through the rollout (checkpointing + recomputation)
        clocks = ClockSampler(local_rank)
        clocks.start()
        theta = torch.tensor([p.dsigma_dT, p.q_power], dtype=torch.float64, device=dev,
                             requires_grad=True)
        ins = {k: state[k].clone().requires_grad_(k != "p") for k in ADJ.STATE_KEYS}
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = ADJ.Rollout.apply(solver, 0, dts, theta,
                                *(ins[k] for k in P.fvm.FIELDS5), ins["p"])
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        J = J_of(out[3])
        J.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        clk = clocks.stop()
        grad = theta.grad.tolist()
        line = {"metric": "adjoint step cost and rollout gradient, FP64",
                "unit": "ms", "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"thermocapillary channel (wall dT 10, rippled interface) + "
                                       f"Gaussian source of power 20, {p.nx}x{p.ny}x{p.nz}, FP64, "
                                       f"projections to 1e-11",
                           "objective": "sum over columns of (H - H_ref)^2 h^2, H_ref the heights of "
                                        "the same rollout with dsigma/dT = 0 and no source",
                           "cells": N, "dt": dt, "rollout_steps": args.adj_steps,
                           "checkpoint_every": args.adj_every},
                "forward_step_ms": fwd_ms, "adjoint_step_ms": adj_ms,
                "adjoint_over_forward": adj_ms / fwd_ms,
                "adjoint_launches_per_step": adj_launches,
                "adjoint_profile_ms": {k: round(v[1], 3) for k, v in prof.items() if v[0]},
                "J": J.item(), "dJ_dtheta": grad,
                "rollout_forward_s": t1 - t0, "rollout_backward_s": t2 - t1,
                "backward_over_forward": (t2 - t1) / (t1 - t0),
                "clocks": clk}
        if args.fd:
            # a second, well-conditioned objective on the same rollout:
            # J_T = sum T^2 h^3 (T changes by O(1), unlike the interface height)
            def JT_of(T):
                return (T ** 2).sum() * p.h ** 3

            theta_T = torch.tensor([p.dsigma_dT, p.q_power], dtype=torch.float64, device=dev,
                                   requires_grad=True)
            ins_T = {k: state[k].clone().requires_grad_(k != "p") for k in ADJ.STATE_KEYS}
            out_T = ADJ.Rollout.apply(solver, 0, dts, theta_T,
                                      *(ins_T[k] for k in P.fvm.FIELDS5), ins_T["p"])
            JT = JT_of(out_T[4])
            JT.backward()
            grad_T = theta_T.grad.tolist()
            fd, fd_T = [], []
            for q, name in enumerate(("dsigma_dT", "q_power")):
                v = getattr(p, name)
                eps = 1e-3 * abs(v)
                Js, JTs = [], []
                for sgn in (1, -1):
                    sv = P.Solver(p.replace(adjoint=0, **{name: v + sgn * eps}), device=dev,
                                  stream=stream)
                    st = {k: x.clone() for k, x in state.items()}
                    ADJ.rollout(sv, st, 0, dts)
                    Js.append(J_of(st["alpha"]).item())
                    JTs.append(JT_of(st["T"]).item())
                    sv.close()
                    del st
                fd.append((Js[0] - Js[1]) / (2 * eps))
                fd_T.append((JTs[0] - JTs[1]) / (2 * eps))
            line["fd"] = {"eps_rel": 1e-3, "dJ_dtheta": fd,
                          "rel_err": [abs(a - b) / abs(b) for a, b in zip(grad, fd)]}
            line["temperature_objective"] = {
                "objective": "sum T^2 h^3 after the same rollout", "J": JT.item(),
                "dJ_dtheta": grad_T, "fd_dJ_dtheta": fd_T,
                "rel_err": [abs(a - b) / abs(b) for a, b in zip(grad_T, fd_T)]}
    print(json.dumps(line), flush=True)


def run_c5(args, rank, world, local_rank):
    """The 512 x 512 x 256 melt-pool surrogate: mixed and FP64 step times for
    multigrid depths 5 to 8 and the full hierarchy, and beside them the FP64
    adjoint step on the same grid (the melt pool's geometry and density
    ratio 7900, with the liquid's viscosity, conductivity and rho c_p in
    both phases: the property set the adjoint supports), one JSON line."""
    import torch

    import cases
    import paper_2209_09671_gb300 as P
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    shape = (512, 512, 256)
    N = shape[0] * shape[1] * shape[2]
    stream = torch.cuda.Stream(device=dev)

    def timed(p, s, steps, warm):
        with torch.cuda.stream(stream):
            sol = P.Solver(p, device=dev, stream=stream)
            st = P.to_device(s, p.precision == cases.MIXED, dev)
            for q in range(warm):
                sol.fvm_step(st, q, 0.0, info=False)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for q in range(steps):
                sol.fvm_step(st, warm + q, 0.0, info=False)
            e1.record(stream)
            stream.synchronize()
            info = sol.fvm_step(st, warm + steps, 0.0, info=True)
            sol.close()
        del st
        torch.cuda.empty_cache()
        ms = e0.elapsed_time(e1) / steps
        return {"ms_per_step": ms, "value": N / (ms / 1e3), "vcycles_last_step": info["vcycles"],
                "rel_residual_last_step": info["rel_residual"]}

    sweep = {}
    for prec, name, steps in ((cases.MIXED, "mixed", 3), (cases.F64, "f64", 2)):
        for depth in (5, 6, 7, 8, 16):
            p, s = cases.melt_pool(*shape, precision=prec)
            p = p.replace(mg_levels=depth)
            sweep.setdefault(name, {})[str(depth)] = timed(p, s, steps, 1)
    # adjoint step beside the forward step at the same size and dt
    p, s = cases.melt_pool(*shape, precision=cases.F64)
    liq = 1
    rcp = p.rho[liq] * p.cp[liq]
    p = p.replace(mu=(p.mu[liq], p.mu[liq]), lam=(p.lam[liq], p.lam[liq]),
                  cp=(rcp / p.rho[0], p.cp[liq]), adjoint=1)
    with torch.cuda.stream(stream):
        sol = P.Solver(p, device=dev, stream=stream)
        st = P.to_device(s, False, dev)
        info = sol.fvm_step(st, 0, 0.0, info=True)
        dt = info["dt"]
        gen = torch.Generator(device=dev)
        gen.manual_seed(20220919)
        lam = {k: torch.rand(st[k].shape, generator=gen, dtype=torch.float64, device=dev) - 0.5
               for k in P.fvm.FIELDS5}
        lam_out = {k: torch.empty_like(st[k]) for k in P.fvm.FIELDS5}
        sol.fvm_step_adjoint(st, 1, dt, lam, lam_out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        sol.fvm_step(st, 1, dt, info=False)
        e1.record(stream)
        stream.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        e0.record(stream)
        sol.fvm_step_adjoint(st, 2, dt, lam, lam_out)
        e1.record(stream)
        stream.synchronize()
        adj_ms = e0.elapsed_time(e1)
        sol.close()
    line = {"metric": "melt-pool surrogate 512x512x256: step time by multigrid depth, adjoint "
                      "step beside it", "unit": "ms", "higher_is_better": False,
            "data": "synthetic", "config": {"workload": "melt-pool surrogate 512x512x256",
                                            "grid": list(shape)},
            "sweep": sweep,
            "adjoint": {"physics": "melt-pool geometry, density ratio 7900, the liquid's mu, "
                                   "lambda and rho c_p in both phases, FP64",
                        "dt": dt, "forward_step_ms": fwd_ms, "adjoint_step_ms": adj_ms,
                        "adjoint_over_forward": adj_ms / fwd_ms}}
    print(json.dumps(line), flush=True)


def run_droplet(args, rank, world, local_rank):
    """The migrating droplet (Table 1) at 100 x 100 in FP64 from rest for
    --droplet-steps steps (at most t = 0.12 s) with dt from the stability
    limits: steps, GPU time, the droplet's centroid displacement and
    migration speed, the largest velocity, the change of the phase volume
    and the mirror asymmetry.  100 = 4 * 25 leaves a 25 x 25 coarsest level
    to the one-CTA CG, which makes each step slow (tens of ms)."""
    import numpy as np
    import torch

    import cases
    import paper_2209_09671_gb300 as P
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p, s0 = cases.ma_bothe_droplet(n=100)
    if args.droplet_coarse_rtol:
        p = p.replace(coarse_rtol=args.droplet_coarse_rtol)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        solver = P.Solver(p, device=dev, stream=stream)
        st = P.to_device(s0, False, dev)
    _, y, _ = cases.cell_centres(p)
    yy = torch.tensor(np.broadcast_to(y, p.shape).copy(), device=dev)

    def centroid():
        return ((st["alpha"] * yy).sum() / st["alpha"].sum()).item()

    vol0 = st["alpha"].sum().item()
    y0 = centroid()
    t, n, hist = 0.0, 0, []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    while t < 0.12 and n < args.droplet_steps:
        info = solver.fvm_step(st, n, 0.0, info=True)
        t += info["dt"]
        n += 1
        if n % 250 == 0:
            hist.append((t, centroid()))
    e1.record(stream)
    stream.synchronize()
    hist.append((t, centroid()))
    a = st["alpha"]
    u, v = st["u"], st["v"]
    t1, c1 = hist[-1]
    tm, cm = min(hist, key=lambda q: abs(q[0] - 0.9 * t1))
    line = {"metric": "migrating droplet (Sec. V-A) at 100x100, FP64",
            "unit": "s", "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Ma-Bothe droplet, Table 1 properties, 200 K/m, 100x100x1",
                       "coarse_rtol": p.coarse_rtol, "mg_rtol": p.mg_rtol},
            "steps": n, "t_end": t, "gpu_seconds": e0.elapsed_time(e1) / 1e3,
            "centroid_shift_m": c1 - y0, "centroid_shift_cells": (c1 - y0) / p.h,
            "migration_speed_end_m_per_s": (c1 - cm) / (t1 - tm) if t1 > tm else None,
            "max_speed_m_per_s": max(u.abs().max().item(), v.abs().max().item()),
            "volume_change_rel": abs(a.sum().item() - vol0) / vol0,
            "mirror_asymmetry_alpha": (a - a.flip(-1)).abs().max().item(),
            "centroid_history": hist}
    print(json.dumps(line), flush=True)


def make_workload(shape, precision, mg_levels=None):
    import cases
    p, s = cases.melt_pool(*shape, precision=precision)
    if mg_levels:
        p = p.replace(mg_levels=mg_levels)
    return p, s


def ranks_barrier():
    """Barrier over the ranks of the default process group (none: no-op)."""
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.barrier()


def max_over_ranks(x: float, device) -> float:
    """Max of x over the ranks of the default process group (x itself when
    there is none); device is where the reduction tensor lives (CUDA for
    NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(cells_per_rank: int, world: int, seconds: float) -> float:
    """Cell-updates per second of the whole job: every rank runs an
    independent replica of the same workload, and the job takes as long as
    its slowest rank (seconds = the max over ranks)."""
    return world * cells_per_rank / seconds


def mixed_vs_f64_errors(P, dev, stream, n=64):
    """Per-field relative L2 of one mixed step against one FP64 step from the
    same float-rounded state (the n^3 melt-pool recipe after four FP64 steps,
    both solved to 1e-10), with max |D u| dt of each; the FP64 GPU step
    equals the FP64 oracle to 1e-11 (parity tests), so it stands in for it."""
    import numpy as np
    import torch

    import cases
    p, s = cases.melt_pool(n, n, n, precision=cases.F64)
    with torch.cuda.stream(stream):
        sol = P.Solver(p, device=dev, stream=stream)
        st = P.to_device(s, False, dev)
        for q in range(4):
            sol.fvm_step(st, q, 0.0, info=False)
        s32 = {k: (v.clone() if k == "p" else v.float().double()) for k, v in st.items()}
        a = {k: v.clone() for k, v in s32.items()}
        inf64 = sol.fvm_step(a, 4, 0.0, info=True)
        sol.close()
        solm = P.Solver(p.replace(precision=cases.MIXED), device=dev, stream=stream)
        b = {k: (v.clone() if k == "p" else v.float()) for k, v in s32.items()}
        infm = solm.fvm_step(b, 4, 0.0, info=True)
        solm.close()
    stream.synchronize()
    errs = {}
    for k in ("u", "v", "w", "p", "T", "alpha"):
        ref = a[k]
        nr = ref.norm().item()
        errs[k] = (b[k].double() - ref).norm().item() / nr if nr > 0 else None
    return {"grid": [n, n, n], "rel_l2_mixed_vs_f64": errs,
            "max_div_dt": {"mixed": infm["max_div_dt"], "f64": inf64["max_div_dt"]},
            "rel_residual": {"mixed": infm["rel_residual"], "f64": inf64["rel_residual"]},
            "reference": "the FP64 GPU step (equal to the FP64 oracle to 1e-11 in the parity "
                         "tests) from the same float-rounded state"}


def channel_side(P, dev, stream, steps):
    """The two-layer thermocapillary channel at 128 x 128 x 64: FP64 and mixed
    steps from its conduction state, cell-updates per second of each."""
    import torch

    import cases
    out = {"grid": [128, 128, 64], "steps": steps}
    for name, prec in (("mixed", cases.MIXED), ("f64", cases.F64)):
        p, s = cases.thermocapillary_channel()
        p = p.replace(precision=prec)
        with torch.cuda.stream(stream):
            sol = P.Solver(p, device=dev, stream=stream)
            st = P.to_device(s, prec == cases.MIXED, dev)
            for q in range(3):
                sol.fvm_step(st, q, 0.0, info=False)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for q in range(steps):
                sol.fvm_step(st, 3 + q, 0.0, info=False)
            e1.record(stream)
            stream.synchronize()
            t = e0.elapsed_time(e1) / 1e3 / steps
            info = sol.fvm_step(st, 3 + steps, 0.0, info=True)
            sol.close()
        out[name] = {"value": p.ncells / t, "ms_per_step": t * 1e3,
                     "vcycles_last_step": info["vcycles"], "max_div_dt": info["max_div_dt"],
                     "rel_residual": info["rel_residual"]}
    return out


def run_ours(args, rank, world, local_rank):
    import torch

    import cases
    import paper_2209_09671_gb300 as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    shape = tuple(args.shape) if args.shape else (args.n,) * 3
    N = shape[0] * shape[1] * shape[2]
    grid_name = "x".join(str(v) for v in shape) if len(set(shape)) > 1 else f"{shape[0]}^3"

    def barrier():
        ranks_barrier()

    stream = torch.cuda.Stream(device=dev)
    # measured arithmetic peaks of this GPU (kernels bound by the FMA pipes)
    fma64 = P.fvm.fvm_fma_peak(P.F64, stream)
    fma32 = P.fvm.fvm_fma_peak(P.MIXED, stream)

    # ---------------- mixed-precision step (the headline) -------------------
    p, s0 = make_workload(shape, cases.MIXED, args.mg_levels)
    if args.mx_inner:
        p = p.replace(mx_inner_cycles=args.mx_inner)
    if args.mg_pre is not None:
        p = p.replace(mg_pre=args.mg_pre)
    if args.mg_post is not None:
        p = p.replace(mg_post=args.mg_post)
    if args.mg_coarse is not None:
        p = p.replace(mg_coarse_sweeps=args.mg_coarse)
    with torch.cuda.stream(stream):
        solver = P.Solver(p, device=dev, stream=stream)
        state = P.to_device(s0, True, dev)
    step_idx = 0
    for _ in range(args.warmup):
        solver.fvm_step(state, step_idx, 0.0, info=False)
        step_idx += 1
    stream.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    solver.fvm_launch_count(reset=True)
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        solver.fvm_step(state, step_idx, 0.0, info=False)
        step_idx += 1
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = solver.fvm_launch_count()
    clk = clocks.stop()
    max_dT = (state["T"].double() - p.T0).abs().max().item()
    # per-kernel durations: the same workload continued for as many steps,
    # every launch bracketed by CUDA events on the solver's stream (eager
    # launches: event timing replaces the graph replay of the refinement loop)
    solver.fvm_profile(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        solver.fvm_step(state, step_idx, 0.0, info=False)
        step_idx += 1
    p1.record(stream)
    stream.synchronize()
    prof_elapsed = p0.elapsed_time(p1) / 1e3
    prof = solver.fvm_profile_read()
    solver.fvm_profile(False)
    info = solver.fvm_step(state, step_idx, 0.0, info=True)   # untimed: state sanity
    step_idx += 1
    t_step = max_over_ranks(elapsed / args.steps, dev)
    value = whole_job_rate(N, world, t_step)

    # dominant kernel and its roofline
    peak, peak_kind = load_peaks()

    def roofline_of(cls, nl, ms):
        per_launch_s = ms / 1e3 / nl
        common = {"kernel": cls, "launches": nl, "mean_launch_us": per_launch_s * 1e6,
                  "share_of_profiled_steps": ms / 1e3 / prof_elapsed,
                  "timing": "CUDA events around every launch of the class over "
                            f"{args.steps} profiled steps of the same workload"}
        if cls in FP64_FLOPS_PER_CELL:
            flops = FP64_FLOPS_PER_CELL[cls] * N
            achieved = flops / per_launch_s / 1e12
            return dict(bound="alu", achieved=achieved, peak=fma64["tflops"],
                        peak_kind="measured FP64 FMA throughput of this GPU (fvm_fma_peak)",
                        unit="TFLOP/s", frac=achieved / fma64["tflops"],
                        traffic=traffic_for(cls, True, N), alg_flops_per_launch=flops, **common)
        bpc = alg_bytes_per_cell(cls, True)
        if bpc is None:
            return None
        cpc = compulsory_bytes_per_cell(cls, True)
        achieved = bpc * N / per_launch_s / 1e9
        traffic = traffic_for(cls, True, N)
        return dict(bound="hbm", achieved=achieved, peak=peak,
                    peak_kind=f"{peak_kind} copy bandwidth", unit="GB/s", frac=achieved / peak,
                    traffic=traffic, alg_bytes_per_launch=bpc * N,
                    compulsory_bytes_per_launch=cpc * N,
                    frac_at_compulsory_bytes=cpc * N / per_launch_s / 1e9 / peak,
                    traffic_alg_ratio=(traffic / (bpc * N)) if traffic else None, **common)

    ranked = sorted(((k, v) for k, v in prof.items() if v[0]), key=lambda kv: -kv[1][1])
    roof = roofline_of(ranked[0][0], *ranked[0][1]) if ranked else None
    hbm_top = None
    for k, v in ranked:
        if alg_bytes_per_cell(k, True) is not None and k not in FP64_FLOPS_PER_CELL:
            hbm_top = roofline_of(k, *v)
            break
    # the FP64-bound defect-correction residual against the measured FP64 FMA rate
    fp64_res = roofline_of("residual64", *prof["residual64"]) if prof.get("residual64", (0,))[0] else None
    kernels = {k: {"launches": v[0], "ms": round(v[1], 3),
                   "share": round(v[1] / 1e3 / prof_elapsed, 4)} for k, v in prof.items() if v[0]}
    n_outer = sum(info["vcycles"]) / 3.0
    nbar_v = n_outer * p.mx_inner_cycles
    b_step = whole_step_alg_bytes(True, nbar_v, n_outer)
    whole = {"alg_bytes_per_cell": b_step, "nbar_v": nbar_v, "n_outer": n_outer,
             "achieved": b_step * N / t_step / 1e9, "peak": peak, "unit": "GB/s",
             "frac": b_step * N / t_step / 1e9 / peak,
             "formula": "3 (120 + 100 nbar_v + 40 n_outer) bytes per cell and step, nbar_v and "
                        "n_outer from the last step's refinement counts"}

    # ---------------- end to end through host buffers -------------------------
    e2e = None
    if not args.no_e2e:
        host = {k: v.to("cpu").pin_memory() for k, v in state.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = h2d
        # the fields' copies cut into chunks spread over several copy streams, so
        # that several copy engines run at once; the solver's stream waits for all
        # of them before the step and they wait for the step before reading back
        n_cs = args.copy_streams
        cstreams = [torch.cuda.Stream(device=dev) for _ in range(n_cs)]
        chunks = []
        for k in state:
            dflat, hflat = state[k].view(-1), host[k].view(-1)
            step_c = -(-dflat.numel() // args.copy_chunks)
            for a in range(0, dflat.numel(), step_c):
                chunks.append((dflat[a:a + step_c], hflat[a:a + step_c]))

        def copies(to_device):
            for cs in cstreams:
                cs.wait_stream(stream)
            for q, (dv, hv) in enumerate(chunks):
                with torch.cuda.stream(cstreams[q % n_cs]):
                    if to_device:
                        dv.copy_(hv, non_blocking=True)
                    else:
                        hv.copy_(dv, non_blocking=True)
            for cs in cstreams:
                stream.wait_stream(cs)

        with torch.cuda.stream(stream):
            for _ in range(2):
                copies(True)
                solver.fvm_step(state, step_idx, 0.0, info=False)
                copies(False)
                step_idx += 1
        stream.synchronize()
        e2e_steps = max(3, args.steps // 2)
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(e2e_steps):
                copies(True)
                solver.fvm_step(state, step_idx, 0.0, info=False)
                copies(False)
                step_idx += 1
        e1.record(stream)
        stream.synchronize()
        barrier()
        e2e_t = max_over_ranks(e0.elapsed_time(e1) / 1e3 / e2e_steps, dev)
        e2e = {"value": whole_job_rate(N, world, e2e_t), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    solver.close()
    del state, solver
    torch.cuda.empty_cache()

    # ---------------- FP64 step (side measurement, same workload) ----------
    f64 = None
    if args.f64_steps > 0:
        p64, s64 = make_workload(shape, cases.F64, args.mg_levels)
        with torch.cuda.stream(stream):
            sol64 = P.Solver(p64, device=dev, stream=stream)
            st64 = P.to_device(s64, False, dev)
        sol64.fvm_step(st64, 0, 0.0, info=False)
        stream.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for q in range(args.f64_steps):
            sol64.fvm_step(st64, 1 + q, 0.0, info=False)
        a1.record(stream)
        stream.synchronize()
        t64 = max_over_ranks(a0.elapsed_time(a1) / 1e3 / args.f64_steps, dev)
        sol64.fvm_profile(True)
        sol64.fvm_step(st64, 1 + args.f64_steps, 0.0, info=False)
        prof64 = sol64.fvm_profile_read()
        sol64.fvm_profile(False)
        inf64 = sol64.fvm_step(st64, 2 + args.f64_steps, 0.0, info=True)
        nv64 = sum(inf64["vcycles"]) / 3.0
        b64 = whole_step_alg_bytes(False, nv64, 0)
        f64 = {"value": whole_job_rate(N, world, t64), "ms_per_step": t64 * 1e3,
               "steps": args.f64_steps, "vcycles_last_step": inf64["vcycles"],
               "max_div_dt": inf64["max_div_dt"], "rel_residual": inf64["rel_residual"],
               "kernels_ms_one_step": {k: round(v[1], 2) for k, v in prof64.items() if v[0]},
               "whole_step": {"alg_bytes_per_cell": b64, "nbar_v": nv64,
                              "frac": b64 * N / t64 / 1e9 / peak},
               "bound": "FP64 FMA pipe"}
        sol64.close()
        del st64, sol64
        torch.cuda.empty_cache()

    accuracy = None if args.no_accuracy else mixed_vs_f64_errors(P, dev, stream)
    channel = None if args.channel_steps <= 0 else channel_side(P, dev, stream, args.channel_steps)

    if rank != 0:
        return
    cpu = None if args.no_cpu else cpu_baselines()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 transport + f64 projection",
        "data": "synthetic",
        "config": {"workload": f"melt-pool surrogate {grid_name} (rho 7900/1, mixed precision)",
                   "grid": list(shape), "precision": "mixed", "mg_rtol": p.mg_rtol,
                   "mg_levels": p.mg_levels,
                   "mx_inner_cycles": p.mx_inner_cycles, "mg_pre": p.mg_pre,
                   "mg_post": p.mg_post, "mg_coarse_sweeps": p.mg_coarse_sweeps,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": f"inputs larger than L2 (state {N * 28 / 2**20:.0f} MiB)"},
        "roofline": roof,
        "roofline_top_hbm_kernel": hbm_top,
        "roofline_residual64": fp64_res,
        "roofline_whole_step": whole,
        "fma_peaks_tflops": {"f64": fma64["tflops"], "f32": fma32["tflops"],
                             "how": "fvm_fma_peak: 8 independent FMA chains per thread, "
                                    "8 x 256 threads per SM, best of 3 launches"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "f64": f64,
        "accuracy_64cubed": accuracy,
        "channel_128x128x64": channel,
        "max_abs_T_minus_T0_after_timed_steps_K": max_dT,
        "last_step_info": info,
        "kernels": kernels,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.adjoint:
        run_adjoint(args, rank, world, local_rank)
        return
    if args.droplet:
        run_droplet(args, rank, world, local_rank)
        return
    if args.c5:
        run_c5(args, rank, world, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
