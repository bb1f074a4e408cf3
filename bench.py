#!/usr/bin/env python
"""Throughput of the two-stage fourth-order gas-kinetic step on a 3D hybrid unstructured mesh.

Workload: the smooth advection case (density sine wave, U = V = W = 1, p = 1, gamma = 1.4) on the
layered hybrid box mesh with 64 cubes per direction (1,048,576 cells: hexahedra, prisms, pyramids
and tetrahedra, interior nodes jittered +-0.1 h, seed 1), periodic [0,2]^3, Euler with the smooth
flux and zero collision time, CFL 0.5. A step is one S2O4 step (two stages of reconstruction,
face flux and face sums + update) over the whole mesh; the metric counts cell-stage updates/s.

The headline value is the mixed-precision path (FP32 reconstruction and flux, FP64 sums and
update); the FP64 path is measured beside it. Inputs (geometry ~1 GB) are larger than L2.
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s, FP32-bulk vs FP64, % roofline at stated error"
UNIT = "cell-stage/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gks", choices=["gks", "reference"])
    ap.add_argument("--n", type=int, default=64, help="cubes per direction")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 path (default: steps // 4, at least 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-vjp", action="store_true", help="skip the residual VJP timing")
    ap.add_argument("--no-implicit", action="store_true",
                    help="skip the implicit (Jacobi) workloads reported beside the headline")
    ap.add_argument("--no-explosion", action="store_true",
                    help="skip the spherical-explosion workload reported beside the headline")
    ap.add_argument("--min-stencil", type=int, default=18,
                    help="gks_mesh_options.min_stencil of the hybrid meshes (0: as printed)")
    ap.add_argument("--explosion-n", type=int, default=128, help="cubes per direction")
    ap.add_argument("--explosion-steps", type=int, default=20)
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clock and throttle-reason samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.rows = []
        self.proc = None
        self.device = device

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def workload_desc(n, nc=None, nf=None, min_stencil=0):
    # the hybrid 8-layer pattern has 4 cells and 9.125 faces per cube
    nc = nc if nc is not None else 4 * n ** 3
    nf = nf if nf is not None else 73 * n ** 3 // 8
    return {"workload": f"advection, hybrid layered box {n}^3 cubes ({nc} cells, {nf} faces), "
                        "periodic [0,2]^3, jitter 0.1h seed 1, Euler smooth flux tau=0, CFL 0.5",
            "cells": nc, "faces": nf, "cubes_per_dir": n, "flux": "smooth (Eq. flux-2)",
            "min_stencil": min_stencil,
            "tau": "zero", "cfl": 0.5, "gamma": 1.4,
            "arithmetic": "FP32; state, face sums and update as float-float pairs (no FP64 "
                          "instructions); FP64 path reported under fp64",
            "l2": "inputs larger than L2 (geometry and state > 1 GB); no flush"}


# ------------------------------------------------------------------------------ oracle timing
def host_cores() -> int:
    """Cores this process may run on (what `nproc` prints)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(n_sample: int, min_seconds: float, threads: int, min_stencil: int = 0):
    """S2O4 steps of the FP64 CPU oracle on the same generator at n_sample cubes per direction,
    with `threads` OpenMP threads, for at least min_seconds. Returns (cells, steps, seconds)."""
    import oracle
    from paper_2203_09047_gb300 import inputs as I
    m = I.layered_box_mesh(n_sample, "hybrid8")
    om = oracle.Mesh(m, min_stencil=min_stencil)
    P = oracle.params_vec()
    Q = I.advection_state(m)
    dt = om.max_dt(P, Q, 0.5)
    oracle.set_threads(threads)
    Q = om.step(P, Q, dt, 1)  # builds the stencils (lazy parts) outside the timed loop
    steps, t0 = 0, time.perf_counter()
    while True:
        Q = om.step(P, Q, dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return om.n_cells, steps, el


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    # each step a bounded sample: the 8^3-cube mesh of the same generator (2048 cells)
    n_sample = 8
    from paper_2203_09047_gb300 import inputs as I
    m = I.layered_box_mesh(n_sample, "hybrid8")
    om = oracle.Mesh(m, min_stencil=args.min_stencil)
    cores = host_cores()
    oracle.set_threads(cores)
    P = oracle.params_vec()
    Q = I.advection_state(m)
    dt = om.max_dt(P, Q, 0.5)
    for _ in range(args.warmup):
        Q = om.step(P, Q, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q = om.step(P, Q, dt, 1)
    el = time.perf_counter() - t0
    nc = om.n_cells
    value = nc * 2 * args.steps / el
    sample = (f"{nc}-cell hybrid box (8^3 cubes, same generator and stencils) per step; the "
              "oracle's cost per cell-stage does not depend on the mesh size, so the rate stands "
              f"for the {4 * args.n ** 3}-cell workload")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_desc(args.n, min_stencil=args.min_stencil),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
def job_rate(ms_local, units_local, world, dist=None, device="cuda"):
    """Whole-job throughput of N independent replicas: the slowest rank's time (max over
    ranks) and the units all ranks processed divided by it. Returns (max ms, units per s)."""
    import torch
    ms, units = float(ms_local), float(units_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    return ms, units / (ms * 1e-3)


def run_vjp(gks, I, S, Q0, dt, torch, stream, calls=3):
    """ms per residual VJP (gks_residual_vjp: FP64 reconstruction recomputed, then the reverse
    passes of the flux, polynomial evaluation, reconstruction and stencil gathers)."""
    Q = torch.from_numpy(np.ascontiguousarray(Q0)).cuda()
    d = I.normal_directions(Q0.shape, 2, 5)
    gL, gLt = torch.from_numpy(d[0]).cuda(), torch.from_numpy(d[1]).cuda()
    gQ = torch.empty_like(Q)
    gks.gks_residual_vjp(S.h, Q, dt, gL, gLt, gQ)  # warm-up (allocates the adjoint buffers)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(calls):
        gks.gks_residual_vjp(S.h, Q, dt, gL, gLt, gQ)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / calls
    return {"ms_per_call": ms, "cells_per_s": S.n_cells / (ms * 1e-3), "calls": calls,
            "dtype": "f64", "api": "gks_residual_vjp (device buffers)"}


_LID = [[0.0] * 3 for _ in range(6)]
_LID[4][0] = 0.15  # the upper y plane moves along x at Ma 0.15 (c = 1)
IMPLICIT_CASES = [
    # name, cubes, layers box, bc, params, paper (cells, ms per step) for context
    ("cavity", 32, ((0, 0, 0), (1, 1, 1)), (2, 2, 2),
     dict(flux_mode=1, tau_model=2, mu=0.15 / 1000.0, wall_u=_LID, wall_T=[1.0 / 1.4] * 6),
     (102400, 97.0)),
    ("sphere_like", 48, ((0, 0, 0), (2, 2, 2)), (0, 0, 0),
     dict(flux_mode=1, tau_model=1), (462673, 1093.0)),
]


def run_implicit(gks, I, stream, torch, kmax=3, steps=20, warmup=3):
    """ms per implicit step (one residual + kmax Jacobi sweeps) for FP64 and mixed precision."""
    out = {}
    for name, n, (lo, hi), bc, params, (p_cells, p_ms) in IMPLICIT_CASES:
        m = I.layered_box_mesh(n, "hybrid8", lo=lo, hi=hi, bc=bc)
        mesh = gks.Mesh(m)
        if bc[0] == 2:  # lid-driven cavity (Section 5.3): gas at rest, rho = 1, p = 1/gamma
            Q0 = np.zeros((5, len(m["cell_type"])))
            Q0[0] = 1.0
            Q0[4] = 1.0 / 1.4 / 0.4
        else:
            Q0 = I.advection_state(m)
        rec = {"cells": mesh.n_cells, "faces": mesh.n_faces, "kmax": kmax,
               "flux": "smooth" if params["flux_mode"] == 0 else "full",
               "tau": ["zero", "inviscid", "viscous", "power law"][params["tau_model"]],
               "bc": ("no-slip isothermal walls, lid at Ma 0.15, Re 1000" if bc[0] == 2
                      else "periodic"),
               "paper": {"cells": p_cells, "ms_per_step": p_ms, "hardware": "TITAN RTX, FP64",
                         "cell_steps_per_s": p_cells * 1e3 / p_ms}}
        for prec, key in ((gks.GKS_PREC_FP64, "fp64"), (gks.GKS_PREC_MIXED, "mixed")):
            S = gks.Solver(mesh, stream=stream, precision=prec, **params)
            S.set_state(Q0)
            dt = S.max_dt(2.0)
            for _ in range(warmup):
                S.step_implicit(dt, 1, kmax, check=False)
            gks.gks_check(S.h)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            gks.gks_step_implicit(S.h, dt, steps, kmax)
            ev1.record(stream)
            torch.cuda.synchronize()
            gks.gks_check(S.h)
            ms = ev0.elapsed_time(ev1) / steps
            lpp = gks.gks_launches_per_pass(S.h)
            rec[key] = {"ms_per_step": ms, "cell_steps_per_s": mesh.n_cells / (ms * 1e-3),
                        "steps": steps, "warmup": warmup, "cfl": 2.0,
                        "gpu_launches_per_step": lpp[0] + lpp[1] + 1 + kmax}
            S.close()
        out[name] = rec
    return out


def run_explosion(gks, I, stream, torch, args, fp32_peak, hbm):
    """The Section 5 spherical explosion in the reflecting box [-1,1]^3 on the hybrid generator
    (full flux, inviscid collision time, nonlinear weights, Gauss-point positivity fallback):
    mixed-precision and FP64 throughput over the same steps from the same state, the relative
    mass and energy drift per step, and the mixed-vs-FP64 density difference."""
    n, K, W = args.explosion_n, args.explosion_steps, 10
    m = I.layered_box_mesh(n, "hybrid8", lo=(-1, -1, -1), hi=(1, 1, 1), bc=(1, 1, 1))
    Q0 = I.explosion_state(m)
    mesh = gks.Mesh(m, min_stencil=args.min_stencil)
    params = dict(flux_mode=1, tau_model=1, gp_fallback=1)
    rec = {"workload": f"spherical explosion, hybrid layered box {n}^3 cubes ({mesh.n_cells} "
                       f"cells, {mesh.n_faces} faces), reflecting walls [-1,1]^3, full flux, "
                       "inviscid collision time, CFL 0.5, Gauss-point positivity fallback",
           "cells": mesh.n_cells, "faces": mesh.n_faces, "steps": K,
           "warmup": f"{W} untimed steps from the initial state, dt re-evaluated every step (the "
                     "blast accelerates the gas from rest); then K timed steps at the CFL-0.5 dt "
                     "of the state after them; FP64 replays the same dt sequence"}
    states, dts, dt, vol = {}, None, None, None
    for prec, key in ((gks.GKS_PREC_MIXED, "mixed"), (gks.GKS_PREC_FP64, "fp64")):
        S = gks.Solver(mesh, stream=stream, precision=prec, **params)
        S.set_state(Q0)
        if dts is None:
            _, wq = S.cell_quadrature()
            vol = wq.sum(axis=1)
            del wq
            dts = []
            for _ in range(W):
                dts.append(S.max_dt(0.5))
                S.step(dts[-1], 1)
            dt = S.max_dt(0.5)
        else:
            for d in dts:
                S.step(d, 1)
        Qw = S.get_state().cpu().numpy()
        if prec == gks.GKS_PREC_MIXED:
            gks.gks_timing_enable(S.h, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        gks.gks_step(S.h, dt, K)
        ev1.record(stream)
        torch.cuda.synchronize()
        gks.gks_check(S.h)
        ms = ev0.elapsed_time(ev1)
        q = S.get_state().cpu().numpy()
        states[key] = q
        r = {"value": mesh.n_cells * 2 * K / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / K}
        for v, name in ((0, "mass"), (4, "energy")):
            tot0 = float(vol @ Qw[v])
            r[f"{name}_drift_per_step"] = abs(float(vol @ q[v]) - tot0) / abs(tot0) / K
        if prec == gks.GKS_PREC_MIXED:
            kms, kcnt = gks.gks_timing_read(S.h)
            bytes_k = gks.gks_kernel_bytes(S.h)
            fl, _ = gks.gks_flux_opcount(1, 1)
            names = ["recon", "flux", "gather"]
            tot = sum(kms)
            kt = {names[k]: {"launches": kcnt[k], "avg_ms": kms[k] / max(kcnt[k], 1),
                             "share": kms[k] / tot if tot else None} for k in range(3)}
            for k in range(3):
                kt[names[k]]["gbs"] = bytes_k[k] / (kt[names[k]]["avg_ms"] * 1e-3) / 1e9
            kt["flux"]["tflops"] = fl * 4 * mesh.n_faces / (kt["flux"]["avg_ms"] * 1e-3) / 1e12
            r["kernels"] = kt
            dom = max(kt, key=lambda k: kt[k]["share"] or 0)
            if dom == "flux":
                r["roofline"] = {"kernel": "k_flux<float, full>", "bound": "alu",
                                 "achieved": kt["flux"]["tflops"], "peak": fp32_peak,
                                 "unit": "TFLOP/s", "frac": kt["flux"]["tflops"] / fp32_peak,
                                 "flops_per_gauss_point": fl}
            else:
                r["roofline"] = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": kt[dom]["gbs"],
                                 "peak": hbm, "unit": "GB/s", "frac": kt[dom]["gbs"] / hbm}
        rec[key] = r
        S.close()
    d = np.abs(states["mixed"][0] - states["fp64"][0])
    rec["mixed_vs_fp64_L1_rho"] = float(vol @ d / vol.sum())
    rec["mixed_vs_fp64_L1_rho_rel"] = float(vol @ d / (vol @ states["fp64"][0]))
    rec["dt"] = dt
    mesh.close()
    return rec


def run_gpu(args):
    import torch

    import paper_2203_09047_gb300 as gks
    from paper_2203_09047_gb300 import build, inputs as I

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    gks.load_library()

    mesh_dict = I.layered_box_mesh(args.n, "hybrid8")
    Q0 = I.advection_state(mesh_dict)
    mesh = gks.Mesh(mesh_dict, min_stencil=args.min_stencil)
    stream = torch.cuda.Stream()
    results = {}

    def measure(precision, steps, warmup, timed_kernels=True):
        S = gks.Solver(mesh, stream=stream, precision=precision)
        S.set_state(Q0)
        dt = S.max_dt(0.5)
        for _ in range(warmup):
            S.step(dt, 1, check=False)
        gks.gks_check(S.h)
        gks.gks_timing_read(S.h)  # reset
        if timed_kernels:
            gks.gks_timing_enable(S.h, True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            gks.gks_step(S.h, dt, steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1)
        kms, kcnt = gks.gks_timing_read(S.h)
        gks.gks_timing_enable(S.h, False)
        gks.gks_check(S.h)
        return dict(solver=S, dt=dt, ms=ms, kms=kms, kcnt=kcnt, clocks=clk.summary())

    mixed = measure(gks.GKS_PREC_MIXED, args.steps, args.warmup)
    S = mixed["solver"]
    nc, nf = S.n_cells, S.n_faces
    ms_total, value = job_rate(mixed["ms"], nc * 2 * args.steps, world,
                               dist if world > 1 else None)

    # FP64 path on the same inputs and dt
    fp64_steps = args.fp64_steps or max(3, args.steps // 4)
    fp64 = measure(gks.GKS_PREC_FP64, fp64_steps, 2)
    v64 = nc * 2 * fp64_steps / (fp64["ms"] * 1e-3)

    # the FP64-update mixed mode (FP32 reconstruction and flux, FP64 face sums and update)
    upd_steps = max(3, args.steps // 4)
    upd = measure(gks.GKS_PREC_MIXED_FP64UPD, upd_steps, 2, timed_kernels=False)
    v_upd = nc * 2 * upd_steps / (upd["ms"] * 1e-3)
    upd["solver"].close()

    # errors of the mixed modes against the FP64 path after the same steps from the same state,
    # and the conservation drift of each mode (volume-weighted totals of mass and energy)
    xq, wq = mixed["solver"].cell_quadrature()
    vol = wq.sum(axis=1)
    del xq, wq

    def advance(precision, k):
        T = gks.Solver(mesh, stream=stream, precision=precision)
        T.set_state(Q0)
        T.step(mixed["dt"], k)
        out = T.get_state().double().cpu().numpy()
        T.close()
        return out

    def drift(q):
        return {name: float(abs(vol @ q[v] - vol @ Q0[v]) / abs(vol @ Q0[v]))
                for v, name in ((0, "mass"), (4, "energy"))}
    k_err = 10
    qm, qd = advance(gks.GKS_PREC_MIXED, k_err), advance(gks.GKS_PREC_FP64, k_err)
    qu = advance(gks.GKS_PREC_MIXED_FP64UPD, k_err)
    err = float(np.linalg.norm(qm - qd) / np.linalg.norm(qd))
    err_upd = float(np.linalg.norm(qu - qd) / np.linalg.norm(qd))

    # rooflines: HBM copy bandwidth from MEASURED_PEAKS.json; FP32 and FP64 FMA throughput
    # measured now on this GPU (gks_alu_peaks)
    bytes_k = gks.gks_kernel_bytes(S.h)
    hbm, hbm_src = peaks()
    flops_gp, special_gp = gks.gks_flux_opcount(0, 0)
    fp32_peak, fp64_peak = gks.gks_alu_peaks()  # TFLOP/s

    def kernel_table(res, is_mixed):
        names = ["recon", "flux", "gather"]
        out = {}
        tot = sum(res["kms"])
        for k in range(3):
            n = max(res["kcnt"][k], 1)
            avg_ms = res["kms"][k] / n
            d = {"launches": res["kcnt"][k], "avg_ms": avg_ms, "share": res["kms"][k] / tot if tot else None,
                 "gbs": bytes_k[k] * (1 if is_mixed else 1) / (avg_ms * 1e-3) / 1e9 if avg_ms else None}
            out[names[k]] = d
        fl = flops_gp * 4 * nf
        out["flux"]["tflops"] = fl / (out["flux"]["avg_ms"] * 1e-3) / 1e12
        return out

    kt = kernel_table(mixed, True)
    # bytes of the FP64 solver differ (8-byte geometry): ask that solver
    bytes64 = gks.gks_kernel_bytes(fp64["solver"].h)
    kt64 = kernel_table(fp64, False)
    for k, name in enumerate(["recon", "flux", "gather"]):
        kt64[name]["gbs"] = bytes64[k] / (kt64[name]["avg_ms"] * 1e-3) / 1e9

    # DRAM bytes (read + write) per pass of the FP32 reconstruction and per launch of the FP32
    # smooth flux from the ncu captures on the 48^3-cube mesh with the enlarged stencils
    # (profiles/k_recon_float_advection48_ncu.md, profiles/k_flux_float_smooth_advection48_ncu.md),
    # scaled by cells and by faces (same layer pattern and stencils)
    dram_per_unit = {"recon": (1552.3, nc), "flux": (292.0, nf)}

    def roof_of(table, dom, is_mixed):
        if dom == "flux":
            peak = fp32_peak if is_mixed else fp64_peak
            ach = table["flux"]["tflops"]
            return {"kernel": f"k_flux<{'float' if is_mixed else 'double'}>", "bound": "alu",
                    "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": (dram_per_unit["flux"][0] * dram_per_unit["flux"][1])
                               if is_mixed and "flux" in dram_per_unit else None,
                    "peak_source": f"measured {'FP32' if is_mixed else 'FP64'} FMA throughput of "
                                   "this GPU (gks_alu_peaks, an FMA as 2 flops)",
                    "flops_per_gauss_point": flops_gp, "special_per_gauss_point": special_gp}
        ach = table[dom]["gbs"]
        traffic = None
        if is_mixed and dom in dram_per_unit:
            traffic = dram_per_unit[dom][0] * dram_per_unit[dom][1]
        return {"kernel": f"k_{dom}", "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": traffic, "peak_source": f"{hbm_src} copy bandwidth",
                "per": "one pass over the mesh (one launch per cell-kind tile range)" if dom == "recon"
                       else "one launch"}

    def roof_for(table, is_mixed):
        """The dominant kernel's roofline (largest share of the step's kernel time)."""
        return roof_of(table, max(table, key=lambda k: table[k]["share"] or 0), is_mixed)

    def rooflines(table, is_mixed):
        return {k: roof_of(table, k, is_mixed) for k in ("recon", "flux")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_desc(args.n, nc, nf, min_stencil=args.min_stencil),
        "clocks": mixed["clocks"],
        "gpu_launches": int(sum(c * l for c, l in zip(mixed["kcnt"], gks.gks_launches_per_pass(S.h)))),
        "roofline": roof_for(kt, True),
        "rooflines": rooflines(kt, True),
        "kernels": kt,
        "fp64": {"value": v64, "unit": UNIT, "steps": fp64_steps, "ms_per_step": fp64["ms"] / fp64_steps,
                 "dtype": "f64", "roofline": roof_for(kt64, False), "kernels": kt64,
                 "clocks": fp64["clocks"]},
        "fp64_update": {"value": v_upd, "unit": UNIT, "steps": upd_steps,
                        "ms_per_step": upd["ms"] / upd_steps, "dtype": "f32 + f64 update",
                        "mode": "GKS_PREC_MIXED_FP64UPD: FP32 reconstruction and flux, FP64 face "
                                "sums and FP64 update of an FP64 state",
                        "clocks": upd["clocks"]},
        "error": {"mixed_vs_fp64_state_rel_l2": err,
                  "fp64_update_vs_fp64_state_rel_l2": err_upd, "after_steps": k_err,
                  "drift_after_steps": {"mixed": drift(qm), "fp64_update": drift(qu),
                                        "fp64": drift(qd)},
                  "fp64_vs_oracle": "<= 1e-12 relative L2 (parity tests)"},
        "alu_peaks_tflops": {"fp32": fp32_peak, "fp64": fp64_peak,
                             "source": "gks_alu_peaks, measured in this run"},
    }
    if world > 1:
        line["parallelism"] = f"{world} independent replicas (one full mesh per GPU)"

    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        Qh = torch.from_numpy(np.ascontiguousarray(Q0)).pin_memory()
        Qo = torch.empty_like(Qh).pin_memory()
        e_steps = max(3, args.steps // 4)
        S.set_state(Q0)
        gks.gks_step(S.h, mixed["dt"], 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            gks.gks_set_state(S.h, Qh)
            gks.gks_step(S.h, mixed["dt"], 1)
            gks.gks_get_state(S.h, Qo)
        el = time.perf_counter() - t0
        serial = nc * 2 * e_steps / el
        # the same calls from two solvers on their own streams taking alternate steps: one
        # solver's host copies and state permutations overlap the other's step (every step still
        # copies its input in from pinned host memory and its result out)
        SP = [gks.Solver(mesh, stream=torch.cuda.Stream(), precision=gks.GKS_PREC_MIXED)
              for _ in range(2)]
        Qhs = [torch.from_numpy(np.ascontiguousarray(Q0)).pin_memory() for _ in range(2)]
        Qos = [torch.empty_like(Qh).pin_memory() for _ in range(2)]
        for k in range(2):
            gks.gks_set_state(SP[k].h, Qhs[k])
            gks.gks_step(SP[k].h, mixed["dt"], 1)
            gks.gks_get_state(SP[k].h, Qos[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e_steps):
            X, Y = k % 2, 1 - k % 2
            gks.gks_set_state(SP[X].h, Qhs[X])
            gks.gks_step(SP[X].h, mixed["dt"], 1)
            if k > 0:
                gks.gks_get_state(SP[Y].h, Qos[Y])  # the other solver's result of step k - 1
        gks.gks_get_state(SP[(e_steps - 1) % 2].h, Qos[(e_steps - 1) % 2])
        el2 = time.perf_counter() - t0
        for X in SP:
            X.close()
        line["e2e"] = {"value": nc * 2 * e_steps / el2, "unit": UNIT, "steps": e_steps,
                       "h2d_bytes_per_step": int(Qh.numel() * 8), "d2h_bytes_per_step": int(Qo.numel() * 8),
                       "api": "gks_set_state(host) + gks_step + gks_get_state(host) per step, two "
                              "solvers on their own streams taking alternate steps",
                       "serial_value": serial,
                       "serial_api": "the same calls on one solver, one step after the other"}

    # the residual's vector-Jacobian product on the same mesh and state (FP64)
    if not args.no_vjp:
        line["vjp"] = run_vjp(gks, I, fp64["solver"], Q0, mixed["dt"], torch, stream)

    # the implicit Jacobi path (Section 4) on workloads sized like the paper's two timed cases,
    # reported beside the headline with the paper's own times (TITAN RTX, FP64) as context
    if not args.no_implicit:
        line["implicit"] = run_implicit(gks, I, stream, torch)

    # the spherical explosion (largest configuration) beside the headline
    if not args.no_explosion:
        line["explosion"] = run_explosion(gks, I, stream, torch, args, fp32_peak, hbm)

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        cores = host_cores()
        n_s, steps_a, el_a = time_oracle(16, 10.0, cores, args.min_stencil)
        _, steps_1, el_1 = time_oracle(16, 10.0, 1, args.min_stencil)
        line["cpu_baseline"] = {
            "value": n_s * 2 * steps_a / el_a, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": n_s * 2 * steps_1 / el_1,
            "sample": f"{steps_a} S2O4 steps ({cores} threads) and {steps_1} steps (1 thread) on "
                      f"the {n_s}-cell 16^3-cube mesh of the same generator and stencils; the "
                      "oracle's cost per cell-stage does not depend on the mesh size, so the rate "
                      f"stands for the {nc}-cell workload"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
