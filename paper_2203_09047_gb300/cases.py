"""Validation cases on the synthetic hybrid meshes, run through the public API on the GPU.

    python -m paper_2203_09047_gb300.cases advection   # convergence 8..64 cubes, FP64 and mixed
    python -m paper_2203_09047_gb300.cases tgv         # Taylor-Green vortex, Re 1600, Pr 0.72
    python -m paper_2203_09047_gb300.cases adjoint     # gradient through 200 S2O4 steps vs FD
    python -m paper_2203_09047_gb300.cases explosion   # spherical explosion, reflecting box
    python -m paper_2203_09047_gb300.cases sod         # Sod shock tube vs the exact solution
    python -m paper_2203_09047_gb300.cases implicit_steady   # implicit steps to a steady state

Each prints one JSON line per result.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import GKS_PREC_FP64, GKS_PREC_MIXED, Mesh, Solver, GksError
from . import inputs as I


def _emit(d):
    print(json.dumps(d), flush=True)


def _exact_advection(t, gamma=1.4):
    def field(x):
        rho, u, p = I.advection_primitive(x, t)
        return I.primitive_to_conserved(rho, u, p, gamma)
    return field


def advection(ns=(8, 16, 32, 64), t_end=0.2, cfl=0.5, layers="hybrid8", jitter=0.1,
              precisions=("fp64", "mixed"), min_stencil=0, **weno):
    """Section 5.1 accuracy test on the hybrid generator: errors against the exact cell averages
    (volume-weighted, unnormalised L1 and L2 of density as in Tables tab-3d-1/2), orders, and
    cell-stage updates/s, for the FP64 and mixed paths. jitter is the node displacement in units
    of h; weno passes WENO parameters (weno_eps = 1e30 gives the linear weights, i.e. P0)."""
    import torch
    out = []
    if isinstance(ns, int):
        ns = (ns,)
    if isinstance(precisions, str):
        precisions = tuple(precisions.split(","))
    for prec, name in ((GKS_PREC_FP64, "fp64"), (GKS_PREC_MIXED, "mixed")):
        if name not in precisions:
            continue
        prev = None
        for n in ns:
            m = I.layered_box_mesh(n, layers, jitter=jitter)
            try:
                S = Solver(m, precision=prec, min_stencil=min_stencil, **weno)
            except GksError as e:
                _emit({"case": "advection", "mesh": layers, "precision": name, "cubes": n,
                       "jitter": jitter, "min_stencil": min_stencil, **weno,
                       "status": f"init: {e}"})
                prev = None
                continue
            Q0 = S.cell_average(_exact_advection(0.0))
            S.set_state(Q0)
            dt = S.max_dt(cfl)
            nsteps = int(np.ceil(t_end / dt - 1e-12))
            dt = t_end / nsteps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            S.step(dt, nsteps, check=False)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            rec = {"case": "advection", "mesh": layers, "precision": name, "cubes": n,
                   "cells": S.n_cells, "jitter": jitter, "min_stencil": min_stencil, **weno,
                   "steps": nsteps, "dt": dt}
            try:
                S.check()
            except GksError as e:
                rec["status"] = f"stopped: {e}"
                _emit(rec)
                out.append(rec)
                prev = None
                S.close()
                continue
            Q = S.get_state().cpu().numpy()
            xq, wq = S.cell_quadrature()
            vol = wq.sum(axis=1)
            ex = S.cell_average(_exact_advection(t_end))
            e = Q[0] - ex[0]
            l1 = float((vol * np.abs(e)).sum())
            l2 = float(np.sqrt((vol * e * e).sum()))
            rec.update({"L1": l1, "L2": l2, "cell_stage_per_s": S.n_cells * 2 * nsteps / el})
            if prev is not None:
                rec["order_L1"] = float(np.log2(prev[0] / l1))
                rec["order_L2"] = float(np.log2(prev[1] / l2))
            prev = (l1, l2)
            _emit(rec)
            out.append(rec)
            S.close()
    return out


def tgv(n=48, steps=200, cfl=0.5, re=1600.0, mach=0.1, pr=0.72, min_stencil=18, t_end=None,
        fp64=True):
    """Taylor-Green vortex on the TGV layer pattern in [0, 2 pi]^3 (whose two transition layers
    take the enlarged stencils, min_stencil 18): kinetic energy and its dissipation rate, mixed
    path against the FP64 path. With t_end the run takes as many steps as that time needs at
    the CFL step (a resolution study at a fixed time). The record carries the viscous
    dissipation rate of the initial field, 3 mu / 4 (the mean of |curl U|^2 is 3/4, rho = 1),
    which the measured rate approaches as the mesh is refined."""
    import torch
    m = I.layered_box_mesh(n, "tgv48", lo=(0, 0, 0), hi=(2 * np.pi,) * 3, jitter=0.05)
    mesh = Mesh(m, min_stencil=min_stencil)
    params = dict(flux_mode=0, tau_model=2, mu=1.0 / re, Pr=pr)

    def field(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        u = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z),
                      np.zeros_like(X)], axis=-1)
        p = 1.0 / (1.4 * mach * mach) + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
        return I.primitive_to_conserved(np.ones_like(X), u, p)

    # cell averages of the initial field by the 27-point quadrature, volumes, the CFL step
    S = Solver(mesh, precision=GKS_PREC_FP64, **params)
    Q0 = S.cell_average(field)
    vol = torch.from_numpy(S.cell_quadrature()[1].sum(axis=1)).cuda()
    S.set_state(Q0)
    dt = S.max_dt(cfl)
    S.close()
    if t_end is not None:
        steps = max(1, int(np.ceil(t_end / dt)))
        dt = t_end / steps
    series = {}
    runs = ((GKS_PREC_FP64, "fp64"), (GKS_PREC_MIXED, "mixed")) if fp64 else ((GKS_PREC_MIXED, "mixed"),)
    for prec, name in runs:
        S = Solver(mesh, precision=prec, **params)
        S.set_state(Q0)
        ke = []
        t0 = time.perf_counter()
        for k in range(steps + 1):
            Q = S.get_state()
            ke.append(float(((0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]) * vol).sum() / vol.sum()))
            if k < steps:
                S.step(dt, 1, check=(k % 20 == 19))
        torch.cuda.synchronize()
        series[name] = (np.array(ke), time.perf_counter() - t0)
        S.close()
    rec = {"case": "tgv", "cubes": n, "cells": mesh.n_cells, "min_stencil": min_stencil,
           "steps": steps, "dt": dt, "t_end": steps * dt, "dissipation_viscous_t0": 0.75 / re}
    for name, (ke, wall) in series.items():
        eps = -np.gradient(ke, dt)
        rec.update({"ke0": ke[0], f"ke_end_{name}": ke[-1], f"dissipation_end_{name}": float(eps[-1]),
                    f"dissipation_mean_{name}": float((ke[0] - ke[-1]) / (steps * dt)),
                    f"wall_s_{name}": wall})
    if fp64:
        k64, km = series["fp64"][0], series["mixed"][0]
        eps64, epsm = -np.gradient(k64, dt), -np.gradient(km, dt)
        rec["ke_max_rel_diff"] = float(np.abs(km - k64).max() / k64[0])
        rec["dissipation_max_rel_diff"] = float(np.abs(epsm - eps64).max() / np.abs(eps64).max())
    _emit(rec)
    return rec


def adjoint(n=32, steps=200, every=20, ndirs=20, mu=1e-3, cfl=0.5, eps=1e-6, layers="hybrid8",
            min_stencil=18):
    """Gradient of J = sum |Omega| rho^2 at the final time with respect to the initial state,
    through `steps` S2O4 steps with checkpoints every `every`, against central differences on
    `ndirs` random directions (Navier-Stokes, full flux, viscous collision time), on the C4 mesh:
    the hybrid generator at 32 cubes with the enlarged stencils (min_stencil 18). With the
    stencils as printed (min_stencil 0) the transition layers' unstable reconstruction makes J
    non-smooth over 200 steps and central differences do not converge."""
    import torch
    from .autograd import s2o4_rollout
    m = I.layered_box_mesh(n, layers)
    S = Solver(m, flux_mode=1, tau_model=2, mu=mu, min_stencil=min_stencil)
    Qc = S.cell_average(_exact_advection(0.0))
    Q0 = I.perturbed_state(Qc, seed=2, amp=0.01)
    S.set_state(Q0)
    dt = S.max_dt(cfl)
    vol = torch.from_numpy(S.cell_quadrature()[1].sum(axis=1)).cuda()

    def J(Q):
        QT = s2o4_rollout(Q, S, dt, steps, checkpoint_every=every)
        return (vol * QT[0] ** 2).sum()

    Qt = torch.from_numpy(Q0).cuda().requires_grad_(True)
    t0 = time.perf_counter()
    J(Qt).backward()
    t_grad = time.perf_counter() - t0
    grad = Qt.grad.detach()
    dirs = I.normal_directions(Q0.shape, ndirs, 3)
    worst = 0.0
    with torch.no_grad():
        for d in dirs:
            dd = torch.from_numpy(d).cuda()
            fd = (J(Qt + eps * dd) - J(Qt - eps * dd)).item() / (2 * eps)
            ad = float((grad * dd).sum())
            worst = max(worst, abs(ad - fd) / abs(fd))
    rec = {"case": "adjoint", "mesh": layers, "min_stencil": min_stencil, "cubes": n,
           "cells": S.n_cells, "steps": steps, "checkpoint_every": every,
           "directions": ndirs, "fd_eps": eps, "max_rel_diff_vs_fd": worst, "gradient_wall_s": t_grad}
    _emit(rec)
    return rec


def exact_riemann(left, right, x, t, x0=0.5, gamma=1.4):
    """Exact solution (rho, u, p) at positions x and time t of the 1D Riemann problem with
    left/right primitive states (rho, u, p) separated at x0: star pressure from
    f_L(p) + f_R(p) + u_R - u_L = 0 (shock branch (p - p_K) sqrt(A_K / (p + B_K)), rarefaction
    branch 2 c_K / (gamma - 1) ((p / p_K)^((gamma - 1) / (2 gamma)) - 1)) by Newton's method,
    then the self-similar solution sampled at (x - x0)/t."""
    g = gamma
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)

    def fk(p, r, pk, ck):
        if p > pk:
            A, B = 2.0 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            sq = np.sqrt(A / (p + B))
            return (p - pk) * sq, sq * (1.0 - 0.5 * (p - pk) / (B + p))
        e = (g - 1) / (2 * g)
        return 2 * ck / (g - 1) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1) / (2 * g)) / (r * ck)

    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = fk(p, rL, pL, cL)
        fR, dR = fk(p, rR, pR, cR)
        dp = (fL + fR + uR - uL) / (dL + dR)
        p = max(1e-10, p - dp)
        if abs(dp) < 1e-15 * p:
            break
    fL, _ = fk(p, rL, pL, cL)
    fR, _ = fk(p, rR, pR, cR)
    us = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    g6 = (g - 1) / (g + 1)
    xi = (np.asarray(x) - x0) / t
    rho, u, pr = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    for j, s in enumerate(xi):
        if s <= us:  # left of the contact
            if p > pL:
                S = uL - cL * np.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                st = (rL, uL, pL) if s < S else (rL * (p / pL + g6) / (g6 * p / pL + 1), us, p)
            else:
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                if s < uL - cL:
                    st = (rL, uL, pL)
                elif s > us - cs:
                    st = (rL * (p / pL) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cL + 0.5 * (g - 1) * (uL - s))
                    st = (rL * (c / cL) ** (2 / (g - 1)), 2 / (g + 1) * (cL + 0.5 * (g - 1) * uL + s),
                          pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if p > pR:
                S = uR + cR * np.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                st = (rR, uR, pR) if s > S else (rR * (p / pR + g6) / (g6 * p / pR + 1), us, p)
            else:
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                if s > uR + cR:
                    st = (rR, uR, pR)
                elif s < us + cs:
                    st = (rR * (p / pR) ** (1 / g), us, p)
                else:
                    c = 2 / (g + 1) * (cR - 0.5 * (g - 1) * (uR - s))
                    st = (rR * (c / cR) ** (2 / (g - 1)), 2 / (g + 1) * (-cR + 0.5 * (g - 1) * uR + s),
                          pR * (c / cR) ** (2 * g / (g - 1)))
        rho[j], u[j], pr[j] = st
    return rho, u, pr, p, us


def sod(n=64, t_end=0.2, cfl=0.5, layers="hex", flux_mode=1, tau_model=1, jitter=0.0,
        **weno):
    """Sod's shock tube (Section 5, Riemann problems) along x in [0,1]^3 (reflecting walls at
    x = 0, 1, which the waves do not reach by t = 0.2; periodic in y, z): left (1, 0, 1), right
    (0.125, 0, 0.1) split at x = 0.5 by the cell's vertex mean; full flux, inviscid collision
    time. Default: uniform hexahedra as the paper's hexahedral run. Density L1 error per unit
    volume against the exact solution's cell averages (27-point quadrature), FP64 and mixed."""
    import torch
    m = I.layered_box_mesh(n, layers, lo=(0, 0, 0), hi=(1, 1, 1), bc=(1, 0, 0), jitter=jitter)
    mesh = Mesh(m)
    x = I.vertex_mean(m)
    left = x[:, 0] < 0.5
    rho0 = np.where(left, 1.0, 0.125)
    p0 = np.where(left, 1.0, 0.1)
    Q0 = np.ascontiguousarray(I.primitive_to_conserved(rho0, np.zeros((len(rho0), 3)), p0))
    out = []
    for prec, name in ((GKS_PREC_FP64, "fp64"), (GKS_PREC_MIXED, "mixed")):
        rec = {"case": "sod", "mesh": layers, "precision": name, "cubes": n, "cells": mesh.n_cells,
               "flux_mode": flux_mode, "tau_model": tau_model, "cfl": cfl, "jitter": jitter,
               **weno}
        try:
            S = Solver(mesh, precision=prec, flux_mode=flux_mode, tau_model=tau_model, **weno)
            S.set_state(Q0)
            dt = S.max_dt(cfl)
            nsteps = int(np.ceil(t_end / dt - 1e-12))
            dt = t_end / nsteps
            t0 = time.perf_counter()
            S.step(dt, nsteps)
            torch.cuda.synchronize()
            rec["wall_s"] = time.perf_counter() - t0
            Q = S.get_state().cpu().numpy()
            xq, wq = S.cell_quadrature()
            vol = wq.sum(axis=1)
            re, _, _, ps, us = exact_riemann((1.0, 0.0, 1.0), (0.125, 0.0, 0.1),
                                             xq[..., 0].ravel(), t_end)
            ex = (re.reshape(wq.shape) * wq).sum(axis=1) / vol
            rec.update({"steps": nsteps, "dt": dt, "p_star": ps, "u_star": us,
                        "L1_rho": float((vol * np.abs(Q[0] - ex)).sum() / vol.sum()),
                        "mass_drift": float(abs((vol * Q[0]).sum() - (vol * Q0[0]).sum()) /
                                            (vol * Q0[0]).sum()),
                        "status": "ok"})
            S.close()
        except GksError as e:
            rec["status"] = f"stopped: {e}"
        _emit(rec)
        out.append(rec)
    return out


RIEMANN = {  # Section 5 (Riemann problems): left and right (rho, u, p), split at x = 0.5, t_end
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.2),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.16),
}


def riemann(problem="sod", mesh="hex", nx=100, cfl=0.5, flux_mode=1, tau_model=1, jitter=0.0,
            min_stencil=None, **weno):
    """The paper's Riemann-problem setup (Section 5): [0,1] x [0,0.1] x [0,0.1] with h = 1/nx,
    non-reflecting x ends (far-field planes holding the left and right states), reflecting y
    and z walls; meshes: nx x nx/10 x nx/10 hexahedra, the same cubes cut into Kuhn tetrahedra,
    or a hybrid of hexahedra, pyramid transition layers and tetrahedra. Full flux, inviscid
    collision time. Density, velocity and pressure L1 errors per unit volume against the exact
    solution's cell averages (27-point quadrature), FP64 and mixed. The hybrid mesh's
    transition layers take the enlarged stencils by default (min_stencil 18: with the stencils
    as printed, the unjittered split pyramids' stencils are rank deficient)."""
    import torch
    if min_stencil is None:
        min_stencil = 18 if mesh == "hybrid" else 0
    (rl, ul, pl), (rr, ur, pr), t_end = RIEMANN[problem]
    nz = max(nx // 10, 1)
    if mesh == "hybrid":
        if nz < 4 or nz % 2:
            raise ValueError("the hybrid Riemann mesh needs an even number (>= 4) of z layers")
        k = (nz - 2) // 2
        layers = ("hex",) * k + ("trans",) + ("tet",) * k + ("transm",)
    else:
        layers = (mesh,) * nz
    m = I.layered_box_mesh(nz, layers, lo=(0, 0, 0), hi=(1, 0.1, 0.1), bc=(3, 1, 1),
                           jitter=jitter, shape=(nx, nz))
    M = Mesh(m, min_stencil=min_stencil)
    x = I.vertex_mean(m)
    left = x[:, 0] < 0.5
    rho0 = np.where(left, rl, rr)
    U0 = np.zeros((len(rho0), 3))
    U0[:, 0] = np.where(left, ul, ur)
    p0 = np.where(left, pl, pr)
    Q0 = np.ascontiguousarray(I.primitive_to_conserved(rho0, U0, p0))
    far = np.tile(np.array([1.0, 0.0, 0.0, 0.0, 1.0]), (6, 1))
    far[0] = (rl, ul, 0.0, 0.0, pl)   # x = 0
    far[3] = (rr, ur, 0.0, 0.0, pr)   # x = 1
    out = []
    for prec, name in ((GKS_PREC_FP64, "fp64"), (GKS_PREC_MIXED, "mixed")):
        rec = {"case": "riemann", "problem": problem, "mesh": mesh, "precision": name, "nx": nx,
               "cells": M.n_cells, "flux_mode": flux_mode, "tau_model": tau_model, "cfl": cfl,
               "t_end": t_end, "jitter": jitter, "min_stencil": min_stencil, **weno}
        try:
            S = Solver(M, precision=prec, flux_mode=flux_mode, tau_model=tau_model, farfield=far,
                       **weno)
            S.set_state(Q0)
            dt = S.max_dt(cfl)
            nsteps = int(np.ceil(t_end / dt - 1e-12))
            dt = t_end / nsteps
            t0 = time.perf_counter()
            S.step(dt, nsteps)
            torch.cuda.synchronize()
            rec["wall_s"] = time.perf_counter() - t0
            Q = S.get_state().cpu().numpy()
            xq, wq = S.cell_quadrature()
            vol = wq.sum(axis=1)
            re, ue, pe, ps, us = exact_riemann((rl, ul, pl), (rr, ur, pr), xq[..., 0].ravel(),
                                               t_end)
            avg = lambda f: (f.reshape(wq.shape) * wq).sum(axis=1) / vol
            rho, u = Q[0], Q[1] / Q[0]
            p = 0.4 * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
            l1 = lambda a, b: float((vol * np.abs(a - b)).sum() / vol.sum())
            rec.update({"steps": nsteps, "dt": dt, "p_star": ps, "u_star": us,
                        "L1_rho": l1(rho, avg(re)), "L1_u": l1(u, avg(ue)),
                        "L1_p": l1(p, avg(pe)), "status": "ok"})
            S.close()
        except GksError as e:
            rec["status"] = f"stopped: {e}"
        _emit(rec)
        out.append(rec)
    return out


def implicit_steady(n=32, layers="hybrid8", steps=400, every=20, cfl=2.0, kmax=3, mu=1e-2,
                    precision="fp64"):
    """Implicit Jacobi steps (Section 4) on a relaxation problem: a gas at rest in a reflecting
    box [0,1]^3 with a smooth 2 % density and pressure bump (viscous smooth flux) rings
    acoustically and decays towards rest by viscosity; the relative L2 norm of the residual
    L(Q) is recorded every `every` steps."""
    m = I.layered_box_mesh(n, layers, lo=(0, 0, 0), hi=(1, 1, 1), bc=(1, 1, 1))
    mesh = Mesh(m)
    Q0 = I.rest_bump_state(m)
    prec = GKS_PREC_FP64 if precision == "fp64" else GKS_PREC_MIXED
    S = Solver(mesh, precision=prec, flux_mode=0, tau_model=2, mu=mu)
    S.set_state(Q0)
    dt = S.max_dt(cfl)
    hist = []
    t0 = time.perf_counter()
    for k in range(0, steps + 1, every):
        Q = S.get_state()
        L, _ = S.residual(Q, dt)
        hist.append((k, float(L.norm() / Q.norm())))
        if k < steps:
            S.step_implicit(dt, every, kmax)
    rec = {"case": "implicit_steady", "mesh": layers, "cubes": n, "cells": mesh.n_cells,
           "precision": precision, "cfl": cfl, "dt": dt, "kmax": kmax, "mu": mu,
           "residual_history": hist, "wall_s": time.perf_counter() - t0}
    _emit(rec)
    S.close()
    return rec


def cavity(n=20, layers="tet", re=100.0, mach=0.15, steps=2000, every=100, cfl=2.0, kmax=3,
           precision="fp64"):
    """Lid-driven cavity (Section 5.3): unit cube, every wall no-slip and isothermal at the gas
    temperature, the upper y plane moving along x at Ma 0.15 (rho = 1, p = 1/gamma, so c = 1),
    mu = U L / Re, full flux with tau = mu/p (the lid starts impulsively: the smooth flux, which
    assumes continuous data, does not carry the jump at the lid), implicit Jacobi steps
    (Section 4) from rest.
    Records the relative residual norm every `every` steps and, at the end, U on the vertical
    centre line (x = z = 1/2) and V on the horizontal one (y = z = 1/2), from the cells whose
    centroids lie within half a cube of the line."""
    m = I.layered_box_mesh(n, layers, lo=(0, 0, 0), hi=(1, 1, 1), bc=(2, 2, 2))
    mesh = Mesh(m)
    gamma, U = 1.4, mach
    T = 1.0 / gamma
    uw = np.zeros((6, 3))
    uw[4, 0] = U
    prec = GKS_PREC_FP64 if precision == "fp64" else GKS_PREC_MIXED
    S = Solver(mesh, precision=prec, flux_mode=1, tau_model=2, mu=U / re, wall_u=uw,
               wall_T=np.full(6, T))
    Q0 = np.zeros((5, mesh.n_cells))
    Q0[0] = 1.0
    Q0[4] = T / (gamma - 1.0)
    S.set_state(Q0)
    dt = S.max_dt(cfl)
    hist = []
    t0 = time.perf_counter()
    for k in range(0, steps + 1, every):
        Q = S.get_state()
        L, _ = S.residual(Q, dt)
        hist.append((k, float(L.norm() / Q.norm())))
        if k < steps:
            S.step_implicit(dt, every, kmax)
    wall = time.perf_counter() - t0
    Q = S.get_state().cpu().numpy()
    xq, wq = S.cell_quadrature()
    c = (xq * wq[..., None]).sum(axis=1) / wq.sum(axis=1)[:, None]
    h = 1.0 / n
    vert = (np.abs(c[:, 0] - 0.5) < 0.5 * h) & (np.abs(c[:, 2] - 0.5) < 0.5 * h)
    horz = (np.abs(c[:, 1] - 0.5) < 0.5 * h) & (np.abs(c[:, 2] - 0.5) < 0.5 * h)
    u = Q[1] / Q[0] / U
    v = Q[2] / Q[0] / U
    prof_u = sorted(zip(c[vert, 1].round(4).tolist(), u[vert].round(5).tolist()))
    prof_v = sorted(zip(c[horz, 0].round(4).tolist(), v[horz].round(5).tolist()))
    rec = {"case": "cavity", "mesh": layers, "cubes": n, "cells": mesh.n_cells,
           "precision": precision, "re": re, "mach": mach, "cfl": cfl, "dt": dt, "kmax": kmax,
           "steps": steps, "residual_history": hist, "wall_s": wall,
           "u_min_vertical": min(x[1] for x in prof_u), "v_max_horizontal": max(x[1] for x in prof_v),
           "v_min_horizontal": min(x[1] for x in prof_v), "u_vertical": prof_u,
           "v_horizontal": prof_v}
    _emit(rec)
    S.close()
    return rec


def couette(n=8, mu=0.05, mach=0.15, steps=3000, every=500, cfl=2.0, kmax=3, flux_mode=1,
            precision="fp64"):
    """Plane Couette flow between a stationary no-slip wall at y = 0 and one moving along x at
    y = 1 (both isothermal at the gas temperature; periodic x and z, n^3 hexahedra), implicit
    steps from rest. The steady momentum solution is the linear profile U = U_w y; records the
    largest |U - U_w y| / U_w over the cells and the residual history."""
    m = I.layered_box_mesh(n, "hex", lo=(0, 0, 0), hi=(1, 1, 1), bc=(0, 2, 0), jitter=0.0)
    mesh = Mesh(m)
    U, T = mach, 1.0 / 1.4
    uw = np.zeros((6, 3))
    uw[4, 0] = U
    prec = GKS_PREC_FP64 if precision == "fp64" else GKS_PREC_MIXED
    S = Solver(mesh, precision=prec, flux_mode=flux_mode, tau_model=2, mu=mu, wall_u=uw,
               wall_T=np.full(6, T))
    Q0 = np.zeros((5, mesh.n_cells))
    Q0[0] = 1.0
    Q0[4] = T / 0.4
    S.set_state(Q0)
    dt = S.max_dt(cfl)
    xq, wq = S.cell_quadrature()
    yc = (xq[..., 1] * wq).sum(axis=1) / wq.sum(axis=1)
    hist = []
    for k in range(0, steps + 1, every):
        Q = S.get_state()
        L, _ = S.residual(Q, dt)
        q = Q.cpu().numpy()
        err = float(np.abs(q[1] / q[0] - U * yc).max() / U)
        hist.append((k, float(L.norm() / Q.norm()), err))
        if k < steps:
            S.step_implicit(dt, every, kmax)
    rec = {"case": "couette", "cubes": n, "cells": mesh.n_cells, "precision": precision,
           "flux_mode": flux_mode, "mu": mu, "cfl": cfl, "dt": dt, "kmax": kmax,
           "history_step_residual_profile_error": hist}
    _emit(rec)
    S.close()
    return rec


def explosion(n=32, t_end=0.25, cfl=0.5, chunk=1, gp_fallback=1, precisions=("fp64", "mixed"),
              min_stencil=18):
    """Spherical explosion in the reflecting box [-1,1]^3 on the hybrid generator (full flux,
    inviscid collision time, WENO nonlinear weights): inside r < 0.4 rho = p = 1, outside
    rho = 0.125, p = 0.1, at rest. The FP64 run takes the CFL-bounded dt every `chunk` steps (1:
    every step; the blast accelerates the gas from rest, so a dt held for several steps from the
    early state exceeds the bound) and the mixed run replays the same dt sequence. Reports per precision: steps, cell-stage updates/s of
    the stepping, relative mass and energy drift (total and per step), min rho and p; and the
    mixed-vs-FP64 density difference (volume-weighted L1 per unit volume, relative to the mean
    density). gp_fallback = 1 takes the first-order state at Gauss points whose reconstruction is
    non-physical (the paper prints no positivity treatment; without it the jump stops the run at
    t = 0 with GKS_E_NONPHYSICAL)."""
    import torch
    if isinstance(precisions, str):
        precisions = tuple(precisions.split(","))
    m = I.layered_box_mesh(n, "hybrid8", lo=(-1, -1, -1), hi=(1, 1, 1), bc=(1, 1, 1))
    mesh = Mesh(m, min_stencil=min_stencil)
    Q0 = I.explosion_state(m)
    params = dict(flux_mode=1, tau_model=1, gp_fallback=gp_fallback)
    base = {"case": "explosion", "cubes": n, "cells": mesh.n_cells, "faces": mesh.n_faces,
            "t_end": t_end, "cfl": cfl, "gp_fallback": gp_fallback, "min_stencil": min_stencil}
    out, states, dts = [], {}, None
    for prec, name in ((GKS_PREC_FP64, "fp64"), (GKS_PREC_MIXED, "mixed")):
        if name not in precisions:
            continue
        rec = dict(base, precision=name)
        S = None
        try:
            S = Solver(mesh, precision=prec, **params)
            S.set_state(Q0)
            xq, wq = S.cell_quadrature()
            vol = wq.sum(axis=1)
            mass0, en0 = float((vol * Q0[0]).sum()), float((vol * Q0[4]).sum())
            sched = [] if dts is None else dts
            t, k, steps, el = 0.0, 0, 0, 0.0
            while (dts is None and t < t_end * (1 - 1e-12)) or (dts is not None and k < len(dts)):
                if dts is None:
                    dt = min(S.max_dt(cfl), (t_end - t) / chunk)
                    sched.append(dt)
                else:
                    dt = dts[k]
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                S.step(dt, chunk, check=False)
                torch.cuda.synchronize()
                el += time.perf_counter() - t0
                S.check()
                t += dt * chunk
                steps += chunk
                k += 1
            Q = S.get_state().cpu().numpy()
            p = 0.4 * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0])
            dm = abs(float((vol * Q[0]).sum()) - mass0) / mass0
            de = abs(float((vol * Q[4]).sum()) - en0) / en0
            rec.update({"status": "ok", "t": t, "steps": steps,
                        "cell_stage_per_s": mesh.n_cells * 2 * steps / el, "stepping_s": el,
                        "mass_drift": dm, "energy_drift": de, "mass_drift_per_step": dm / steps,
                        "energy_drift_per_step": de / steps, "min_rho": float(Q[0].min()),
                        "min_p": float(p.min()), "max_rho": float(Q[0].max())})
            states[name] = (Q, vol)
            dts = sched
        except GksError as e:
            rec["status"] = f"stopped: {e}"
        finally:
            if S is not None:
                S.close()
        _emit(rec)
        out.append(rec)
    if "fp64" in states and "mixed" in states:
        (Qd, vol), (Qm, _) = states["fp64"], states["mixed"]
        l1 = float((vol * np.abs(Qm[0] - Qd[0])).sum() / vol.sum())
        rec = dict(base, mixed_vs_fp64_L1_rho=l1,
                   mixed_vs_fp64_L1_rho_rel=l1 / float((vol * Qd[0]).sum() / vol.sum()),
                   mixed_vs_fp64_max_rho=float(np.abs(Qm[0] - Qd[0]).max()))
        _emit(rec)
        out.append(rec)
    mesh.close()
    return out


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "advection"
    kwargs = {}
    for a in sys.argv[2:]:
        k, v = a.split("=")
        try:
            kwargs[k] = int(v)
        except ValueError:
            try:
                kwargs[k] = float(v)
            except ValueError:
                kwargs[k] = v
    {"advection": advection, "tgv": tgv, "adjoint": adjoint, "explosion": explosion,
     "sod": sod, "implicit_steady": implicit_steady, "cavity": cavity,
     "riemann": riemann, "couette": couette}[which](**kwargs)
