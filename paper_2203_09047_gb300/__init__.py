"""GB300 gas-kinetic solver for 3D hybrid unstructured meshes (arXiv 2203.09047).

A thin ctypes binding of the C ABI declared in include/gks.h. Every step of the hot path
(reconstruction, gas-kinetic flux, face sums, two-stage update, time-step bound) runs in the CUDA
kernels of libgks.so; this module only marshals arguments (torch tensors pass their data_ptr()).
There is no CPU fallback: importing the binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgks.so")

GKS_OK, GKS_E_INVAL, GKS_E_NOMEM, GKS_E_CUDA, GKS_E_MESH, GKS_E_SINGULAR, GKS_E_NONPHYSICAL, \
    GKS_E_TIMEOUT = range(8)
STATUS_NAMES = ["GKS_OK", "GKS_E_INVAL", "GKS_E_NOMEM", "GKS_E_CUDA", "GKS_E_MESH",
                "GKS_E_SINGULAR", "GKS_E_NONPHYSICAL", "GKS_E_TIMEOUT"]
GKS_FLUX_SMOOTH, GKS_FLUX_FULL = 0, 1
GKS_TAU_ZERO, GKS_TAU_INVISCID, GKS_TAU_VISCOUS, GKS_TAU_POWER_LAW = 0, 1, 2, 3
GKS_BC_PERIODIC, GKS_BC_REFLECT, GKS_BC_NOSLIP, GKS_BC_FARFIELD = 0, 1, 2, 3
GKS_PREC_FP64, GKS_PREC_MIXED, GKS_PREC_MIXED_FP64UPD = 0, 1, 2


class gks_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("flux_mode", ctypes.c_int), ("tau_model", ctypes.c_int),
                ("tau_eps", ctypes.c_double), ("tau_C", ctypes.c_double),
                ("weno_gamma", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("weno_pow", ctypes.c_int), ("precision", ctypes.c_int),
                ("T_ref", ctypes.c_double), ("mu_pow", ctypes.c_double),
                ("wall_u", (ctypes.c_double * 3) * 6), ("wall_T", ctypes.c_double * 6),
                ("farfield", (ctypes.c_double * 5) * 6), ("gp_fallback", ctypes.c_int)]


GKS_REORDER_NONE, GKS_REORDER_MORTON, GKS_REORDER_RCM = 0, 1, 2


class gks_mesh_options(ctypes.Structure):
    _fields_ = [("reorder", ctypes.c_int), ("min_stencil", ctypes.c_int)]


class GksError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgks.so (built by paper_2203_09047_gb300.build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2203_09047_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, D, I64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    st = ctypes.c_int
    L.gks_params_default.argtypes = [ctypes.POINTER(gks_params)]
    L.gks_params_default.restype = None
    L.gks_mesh_create.argtypes = [I64, P, I64, P, P, P, P, P, ctypes.POINTER(P)]
    L.gks_mesh_create.restype = st
    L.gks_mesh_create_ex.argtypes = [I64, P, I64, P, P, P, P, P, ctypes.POINTER(gks_mesh_options),
                                     ctypes.POINTER(P)]
    L.gks_mesh_create_ex.restype = st
    L.gks_mesh_counts.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.gks_mesh_counts.restype = st
    L.gks_mesh_last_error.argtypes = []
    L.gks_mesh_last_error.restype = ctypes.c_char_p
    L.gks_init.argtypes = [P, ctypes.POINTER(gks_params), P, ctypes.POINTER(P)]
    L.gks_init.restype = st
    L.gks_set_state.argtypes = [P, P]
    L.gks_set_state.restype = st
    L.gks_get_state.argtypes = [P, P]
    L.gks_get_state.restype = st
    L.gks_max_dt.argtypes = [P, ctypes.c_double, D]
    L.gks_max_dt.restype = st
    L.gks_step.argtypes = [P, ctypes.c_double, ctypes.c_int]
    L.gks_step.restype = st
    L.gks_step_implicit.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.gks_step_implicit.restype = st
    L.gks_check.argtypes = [P]
    L.gks_check.restype = st
    L.gks_residual.argtypes = [P, P, ctypes.c_double, P, P]
    L.gks_residual.restype = st
    L.gks_residual_vjp.argtypes = [P, P, ctypes.c_double, P, P, P]
    L.gks_residual_vjp.restype = st
    L.gks_timing_enable.argtypes = [P, ctypes.c_int]
    L.gks_timing_enable.restype = st
    L.gks_timing_read.argtypes = [P, D, ctypes.POINTER(I64)]
    L.gks_timing_read.restype = st
    L.gks_cell_quadrature.argtypes = [P, P, P]
    L.gks_cell_quadrature.restype = st
    L.gks_kernel_bytes.argtypes = [P, D]
    L.gks_kernel_bytes.restype = st
    L.gks_launches_per_pass.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.gks_launches_per_pass.restype = st
    L.gks_flux_opcount.argtypes = [ctypes.c_int, ctypes.c_int, D, D]
    L.gks_flux_opcount.restype = ctypes.c_int
    L.gks_cfl_dt_noalloc.argtypes = [I64, P, P, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, P, P]
    L.gks_cfl_dt_noalloc.restype = st
    L.gks_partition_create.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]
    L.gks_partition_create.restype = st
    L.gks_partition_counts.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.gks_partition_counts.restype = st
    L.gks_partition_cells.argtypes = [P, P, P, P]
    L.gks_partition_cells.restype = st
    L.gks_partition_send.argtypes = [P, ctypes.c_int, ctypes.POINTER(I64), P]
    L.gks_partition_send.restype = st
    L.gks_partition_destroy.argtypes = [P]
    L.gks_partition_destroy.restype = None
    L.gks_debug_recon_wait.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.gks_debug_recon_wait.restype = st
    L.gks_alu_peaks.argtypes = [D, D]
    L.gks_alu_peaks.restype = st
    L.gks_s2o4_stage.argtypes = [I64, ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
    L.gks_s2o4_stage.restype = st
    L.gks_s2o4_stage_vjp.argtypes = [I64, ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
    L.gks_s2o4_stage_vjp.restype = st
    for name in ("gks_gp_flux_host", "gks_gp_flux_vjp_host", "gks_gp_face_host"):
        getattr(L, name).restype = ctypes.c_int
    L.gks_gp_face_f32_pair.argtypes = [P, ctypes.c_int, P, P]
    L.gks_gp_face_f32_pair.restype = ctypes.c_int
    L.gks_wall_ghost_host.argtypes = [P, ctypes.c_int] + [P] * 8
    L.gks_wall_ghost_host.restype = None
    L.gks_wall_flux_fix_host.argtypes = [P, ctypes.c_int, P]
    L.gks_wall_flux_fix_host.restype = None
    L.gks_last_error.argtypes = [P]
    L.gks_last_error.restype = ctypes.c_char_p
    L.gks_destroy.argtypes = [P]
    L.gks_destroy.restype = None
    L.gks_mesh_destroy.argtypes = [P]
    L.gks_mesh_destroy.restype = None
    _lib = L
    return L


def _ptr(a) -> int:
    """Raw address of a contiguous float64/int array: torch tensor (host or device) or numpy."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    return a.ctypes.data


# ---------------------------------------------------------------------------- C-ABI names
def gks_params_default(**overrides) -> gks_params:
    p = gks_params()
    load_library().gks_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        if k == "wall_u":
            v = np.asarray(v, dtype=np.float64).reshape(6, 3)
            for w in range(6):
                for a in range(3):
                    p.wall_u[w][a] = float(v[w, a])
        elif k == "wall_T":
            v = np.asarray(v, dtype=np.float64).reshape(6)
            for w in range(6):
                p.wall_T[w] = float(v[w])
        elif k == "farfield":  # one state for every plane, or [6][5]
            v = np.asarray(v, dtype=np.float64)
            v = np.broadcast_to(v, (6, 5)) if v.size == 5 else v.reshape(6, 5)
            for w in range(6):
                for j in range(5):
                    p.farfield[w][j] = float(v[w, j])
        else:
            setattr(p, k, v)
    return p


def gks_mesh_create(xyz, cell_type, cell_nodes, bc, lo, hi, reorder: int = GKS_REORDER_MORTON,
                    min_stencil: int = 0) -> ctypes.c_void_p:
    L = load_library()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    ct = np.ascontiguousarray(cell_type, dtype=np.int8)
    cn = np.ascontiguousarray(cell_nodes, dtype=np.int64)
    bc = np.ascontiguousarray(bc, dtype=np.int32)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    out = ctypes.c_void_p()
    opt = gks_mesh_options(int(reorder), int(min_stencil))
    s = L.gks_mesh_create_ex(len(xyz), xyz.ctypes.data, len(ct), ct.ctypes.data, cn.ctypes.data,
                             bc.ctypes.data, lo.ctypes.data, hi.ctypes.data, ctypes.byref(opt),
                             ctypes.byref(out))
    if s != GKS_OK:
        raise GksError(s, L.gks_mesh_last_error().decode())
    return out


def gks_mesh_counts(mesh) -> tuple:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().gks_mesh_counts(mesh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def gks_init(mesh, params: gks_params, stream: int = 0) -> ctypes.c_void_p:
    L = load_library()
    out = ctypes.c_void_p()
    s = L.gks_init(mesh, ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(out))
    if s != GKS_OK:
        raise GksError(s, L.gks_mesh_last_error().decode())
    return out


def _check(s, solver=None):
    if s != GKS_OK:
        msg = load_library().gks_last_error(solver).decode() if solver else ""
        raise GksError(s, msg)


def gks_set_state(solver, Q):
    _check(load_library().gks_set_state(solver, _ptr(Q)), solver)


def gks_get_state(solver, Q):
    _check(load_library().gks_get_state(solver, _ptr(Q)), solver)


def gks_max_dt(solver, cfl: float) -> float:
    out = ctypes.c_double()
    _check(load_library().gks_max_dt(solver, cfl, ctypes.byref(out)), solver)
    return out.value


def gks_step(solver, dt: float, nsteps: int = 1):
    _check(load_library().gks_step(solver, dt, nsteps), solver)


def gks_step_implicit(solver, dt: float, nsteps: int = 1, kmax: int = 3):
    _check(load_library().gks_step_implicit(solver, dt, nsteps, kmax), solver)


def gks_check(solver):
    _check(load_library().gks_check(solver), solver)


def gks_residual(solver, Q, dt: float, L, Lt):
    _check(load_library().gks_residual(solver, _ptr(Q), dt, _ptr(L), _ptr(Lt)), solver)


def gks_residual_vjp(solver, Q, dt: float, gL, gLt, gQ):
    _check(load_library().gks_residual_vjp(solver, _ptr(Q), dt, _ptr(gL), _ptr(gLt), _ptr(gQ)),
           solver)


def gks_timing_enable(solver, enable: bool = True):
    _check(load_library().gks_timing_enable(solver, 1 if enable else 0), solver)


def gks_timing_read(solver):
    """(ms[3], counts[3]) for reconstruction, face flux, face sum + update since the last read."""
    ms = (ctypes.c_double * 3)()
    cnt = (ctypes.c_int64 * 3)()
    _check(load_library().gks_timing_read(solver, ms, cnt), solver)
    return list(ms), list(cnt)


def gks_cell_quadrature(solver, xq, wq):
    _check(load_library().gks_cell_quadrature(solver, _ptr(xq), _ptr(wq)), solver)


def gks_kernel_bytes(solver):
    """Algorithmic bytes per pass of (reconstruction, flux, face sum + update)."""
    b = (ctypes.c_double * 3)()
    _check(load_library().gks_kernel_bytes(solver, b), solver)
    return list(b)


def gks_launches_per_pass(solver):
    """Kernel launches in one pass of (reconstruction, flux, face sum + update)."""
    n = (ctypes.c_int64 * 3)()
    _check(load_library().gks_launches_per_pass(solver, n), solver)
    return list(n)


def gks_flux_opcount(flux_mode: int, tau_model: int):
    """(flops, special-function calls) of one face Gauss point of the flux kernel."""
    f, sp = ctypes.c_double(), ctypes.c_double()
    if load_library().gks_flux_opcount(flux_mode, tau_model, ctypes.byref(f), ctypes.byref(sp)):
        raise GksError(GKS_E_NONPHYSICAL, "op count failed")
    return f.value, sp.value


def gks_cfl_dt_noalloc(n_cells: int, Q, h, gamma: float, mu: float, cfl: float, dt_out,
                       stream: int = 0):
    """Allocation-free CFL bound: Q [5, n] and h [n] device float64, dt_out a device float64[1]."""
    L = load_library()
    s = L.gks_cfl_dt_noalloc(n_cells, _ptr(Q), _ptr(h), gamma, mu, cfl, _ptr(dt_out),
                             ctypes.c_void_p(stream))
    if s != GKS_OK:
        raise GksError(s, L.gks_last_error(None).decode())


def gks_debug_recon_wait(solver, wait_tries: int, withhold_copies: bool):
    _check(load_library().gks_debug_recon_wait(solver, int(wait_tries), 1 if withhold_copies else 0),
           solver)


def gks_alu_peaks():
    """Measured (FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    s = lib.gks_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if s != GKS_OK:
        raise GksError(s, lib.gks_last_error(None).decode())
    return a.value, b.value


def gks_s2o4_stage(stage: int, dt: float, Q, L, Lt, Lts, out, stream: int = 0):
    """out = the stage-1 or stage-2 combination of Section 3.3 (device float64 tensors, same
    shape; Lts may be None in stage 1)."""
    lib = load_library()
    s = lib.gks_s2o4_stage(Q.numel(), stage, dt, _ptr(Q), _ptr(L), _ptr(Lt),
                           None if Lts is None else _ptr(Lts), _ptr(out), ctypes.c_void_p(stream))
    if s != GKS_OK:
        raise GksError(s, lib.gks_last_error(None).decode())


def gks_s2o4_stage_vjp(stage: int, dt: float, g, gQ, gL, gLt, gLts, stream: int = 0):
    """Cotangents of Q, L, Lt (and Lts in stage 2) for a cotangent g of the stage output."""
    lib = load_library()
    s = lib.gks_s2o4_stage_vjp(g.numel(), stage, dt, _ptr(g), _ptr(gQ), _ptr(gL), _ptr(gLt),
                               None if gLts is None else _ptr(gLts), ctypes.c_void_p(stream))
    if s != GKS_OK:
        raise GksError(s, lib.gks_last_error(None).decode())


def gks_destroy(solver):
    load_library().gks_destroy(solver)


def gks_mesh_destroy(mesh):
    load_library().gks_mesh_destroy(mesh)


# ---------------------------------------------------------------------------- convenience
class Mesh:
    """Owns a gks_mesh handle built from an inputs-style mesh dict (host-side topology only)."""

    def __init__(self, mesh: dict, reorder: int = GKS_REORDER_MORTON, min_stencil: int = 0):
        self.h = gks_mesh_create(mesh["xyz"], mesh["cell_type"], mesh["cell_nodes"], mesh["bc"],
                                 mesh["lo"], mesh["hi"], reorder, min_stencil)
        self.n_cells, self.n_faces, self.n_stencil = gks_mesh_counts(self.h)

    def close(self):
        if getattr(self, "h", None):
            gks_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns a solver handle; states are torch float64 tensors [5, n_cells] on the solver's CUDA
    device (or pinned host tensors for host-side transfers). `mesh` is an inputs-style dict or a
    Mesh (which may be shared by several solvers)."""

    def __init__(self, mesh, stream=None, reorder=None, min_stencil=None, **params):
        """reorder / min_stencil are mesh options (gks_mesh_options), for a mesh dict only."""
        import torch
        self.torch = torch
        own = not isinstance(mesh, Mesh)
        if not own and (reorder is not None or min_stencil is not None):
            raise ValueError("reorder and min_stencil belong to the Mesh, which is already built")
        M = Mesh(mesh, GKS_REORDER_MORTON if reorder is None else reorder,
                 0 if min_stencil is None else min_stencil) if own else mesh
        self.n_cells, self.n_faces, self.n_stencil = M.n_cells, M.n_faces, M.n_stencil
        self.params = gks_params_default(**params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        try:
            self.h = gks_init(M.h, self.params, self.stream.cuda_stream)
        finally:
            if own:
                M.close()

    def close(self):
        if getattr(self, "h", None):
            gks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, Q):
        t = self.torch
        if isinstance(Q, np.ndarray):
            Q = t.from_numpy(Q)
        return Q.to(device="cuda", dtype=t.float64).contiguous()

    def set_state(self, Q):
        Q = self._dev(Q)
        gks_set_state(self.h, Q)
        self.stream.synchronize()

    def get_state(self):
        Q = self.torch.empty((5, self.n_cells), dtype=self.torch.float64, device="cuda")
        gks_get_state(self.h, Q)
        return Q

    def max_dt(self, cfl: float) -> float:
        return gks_max_dt(self.h, cfl)

    def step(self, dt: float, nsteps: int = 1, check: bool = True):
        gks_step(self.h, dt, nsteps)
        if check:
            gks_check(self.h)

    def check(self):
        """Raise GksError if an earlier step met a non-physical state (gks_check)."""
        gks_check(self.h)

    def step_implicit(self, dt: float, nsteps: int = 1, kmax: int = 3, check: bool = True):
        """Implicit backward-Euler steps with kmax Jacobi iterations (Section 4)."""
        gks_step_implicit(self.h, dt, nsteps, kmax)
        if check:
            gks_check(self.h)

    def residual(self, Q, dt: float):
        Q = self._dev(Q)
        L = self.torch.empty_like(Q)
        Lt = self.torch.empty_like(Q)
        gks_residual(self.h, Q, dt, L, Lt)
        return L, Lt

    def cell_quadrature(self):
        """(points [n, 27, 3], weights [n, 27]) as float64 numpy arrays, caller order."""
        xq = np.empty((self.n_cells, 27, 3))
        wq = np.empty((self.n_cells, 27))
        gks_cell_quadrature(self.h, xq, wq)
        return xq, wq

    def cell_average(self, field):
        """Cell averages [5, n] of field(x[..., 3]) -> [5, ...] by the 27-point quadrature."""
        xq, wq = self.cell_quadrature()
        vals = field(xq)
        return np.ascontiguousarray((vals * wq[None]).sum(axis=-1) / wq.sum(axis=-1)[None])

    def residual_vjp(self, Q, dt: float, gL, gLt):
        Q, gL, gLt = self._dev(Q), self._dev(gL), self._dev(gLt)
        gQ = self.torch.empty_like(Q)
        gks_residual_vjp(self.h, Q, dt, gL, gLt, gQ)
        return gQ
