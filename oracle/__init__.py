"""ctypes wrapper of the FP64 CPU oracle (gks_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the CPU-baseline leg of
the benchmark. The product path (the CUDA library and its binding) never imports this package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gks_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_gks.so")
_lib = None

# Parameter vector layout: gamma, mu, Pr, flux_mode, tau_model, tau_eps, tau_C, weno_gamma,
# weno_eps, weno_pow, weno_linear, T_ref, mu_pow, then per wall plane (axis + 3 side, side 1 the
# upper plane) the wall velocity (3) and temperature (<= 0: adiabatic), then per plane the
# far-field state (rho, U, V, W, p), then the Gauss-point positivity fallback switch.
DEFAULTS = dict(gamma=1.4, mu=0.0, Pr=1.0, flux_mode=0, tau_model=0, tau_eps=0.01, tau_C=1.0,
                weno_gamma=0.0125, weno_eps=1e-8, weno_pow=1, weno_linear=0, T_ref=1.0,
                mu_pow=0.7)
_ORDER = ["gamma", "mu", "Pr", "flux_mode", "tau_model", "tau_eps", "tau_C", "weno_gamma",
          "weno_eps", "weno_pow", "weno_linear", "T_ref", "mu_pow"]


def params_vec(wall_u=None, wall_T=None, farfield=None, gp_fallback=0, **kw) -> np.ndarray:
    """wall_u [6][3] and wall_T [6]: velocity and temperature of each wall plane (axis + 3 side);
    zero velocity and adiabatic walls by default. farfield: (rho, U, V, W, p) of the far field,
    one for all planes or [6][5] per plane (default 1, 0, 0, 0, 1/1.4)."""
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    walls = np.zeros((6, 4))
    if wall_u is not None:
        walls[:, :3] = np.asarray(wall_u, dtype=np.float64).reshape(6, 3)
    if wall_T is not None:
        walls[:, 3] = np.asarray(wall_T, dtype=np.float64).reshape(6)
    ff = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / 1.4]) if farfield is None else \
        np.asarray(farfield, dtype=np.float64)
    ff = np.broadcast_to(ff, (6, 5)).ravel() if ff.size == 5 else ff.reshape(30)
    return np.concatenate([np.array([float(d[k]) for k in _ORDER], dtype=np.float64),
                           walls.ravel(), ff, [float(gp_fallback)]])


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        L.oracle_mesh_create.restype = P
        L.oracle_mesh_create.argtypes = [ctypes.c_int64, D, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int8),
                                         ctypes.POINTER(ctypes.c_int64), I, D, D, ctypes.c_int,
                                         ctypes.c_int, I, ctypes.c_char_p, ctypes.c_int]
        L.oracle_mesh_destroy.argtypes = [P]
        L.oracle_n_faces.restype = ctypes.c_int64
        L.oracle_n_faces.argtypes = [P]
        L.oracle_cell_info.argtypes = [P, D, D, I, I, I]
        L.oracle_stencil_conditioning.argtypes = [P, D]
        L.oracle_face_info.argtypes = [P, I, I, D, D, D, D]
        L.oracle_cell_average.argtypes = [P, ctypes.c_int, ctypes.c_double, D, D]
        L.oracle_reconstruct_at.argtypes = [P, D, D, ctypes.c_int, I, D, D]
        L.oracle_gp_flux.argtypes = [D, D, D, D, D, ctypes.c_double, D]
        L.oracle_weno_detail.argtypes = [P, D, D, ctypes.c_int, D, D, D, D, D, I, D]
        L.oracle_weno_weights.restype = ctypes.c_double
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = None
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = ctypes.c_int
        L.oracle_weno_weights.argtypes = [D, ctypes.c_int, D, D]
        L.oracle_time_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, D]
        L.oracle_wall_ghost.argtypes = [D, ctypes.c_int, ctypes.c_int, D, D, D, D]
        L.oracle_slope.argtypes = [ctypes.c_double] * 5 + [D, D]
        L.oracle_residual.argtypes = [P, D, D, ctypes.c_double, D, D, ctypes.c_char_p, ctypes.c_int]
        L.oracle_residual_jvp.argtypes = [P, D, D, D, ctypes.c_double, D, D, D, D]
        L.oracle_residual_cells.argtypes = [P, D, D, ctypes.c_double, ctypes.c_int, I, D, D]
        L.oracle_step.argtypes = [P, D, D, ctypes.c_double, ctypes.c_int]
        L.oracle_step_implicit.argtypes = [P, D, D, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.oracle_step_jvp.argtypes = [P, D, D, D, ctypes.c_double, ctypes.c_int]
        L.oracle_s2o4_stage1.argtypes = [ctypes.c_int64, D, D, D, ctypes.c_double, D]
        L.oracle_s2o4_stage2.argtypes = [ctypes.c_int64, D, D, D, D, ctypes.c_double, D]
        L.oracle_max_dt.argtypes = [P, D, D, ctypes.c_double, D]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


class OracleError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"oracle status {status}: {msg}")
        self.status = status


class Mesh:
    """The oracle's view of a mesh: topology, geometry and stencils built from the inputs."""

    def __init__(self, mesh: dict, lazy: bool = False, min_stencil: int = 0):
        """min_stencil > 0: big stencils with fewer members take face neighbours of their members
        (a third ring, in stencil and face-label order) until they have min_stencil."""
        L = lib()
        xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        ct = np.ascontiguousarray(mesh["cell_type"], dtype=np.int8)
        cn = np.ascontiguousarray(mesh["cell_nodes"], dtype=np.int64)
        bc = np.ascontiguousarray(mesh["bc"], dtype=np.int32)
        lo = np.ascontiguousarray(mesh["lo"], dtype=np.float64)
        hi = np.ascontiguousarray(mesh["hi"], dtype=np.float64)
        st = ctypes.c_int(0)
        err = ctypes.create_string_buffer(256)
        self.h = L.oracle_mesh_create(len(xyz), _d(xyz), len(ct),
                                      ct.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                      cn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _i(bc),
                                      _d(lo), _d(hi), 1 if lazy else 0, int(min_stencil),
                                      ctypes.byref(st), err, 256)
        if not self.h:
            raise OracleError(st.value, err.value.decode())
        self.n_cells = len(ct)
        self.n_faces = int(L.oracle_n_faces(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_mesh_destroy(self.h)
            self.h = None

    def cell_info(self):
        n = self.n_cells
        vol, cen = np.zeros(n), np.zeros((n, 3))
        K, M, plain = (np.zeros(n, dtype=np.int32) for _ in range(3))
        lib().oracle_cell_info(self.h, _d(vol), _d(cen), _i(K), _i(M), _i(plain))
        return dict(vol=vol, centroid=cen, K=K, M=M, plain=plain.astype(bool))

    def stencil_conditioning(self):
        out = np.zeros(self.n_cells)
        lib().oracle_stencil_conditioning(self.h, _d(out))
        return out

    def face_info(self):
        nf = self.n_faces
        owner, nb = np.zeros(nf, dtype=np.int32), np.zeros(nf, dtype=np.int32)
        shift, xg, nrm, w = np.zeros((nf, 3)), np.zeros((nf, 4, 3)), np.zeros((nf, 4, 3)), np.zeros((nf, 4))
        lib().oracle_face_info(self.h, _i(owner), _i(nb), _d(shift), _d(xg), _d(nrm), _d(w))
        return dict(owner=owner, nb=nb, shift=shift, xg=xg, normal=nrm, w=w)

    def cell_average(self, field: int, t: float = 0.0, fp=None) -> np.ndarray:
        fp = np.ascontiguousarray(np.zeros(1) if fp is None else fp, dtype=np.float64)
        Q = np.zeros((5, self.n_cells))
        st = lib().oracle_cell_average(self.h, field, t, _d(fp), _d(Q))
        if st:
            raise OracleError(st)
        return Q

    def advection_average(self, t=0.0, gamma=1.4):
        return self.cell_average(0, t, np.array([gamma]))

    def reconstruct_at(self, params, Q, cells, x):
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        x = np.ascontiguousarray(x, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros((len(cells), 5, 4))
        lib().oracle_reconstruct_at(self.h, _d(params), _d(Q), len(cells), _i(cells), _d(x), _d(out))
        return out

    def weno_detail(self, params, Q, cell):
        """The parts of one cell's WENO reconstruction (Section 2), per conserved variable:
        a [5][9] (P0 in the basis x, y, z, xx, yy, zz, xy, xz, yz of coordinates about the
        centroid scaled by h = |Omega|^(1/3)), b [5][M][3], beta [5][M+1], wbar [5][M+1],
        tau [5], and h."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        a, b = np.zeros((5, 9)), np.zeros((5, 16, 3))
        beta, wbar, tau = np.zeros((5, 17)), np.zeros((5, 17)), np.zeros(5)
        M, h = ctypes.c_int(0), np.zeros(1)
        st = lib().oracle_weno_detail(self.h, _d(params), _d(Q), int(cell), _d(a), _d(b), _d(beta),
                                      _d(wbar), _d(tau), ctypes.byref(M), _d(h))
        if st:
            raise OracleError(st)
        M = M.value
        return dict(a=a, b=b[:, :M], beta=beta[:, :M + 1], wbar=wbar[:, :M + 1], tau=tau, M=M,
                    h=float(h[0]))

    def residual(self, params, Q, dt):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        L, Lt = np.zeros_like(Q), np.zeros_like(Q)
        err = ctypes.create_string_buffer(256)
        st = lib().oracle_residual(self.h, _d(params), _d(Q), dt, _d(L), _d(Lt), err, 256)
        if st:
            raise OracleError(st, err.value.decode())
        return L, Lt

    def residual_cells(self, params, Q, dt, cells):
        """L and Lt [len(cells), 5] of the listed cells only."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        L, Lt = np.zeros((len(cells), 5)), np.zeros((len(cells), 5))
        st = lib().oracle_residual_cells(self.h, _d(params), _d(Q), dt, len(cells), _i(cells), _d(L), _d(Lt))
        if st:
            raise OracleError(st)
        return L, Lt

    def residual_jvp(self, params, Q, dQ, dt):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        dQ = np.ascontiguousarray(dQ, dtype=np.float64)
        L, Lt, dL, dLt = (np.zeros_like(Q) for _ in range(4))
        st = lib().oracle_residual_jvp(self.h, _d(params), _d(Q), _d(dQ), dt, _d(L), _d(Lt), _d(dL), _d(dLt))
        if st:
            raise OracleError(st)
        return L, Lt, dL, dLt

    def step(self, params, Q, dt, nsteps=1):
        Q = np.array(Q, dtype=np.float64, order="C", copy=True)
        st = lib().oracle_step(self.h, _d(params), _d(Q), dt, nsteps)
        if st:
            raise OracleError(st)
        return Q

    def step_implicit(self, params, Q, dt, nsteps=1, kmax=3):
        """Implicit backward-Euler steps, kmax Jacobi iterations each (Section 4)."""
        Q = np.array(Q, dtype=np.float64, order="C", copy=True)
        st = lib().oracle_step_implicit(self.h, _d(params), _d(Q), dt, nsteps, kmax)
        if st:
            raise OracleError(st)
        return Q

    def step_jvp(self, params, Q, dQ, dt, nsteps=1):
        Q = np.array(Q, dtype=np.float64, order="C", copy=True)
        dQ = np.array(dQ, dtype=np.float64, order="C", copy=True)
        st = lib().oracle_step_jvp(self.h, _d(params), _d(Q), _d(dQ), dt, nsteps)
        if st:
            raise OracleError(st)
        return Q, dQ

    def max_dt(self, params, Q, cfl):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros(1)
        st = lib().oracle_max_dt(self.h, _d(params), _d(Q), cfl, _d(out))
        if st:
            raise OracleError(st)
        return float(out[0])


def gp_flux(params, ql, dql, qr, dqr, dt):
    """Local-frame Gauss-point flux: returns F[2][5] = time integrals over [0,dt/2] and [0,dt]."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (ql, dql, qr, dqr)]
    F = np.zeros((2, 5))
    st = lib().oracle_gp_flux(_d(params), *[_d(a) for a in arrs], dt, _d(F))
    if st:
        raise OracleError(st)
    return F


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle's loops use from now on."""
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def weno_weights(params, beta):
    """Normalised nonlinear weights wbar[0..M] and tau from indicators beta[0..M] (Section 2)."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    wbar = np.zeros_like(beta)
    tau = lib().oracle_weno_weights(_d(params), len(beta) - 1, _d(beta), _d(wbar))
    return wbar, float(tau)


def wall_ghost(params, kind, plane, v, g):
    """Ghost value and gradient (global frame, g[5][3] = d v_r / d x_b) at a point of a wall of
    the given kind (1 slip, 2 no-slip) on plane axis + 3 side."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(5, 3)
    vg, gg = np.zeros(5), np.zeros((5, 3))
    lib().oracle_wall_ghost(_d(params), int(kind), int(plane), _d(v), _d(g), _d(vg), _d(gg))
    return vg, gg


def time_coeffs(tau, delta):
    c = np.zeros(6)
    lib().oracle_time_coeffs(tau, delta, _d(c))
    return c


def slope(U, V, W, lam, K, b):
    b = np.ascontiguousarray(b, dtype=np.float64)
    a = np.zeros(5)
    lib().oracle_slope(U, V, W, lam, K, _d(b), _d(a))
    return a


def s2o4(Q, L, Lt, Lts, dt):
    """(Q*, Q^{n+1}) from the oracle's two stage updates (Lts is the stage-2 time derivative)."""
    Q, L, Lt, Lts = (np.ascontiguousarray(a, dtype=np.float64) for a in (Q, L, Lt, Lts))
    Qs, Qn = np.zeros_like(Q), np.zeros_like(Q)
    lib().oracle_s2o4_stage1(Q.size, _d(Q), _d(L), _d(Lt), dt, _d(Qs))
    lib().oracle_s2o4_stage2(Q.size, _d(Q), _d(L), _d(Lt), _d(Lts), dt, _d(Qn))
    return Qs, Qn
