"""The CUDA path's Gauss-point flux arithmetic, instantiated on the host in FP64 (same
templates as the kernels): forward against the oracle's generic moment formulation, and the
hand-written vector-Jacobian product against central differences. No GPU needed."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2203_09047_gb300 as gks
from paper_2203_09047_gb300 import build

CASES = [(0, 0), (0, 2), (1, 1), (1, 2), (1, 0)]
D = ctypes.POINTER(ctypes.c_double)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(D)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gks.load_library()


def _state(rng):
    rho = 1.0 + 0.3 * rng.random()
    U = rng.normal(size=3) * 0.5
    p = 0.8 + 0.4 * rng.random()
    return np.array([rho, rho * U[0], rho * U[1], rho * U[2], p / 0.4 + 0.5 * rho * U @ U])


def _flux(lib, P, x, dt):
    Fn, Ft = np.zeros(5), np.zeros(5)
    st = lib.gks_gp_flux_host(_d(P), _d(x[:5]), _d(x[5:20]), _d(x[20:25]), _d(x[25:40]),
                              ctypes.c_double(dt), Fn.ctypes.data_as(D), Ft.ctypes.data_as(D))
    assert st == 0
    return np.concatenate([Fn, Ft])


@pytest.mark.parametrize("mode,tau_model", CASES)
def test_gp_flux_matches_oracle(lib, mode, tau_model):
    rng = np.random.default_rng(100 + 7 * mode + tau_model)
    P = np.array([1.4, 2e-3, 0.01, 1.0, mode, tau_model, 1.0])
    Po = oracle.params_vec(flux_mode=mode, tau_model=tau_model, mu=2e-3)
    for _ in range(6):
        ql, qr = _state(rng), _state(rng)
        dql, dqr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        dt = 0.01
        F = _flux(lib, P, np.concatenate([ql, dql.ravel(), qr, dqr.ravel()]), dt)
        Fo = oracle.gp_flux(Po, ql, dql, qr, dqr, dt)
        Fn_o, Ft_o = (4 * Fo[0] - Fo[1]) / dt, 4 * (Fo[1] - 2 * Fo[0]) / dt ** 2
        np.testing.assert_allclose(F[:5], Fn_o, rtol=0, atol=1e-11 * np.abs(Fn_o).max())
        np.testing.assert_allclose(F[5:], Ft_o, rtol=0, atol=1e-10 * np.abs(Ft_o).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_gp_flux_large_collision_time_matches_oracle(lib, mode):
    """mu = 0.2: tau = mu/p + ... makes the tau terms (the second-moment flux of the slopes, E1)
    a tenth of F^n, so they are pinned to the oracle too."""
    rng = np.random.default_rng(170 + mode)
    P = np.array([1.4, 0.2, 0.01, 1.0, mode, 2, 1.0])
    Po = oracle.params_vec(flux_mode=mode, tau_model=2, mu=0.2)
    for _ in range(6):
        ql, qr = _state(rng), _state(rng)
        dql, dqr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        dt = 0.01
        F = _flux(lib, P, np.concatenate([ql, dql.ravel(), qr, dqr.ravel()]), dt)
        Fo = oracle.gp_flux(Po, ql, dql, qr, dqr, dt)
        Fn_o, Ft_o = (4 * Fo[0] - Fo[1]) / dt, 4 * (Fo[1] - 2 * Fo[0]) / dt ** 2
        np.testing.assert_allclose(F[:5], Fn_o, rtol=0, atol=1e-11 * np.abs(Fn_o).max())
        np.testing.assert_allclose(F[5:], Ft_o, rtol=0, atol=1e-10 * np.abs(Ft_o).max())


def test_gp_flux_prandtl_fix_matches_oracle(lib):
    rng = np.random.default_rng(150)
    P = np.array([1.4, 3e-3, 0.01, 1.0, 0, 2, 0.72])
    Po = oracle.params_vec(flux_mode=0, tau_model=2, mu=3e-3, Pr=0.72)
    for _ in range(6):
        ql, qr = _state(rng), _state(rng)
        dql, dqr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        dt = 0.01
        F = _flux(lib, P, np.concatenate([ql, dql.ravel(), qr, dqr.ravel()]), dt)
        Fo = oracle.gp_flux(Po, ql, dql, qr, dqr, dt)
        Fn_o, Ft_o = (4 * Fo[0] - Fo[1]) / dt, 4 * (Fo[1] - 2 * Fo[0]) / dt ** 2
        np.testing.assert_allclose(F[:5], Fn_o, rtol=0, atol=1e-11 * np.abs(Fn_o).max())
        np.testing.assert_allclose(F[5:], Ft_o, rtol=0, atol=1e-10 * np.abs(Ft_o).max())


@pytest.mark.parametrize("mode,tau_model", CASES)
def test_gp_flux_vjp_matches_central_differences(lib, mode, tau_model):
    rng = np.random.default_rng(200 + 7 * mode + tau_model)
    P = np.array([1.4, 2e-3, 0.01, 1.0, mode, tau_model, 1.0])
    dt = 0.01
    for _ in range(3):
        ql, qr = _state(rng), _state(rng)
        dql, dqr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
        x = np.concatenate([ql, dql.ravel(), qr, dqr.ravel()])
        g = rng.normal(size=10)
        out = [np.zeros(5), np.zeros(15), np.zeros(5), np.zeros(15)]
        st = lib.gks_gp_flux_vjp_host(_d(P), _d(ql), _d(dql), _d(qr), _d(dqr), ctypes.c_double(dt),
                                      _d(g[:5]), _d(g[5:]), *[o.ctypes.data_as(D) for o in out])
        assert st == 0
        gx = np.concatenate(out)
        fd = np.zeros(40)
        for k in range(40):
            h = 1e-6 * max(1.0, abs(x[k]))
            e = np.zeros(40)
            e[k] = h
            fd[k] = g @ (_flux(lib, P, x + e, dt) - _flux(lib, P, x - e, dt)) / (2 * h)
        assert np.abs(gx - fd).max() < 1e-7 * np.abs(fd).max()


@pytest.mark.parametrize("mode,tau_model", [(0, 0), (1, 2)])
def test_global_frame_vjp_matches_central_differences(lib, mode, tau_model):
    """Rotation into the Gauss point's frame, flux, rotation back and weight, reversed."""
    rng = np.random.default_rng(300 + mode)
    P = np.array([1.4, 2e-3, 0.01, 1.0, mode, tau_model, 1.0])
    n1 = rng.normal(size=3)
    n1 /= np.linalg.norm(n1)
    w, dt = 0.037, 0.01
    vl, vr = _state(rng), _state(rng)
    gl, gr = rng.normal(size=15) * 0.2, rng.normal(size=15) * 0.2
    x = np.concatenate([vl, gl, vr, gr])

    def f(x):
        acc = np.zeros(10)
        assert lib.gks_gp_face_host(_d(P), _d(x[:5]), _d(x[5:20]), _d(x[20:25]), _d(x[25:40]), _d(n1),
                                    ctypes.c_double(w), ctypes.c_double(dt), acc.ctypes.data_as(D),
                                    None, None, None, None, None) == 0
        return acc

    g = rng.normal(size=10)
    acc = np.zeros(10)
    out = [np.zeros(5), np.zeros(15), np.zeros(5), np.zeros(15)]
    assert lib.gks_gp_face_host(_d(P), _d(vl), _d(gl), _d(vr), _d(gr), _d(n1), ctypes.c_double(w),
                                ctypes.c_double(dt), acc.ctypes.data_as(D), _d(g),
                                *[o.ctypes.data_as(D) for o in out]) == 0
    gx = np.concatenate(out)
    fd = np.zeros(40)
    for k in range(40):
        h = 1e-6 * max(1.0, abs(x[k]))
        e = np.zeros(40)
        e[k] = h
        fd[k] = g @ (f(x + e) - f(x - e)) / (2 * h)
    assert np.abs(gx - fd).max() < 1e-7 * np.abs(fd).max()
