"""The CUDA path's Gauss-point flux arithmetic, instantiated on the host in FP64 (same
templates as the kernels): forward against the oracle's generic moment formulation, and the
hand-written vector-Jacobian product against central differences. No GPU needed."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2203_09047_gb300 as gks
from paper_2203_09047_gb300 import build

CASES = [(0, 0), (0, 2), (1, 1), (1, 2), (1, 0), (0, 3), (1, 3)]
T_REF = 0.9  # power-law reference temperature of the tau_model 3 cases
D = ctypes.POINTER(ctypes.c_double)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(D)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gks.load_library()


def _hp(mode, tau_model, mu=2e-3, Pr=1.0, T_ref=T_REF, mu_pow=0.7, wall_u=None, wall_T=None,
        farfield=(1.0, 0.0, 0.0, 0.0, 1.0 / 1.4)):
    """Parameter vector of the host entries: gamma, mu, tau_eps, tau_C, flux_mode, tau_model, Pr,
    T_ref, mu_pow, wall_u[6][3], wall_T[6], farfield[6][5]."""
    wu = np.zeros(18) if wall_u is None else np.asarray(wall_u, dtype=np.float64).ravel()
    wT = np.zeros(6) if wall_T is None else np.asarray(wall_T, dtype=np.float64).ravel()
    ff = np.asarray(farfield, dtype=np.float64)
    ff = np.broadcast_to(ff, (6, 5)).ravel() if ff.size == 5 else ff.ravel()
    return np.concatenate([[1.4, mu, 0.01, 1.0, mode, tau_model, Pr, T_ref, mu_pow], wu, wT, ff])


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
    P = _hp(mode, tau_model)
    Po = oracle.params_vec(flux_mode=mode, tau_model=tau_model, mu=2e-3, T_ref=T_REF)
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
    P = _hp(mode, 2, mu=0.2)
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
    P = _hp(0, 2, mu=3e-3, Pr=0.72)
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
    P = _hp(mode, tau_model)
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
    P = _hp(mode, tau_model)
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


def _wall_params(rng, iso):
    uw = rng.normal(size=(6, 3)) * 0.3
    Tw = (0.6 + 0.5 * rng.random(6)) if iso else np.zeros(6)
    return uw, Tw


@pytest.mark.parametrize("code", [0, 4, 6, 8, 10, 11])
@pytest.mark.parametrize("iso", [False, True])
def test_wall_ghost_matches_oracle(lib, code, iso):
    """The kernels' Gauss-point ghost (codes: axis + 3 side, + 6 for no-slip) against the
    oracle's wall map, value and gradient."""
    rng = np.random.default_rng(400 + code + 20 * iso)
    uw, Tw = _wall_params(rng, iso)
    P = _hp(0, 2, wall_u=uw, wall_T=Tw)
    Po = oracle.params_vec(flux_mode=0, tau_model=2, mu=2e-3, wall_u=uw, wall_T=Tw)
    kind, plane = (2, code - 6) if code >= 6 else (1, code)
    for _ in range(4):
        v, g = _state(rng), rng.normal(size=(5, 3)) * 0.3
        vg, gg = np.zeros(5), np.zeros(15)
        lib.gks_wall_ghost_host(_d(P), code, _d(v), _d(g), vg.ctypes.data_as(D),
                                gg.ctypes.data_as(D), None, None, None, None)
        vo, go = oracle.wall_ghost(Po, kind, plane, v, g)
        np.testing.assert_allclose(vg, vo, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(gg.reshape(5, 3), go, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("code", [1, 7, 9, 12, 16])
@pytest.mark.parametrize("iso", [False, True])
def test_wall_ghost_vjp_matches_central_differences(lib, code, iso):
    """Slip, no-slip (adiabatic, isothermal) and far-field ghosts (codes 12 + plane; subsonic
    in- or outflow for these states)."""
    rng = np.random.default_rng(450 + code + 20 * iso)
    uw, Tw = _wall_params(rng, iso)
    finf = (1.1, 0.2, -0.15, 0.1, 0.8) if iso else (0.9, -0.3, 0.05, 0.2, 0.7)
    P = _hp(0, 2, wall_u=uw, wall_T=Tw, farfield=finf)
    v, g = _state(rng), rng.normal(size=15) * 0.3
    x = np.concatenate([v, g])

    def f(x):
        vg, gg = np.zeros(5), np.zeros(15)
        lib.gks_wall_ghost_host(_d(P), code, _d(x[:5]), _d(x[5:]), vg.ctypes.data_as(D),
                                gg.ctypes.data_as(D), None, None, None, None)
        return np.concatenate([vg, gg])

    y = rng.normal(size=20)
    vg, gg, gv, ga = np.zeros(5), np.zeros(15), np.zeros(5), np.zeros(15)
    lib.gks_wall_ghost_host(_d(P), code, _d(v), _d(g), vg.ctypes.data_as(D), gg.ctypes.data_as(D),
                            _d(y[:5]), _d(y[5:]), gv.ctypes.data_as(D), ga.ctypes.data_as(D))
    gx = np.concatenate([gv, ga])
    fd = np.array([y @ (f(x + h * e) - f(x - h * e)) / (2 * h)
                   for e, h in ((np.eye(20)[k], 1e-6 * max(1.0, abs(x[k]))) for k in range(20))])
    assert np.abs(gx - fd).max() < 1e-8 * max(1.0, np.abs(fd).max())


def test_wall_flux_fix(lib):
    """Slip: only the normal momentum passes; no-slip: no mass, and at an adiabatic wall the
    energy flux is U_w . F_m (the isothermal wall keeps it)."""
    rng = np.random.default_rng(480)
    uw, Tw = rng.normal(size=(6, 3)), np.array([0, 0.7, 0, 0, 0.9, 0])
    P = _hp(0, 2, wall_u=uw, wall_T=Tw)
    for code in range(12):
        acc = rng.normal(size=10)
        out = acc.copy()
        lib.gks_wall_flux_fix_host(_d(P), code, out.ctypes.data_as(D))
        ax, pl = code % 3, code % 6
        exp = acc.copy()
        exp[[0, 5]] = 0.0
        if code < 6:
            for v in range(1, 5):
                if v != 1 + ax:
                    exp[[v, 5 + v]] = 0.0
        elif Tw[pl] <= 0:
            exp[4], exp[9] = uw[pl] @ acc[1:4], uw[pl] @ acc[6:9]
        np.testing.assert_allclose(out, exp, rtol=1e-15, atol=1e-16)  # dot-product rounding


@pytest.mark.parametrize("code", [12, 13, 15, 17])
def test_farfield_ghost_matches_oracle(lib, code):
    """Far-field planes (codes 12 + axis + 3 side): the characteristic state against the
    oracle, subsonic in- and outflow and both supersonic limits."""
    rng = np.random.default_rng(500 + code)
    finf = (1.05, 0.25, -0.1, 0.08, 0.7)
    P = _hp(0, 2, farfield=finf)
    Po = oracle.params_vec(flux_mode=0, tau_model=2, mu=2e-3, farfield=finf)
    ax = code % 3
    sg = 1.0 if (code % 6) >= 3 else -1.0
    for mach_n in (-1.6, -0.5, 0.3, 0.8, 1.4):
        v = _state(rng)
        rho, U = v[0], v[1:4] / v[0]
        p = 0.4 * (v[4] - 0.5 * rho * U @ U)
        U[ax] = sg * mach_n * np.sqrt(1.4 * p / rho)
        v = np.array([rho, *(rho * U), p / 0.4 + 0.5 * rho * U @ U])
        g = rng.normal(size=(5, 3))
        vg, gg = np.zeros(5), np.zeros(15)
        lib.gks_wall_ghost_host(_d(P), code, _d(v), _d(g), vg.ctypes.data_as(D),
                                gg.ctypes.data_as(D), None, None, None, None)
        vo, go = oracle.wall_ghost(Po, 3, code - 12, v, g)
        np.testing.assert_allclose(vg, vo, rtol=1e-13, atol=1e-14)
        assert not gg.any() and not go.any()
