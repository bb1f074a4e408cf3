"""No-slip walls (adiabatic, isothermal, moving) and the power-law viscosity of Section 5 on the
GPU, through the C ABI, against the FP64 oracle on the same seeded inputs.

Bars as in the other parity tests: FP64 relative L2 1e-12, mixed mode 2e-4 for the residual;
the VJP by the dot-product identity against the oracle's dual-number JVP to 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL_L = 2e-4


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()


_cache = {}


def mesh_pair(n, layers, bc, lo=(0, 0, 0), hi=(1, 1, 1)):
    key = (n, layers, bc, lo, hi)
    if key not in _cache:
        m = I.layered_box_mesh(n, layers, lo=lo, hi=hi, bc=bc)
        _cache[key] = (m, oracle.Mesh(m))
    return _cache[key]


def lid_walls(T=None):
    """Lid-driven cavity walls: the upper y plane (axis 1, side 1: plane 4) moves along x and z;
    every wall isothermal at T (adiabatic for None)."""
    uw = np.zeros((6, 3))
    uw[4] = (0.2, 0.0, 0.05)
    Tw = np.zeros(6) if T is None else np.full(6, T)
    return uw, Tw


def cavity_state(om, seed, T=1.0 / 1.4):
    q = np.array([1.0, 0.0, 0.0, 0.0, T / 0.4])   # rho = 1, p = rho T
    return I.perturbed_state(np.tile(q[:, None], (1, om.n_cells)), seed=seed, amp=0.02)


CASES = {
    "viscous_adiabatic": (dict(flux_mode=1, tau_model=2, mu=2e-3), None),
    "viscous_isothermal": (dict(flux_mode=0, tau_model=2, mu=2e-3), 0.8),
    "power_law_isothermal": (dict(flux_mode=1, tau_model=3, mu=2e-3, T_ref=0.7, mu_pow=0.7), 0.75),
    "inviscid_adiabatic": (dict(flux_mode=1, tau_model=1), None),
}


@pytest.mark.parametrize("layers", ["hybrid8", "tet"])
@pytest.mark.parametrize("case", list(CASES))
def test_cavity_residual_matches_oracle(case, layers):
    m, om = mesh_pair(8, layers, (2, 2, 2))
    p, T = CASES[case]
    uw, Tw = lid_walls(T)
    Q = cavity_state(om, seed=50)
    Lo, Lto = om.residual(oracle.params_vec(wall_u=uw, wall_T=Tw, **p), Q, 0.004)
    S = gks.Solver(m, wall_u=uw, wall_T=Tw, **p)
    L, Lt = S.residual(Q, 0.004)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL
    Sm = gks.Solver(m, precision=gks.GKS_PREC_MIXED, wall_u=uw, wall_T=Tw, **p)
    Lm, _ = Sm.residual(Q, 0.004)
    assert rel(Lm.cpu(), Lo) < MIXED_TOL_L


def test_mixed_wall_kinds_and_moving_walls_match_oracle():
    """Periodic x, no-slip y (both planes moving, one isothermal), slip z: images reflected
    across a slip and a moving no-slip plane in either order."""
    m, om = mesh_pair(8, "hybrid8", (0, 2, 1))
    uw = np.zeros((6, 3))
    uw[1] = (-0.1, 0.0, 0.07)
    uw[4] = (0.15, 0.0, -0.05)
    Tw = np.array([0, 0, 0, 0, 0.8, 0])
    p = dict(flux_mode=1, tau_model=3, mu=3e-3, T_ref=0.7)
    Q = cavity_state(om, seed=51)
    Lo, Lto = om.residual(oracle.params_vec(wall_u=uw, wall_T=Tw, **p), Q, 0.004)
    for prec, tol in ((gks.GKS_PREC_FP64, FP64_TOL), (gks.GKS_PREC_MIXED, MIXED_TOL_L)):
        S = gks.Solver(m, precision=prec, wall_u=uw, wall_T=Tw, **p)
        L, Lt = S.residual(Q, 0.004)
        assert rel(L.cpu(), Lo) < tol
        if prec == gks.GKS_PREC_FP64:
            assert rel(Lt.cpu(), Lto) < tol


def test_cavity_steps_and_time_step_match_oracle():
    m, om = mesh_pair(8, "hybrid8", (2, 2, 2))
    p, T = CASES["power_law_isothermal"]
    uw, Tw = lid_walls(T)
    P = oracle.params_vec(wall_u=uw, wall_T=Tw, **p)
    Q = cavity_state(om, seed=52)
    S = gks.Solver(m, wall_u=uw, wall_T=Tw, **p)
    S.set_state(Q)
    dt = S.max_dt(0.4)
    dto = om.max_dt(P, Q, 0.4)
    assert abs(dt - dto) <= 1e-13 * dto
    S.step(dt, 3)
    Qo = om.step(P, Q, dt, 3)
    assert rel(S.get_state().cpu(), Qo) < FP64_TOL


def test_cavity_implicit_steps_match_oracle():
    m, om = mesh_pair(8, "hybrid8", (2, 2, 2))
    p, T = CASES["viscous_isothermal"]
    uw, Tw = lid_walls(T)
    P = oracle.params_vec(wall_u=uw, wall_T=Tw, **p)
    Q = cavity_state(om, seed=53)
    dt = 4.0 * om.max_dt(P, Q, 0.5)
    Qo = om.step_implicit(P, Q, dt, 2, 3)
    S = gks.Solver(m, wall_u=uw, wall_T=Tw, **p)
    S.set_state(Q)
    S.step_implicit(dt, 2, 3)
    assert rel(S.get_state().cpu(), Qo) < FP64_TOL
    Sm = gks.Solver(m, precision=gks.GKS_PREC_MIXED, wall_u=uw, wall_T=Tw, **p)
    Sm.set_state(Q)
    Sm.step_implicit(dt, 2, 3)
    # mixed mode: relative to the state change, the residual bar of the parity tests
    d = np.linalg.norm(Qo - Q)
    assert np.linalg.norm(Sm.get_state().cpu().numpy() - Qo) <= MIXED_TOL_L * d


@pytest.mark.parametrize("T", [None, 0.8])
def test_cavity_vjp_dot_product_with_oracle_jvp(T):
    m, om = mesh_pair(8, "hybrid8", (2, 2, 2))
    p = dict(flux_mode=1, tau_model=3, mu=2e-3, T_ref=0.7)
    uw, Tw = lid_walls(T)
    Q = cavity_state(om, seed=54)
    gL, gLt, dQ = I.normal_directions(Q.shape, 3, 55)
    S = gks.Solver(m, wall_u=uw, wall_T=Tw, **p)
    gQ = S.residual_vjp(Q, 0.004, gL, gLt).cpu().numpy()
    _, _, dL, dLt = om.residual_jvp(oracle.params_vec(wall_u=uw, wall_T=Tw, **p), Q, dQ, 0.004)
    lhs = (gQ * dQ).sum()
    rhs = (gL * dL).sum() + (gLt * dLt).sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


def test_gas_moving_with_the_walls_stays_uniform():
    """Walls at both y planes moving with a uniform gas (periodic x, z): the ghosts equal the gas,
    so steps leave it unchanged (to rounding) in both precisions."""
    m, om = mesh_pair(8, "hybrid8", (0, 2, 0))
    U = np.array([0.3, 0.0, -0.2])
    q = np.array([1.1, *(1.1 * U), 2.0 / 0.4 + 0.5 * 1.1 * U @ U])
    Q = np.tile(q[:, None], (1, om.n_cells))
    uw = np.zeros((6, 3))
    uw[1] = uw[4] = U
    for prec, tol in ((gks.GKS_PREC_FP64, 1e-13), (gks.GKS_PREC_MIXED, 1e-6)):
        S = gks.Solver(m, precision=prec, flux_mode=1, tau_model=2, mu=1e-3, wall_u=uw)
        S.set_state(Q)
        S.step(2e-3, 3)
        err = np.abs(S.get_state().cpu().numpy() - Q).max()
        assert err < tol * np.abs(Q).max(), err


def test_closed_noslip_box_conserves_mass_and_energy():
    """Stationary adiabatic no-slip walls: no mass and no energy crosses them (FP64 sums)."""
    m, om = mesh_pair(8, "hybrid8", (2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1))
    vol = torch.from_numpy(om.cell_info()["vol"]).cuda()
    Q = cavity_state(om, seed=56)
    for prec in (gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED):
        S = gks.Solver(m, precision=prec, flux_mode=1, tau_model=2, mu=1e-3)
        S.set_state(Q)
        S.step(S.max_dt(0.4), 4)
        tot0 = (torch.from_numpy(Q).cuda() * vol).sum(dim=1)
        tot1 = (S.get_state() * vol).sum(dim=1)
        for v in (0, 4):
            assert abs(float(tot1[v] - tot0[v])) <= 1e-12 * abs(float(tot0[v]))


# ------------------------------------------------------------------ far field (Riemann invariants)
FINF = (1.0, 0.3, -0.1, 0.05, 1.0 / 1.4)


def farfield_state(om, seed, finf=FINF):
    r, U, p = finf[0], np.array(finf[1:4]), finf[4]
    q = np.array([r, *(r * U), p / 0.4 + 0.5 * r * U @ U])
    return I.perturbed_state(np.tile(q[:, None], (1, om.n_cells)), seed=seed, amp=0.03)


@pytest.mark.parametrize("bc", [(3, 3, 3), (3, 1, 2)])
def test_farfield_residual_matches_oracle(bc):
    """Far-field planes (all six; or x far field with a slip y wall and a moving no-slip z wall):
    ghost cells reached across far-field planes are refreshed from the characteristic map."""
    m, om = mesh_pair(8, "hybrid8", bc)
    uw = np.zeros((6, 3))
    uw[5] = (0.1, -0.05, 0.0)
    p = dict(flux_mode=1, tau_model=2, mu=2e-3)
    Q = farfield_state(om, seed=60)
    Lo, Lto = om.residual(oracle.params_vec(wall_u=uw, farfield=FINF, **p), Q, 0.004)
    for prec, tol in ((gks.GKS_PREC_FP64, FP64_TOL), (gks.GKS_PREC_MIXED, MIXED_TOL_L)):
        S = gks.Solver(m, precision=prec, wall_u=uw, farfield=FINF, **p)
        L, Lt = S.residual(Q, 0.004)
        assert rel(L.cpu(), Lo) < tol
        if prec == gks.GKS_PREC_FP64:
            assert rel(Lt.cpu(), Lto) < tol


def test_farfield_steps_and_implicit_match_oracle():
    m, om = mesh_pair(8, "hybrid8", (3, 3, 3))
    p = dict(flux_mode=0, tau_model=2, mu=2e-3)
    P = oracle.params_vec(farfield=FINF, **p)
    Q = farfield_state(om, seed=61)
    S = gks.Solver(m, farfield=FINF, **p)
    S.set_state(Q)
    dt = S.max_dt(0.4)
    S.step(dt, 3)
    assert rel(S.get_state().cpu(), om.step(P, Q, dt, 3)) < FP64_TOL
    S.set_state(Q)
    S.step_implicit(4 * dt, 2, 3)
    assert rel(S.get_state().cpu(), om.step_implicit(P, Q, 4 * dt, 2, 3)) < FP64_TOL


@pytest.mark.parametrize("bc", [(3, 3, 3), (3, 1, 2)])
def test_farfield_vjp_dot_product_with_oracle_jvp(bc):
    """The VJP through far-field planes (the characteristic map at the Gauss points and in the
    stencil ghosts, reversed) against the oracle's dual-number directional derivative."""
    m, om = mesh_pair(8, "hybrid8", bc)
    uw = np.zeros((6, 3))
    uw[5] = (0.1, -0.05, 0.0)
    p = dict(flux_mode=1, tau_model=2, mu=2e-3)
    Q = farfield_state(om, seed=63)
    gL, gLt, dQ = I.normal_directions(Q.shape, 3, 64)
    S = gks.Solver(m, farfield=FINF, wall_u=uw, **p)
    gQ = S.residual_vjp(Q, 0.004, gL, gLt).cpu().numpy()
    _, _, dL, dLt = om.residual_jvp(oracle.params_vec(farfield=FINF, wall_u=uw, **p), Q, dQ, 0.004)
    lhs, rhs = (gQ * dQ).sum(), (gL * dL).sum() + (gLt * dLt).sum()
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


@pytest.mark.parametrize("finf", [FINF, (1.0, 1.6, 0.3, -0.2, 1.0 / 1.4)])
def test_farfield_box_keeps_the_free_stream(finf):
    m, om = mesh_pair(8, "hybrid8", (3, 3, 3))
    r, U, p = finf[0], np.array(finf[1:4]), finf[4]
    q = np.array([r, *(r * U), p / 0.4 + 0.5 * r * U @ U])
    Q = np.tile(q[:, None], (1, om.n_cells))
    for prec, tol in ((gks.GKS_PREC_FP64, 1e-13), (gks.GKS_PREC_MIXED, 1e-6)):
        S = gks.Solver(m, precision=prec, flux_mode=1, tau_model=1, farfield=finf)
        S.set_state(Q)
        S.step(2e-3, 3)
        err = np.abs(S.get_state().cpu().numpy() - Q).max()
        assert err < tol * np.abs(Q).max(), err


@pytest.mark.parametrize("layers", [("hex",) * 4, ("tet",) * 4, ("hex", "trans", "tet", "transm")])
def test_riemann_tube_with_farfield_ends_matches_oracle(layers):
    """The Riemann-problem setup of Section 5 at h = 1/40: [0,1] x [0,0.1] x [0,0.1], far-field
    x ends holding the left and right Lax states (one state per plane), slip y and z walls. The
    jump is smoothed over a few cells (tanh profile): the sharp jump reconstructs to negative
    pressure at Gauss points of the tetrahedral mesh (no limiter in the paper), which both sides
    report as non-physical."""
    m = I.layered_box_mesh(4, layers, lo=(0, 0, 0), hi=(1, 0.1, 0.1), bc=(3, 1, 1), jitter=0.05,
                           shape=(40, 4))
    om = oracle.Mesh(m)
    x = I.vertex_mean(m)
    wl = 0.5 * (1.0 - np.tanh((x[:, 0] - 0.5) / 0.05))   # 1 on the left, 0 on the right
    mix = lambda a, b: wl * a + (1.0 - wl) * b
    U0 = np.zeros((len(wl), 3))
    U0[:, 0] = mix(0.698, 0.0)
    Q = np.ascontiguousarray(I.primitive_to_conserved(mix(0.445, 0.5), U0, mix(3.528, 0.571)))
    far = np.tile(np.array([1.0, 0.0, 0.0, 0.0, 1.0]), (6, 1))
    far[0] = (0.445, 0.698, 0.0, 0.0, 3.528)
    far[3] = (0.5, 0.0, 0.0, 0.0, 0.571)
    p = dict(flux_mode=1, tau_model=1)
    P = oracle.params_vec(farfield=far, **p)
    Lo, Lto = om.residual(P, Q, 1e-3)
    S = gks.Solver(m, farfield=far, **p)
    L, Lt = S.residual(Q, 1e-3)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL
    S.set_state(Q)
    dt = S.max_dt(0.4)
    S.step(dt, 4)
    assert rel(S.get_state().cpu(), om.step(P, Q, dt, 4)) < FP64_TOL
