"""Pins of the oracle's viscous extras (Section 5): the power-law viscosity mu(T) of Section 5.4
and the wall conditions the paper's cases use (slip walls, no-slip adiabatic and isothermal
walls, moving walls).

The paper gives no formulas for the walls. The pins check what any reading must satisfy: data
that continue smoothly through the wall make the ghost pair continuous, so the Gauss-point flux
is the Navier-Stokes flux of the BGK model (Chapman-Enskog); a gas at rest, or moving with the
walls, stays so; closed boxes keep their mass (and, with adiabatic stationary walls, their
energy); a linear shear flow over a stationary wall has the exact viscous residual.
"""
import numpy as np
import pytest

import oracle
from paper_2203_09047_gb300 import inputs as I
from test_oracle_pins import GAMMA, _fit, _ns_flux, _random_state


@pytest.mark.parametrize("mode", [0, 1])
def test_power_law_flux_is_chapman_enskog(mode):
    """tau = mu (T0/T_ref)^0.7 / p0: with continuous data the flux is the Navier-Stokes flux with
    the viscosity of the state's temperature T = p / rho (Section 5.4)."""
    rng = np.random.default_rng(60 + mode)
    mu, T_ref = 3e-3, 0.6
    P = oracle.params_vec(flux_mode=mode, tau_model=3, mu=mu, T_ref=T_ref, mu_pow=0.7)
    for _ in range(5):
        q = _random_state(rng)
        dq = rng.normal(size=(3, 5)) * 0.2
        p = (GAMMA - 1) * (q[4] - 0.5 * q[1:4] @ q[1:4] / q[0])
        muT = mu * (p / q[0] / T_ref) ** 0.7
        Fn, _ = _fit(oracle.gp_flux(P, q, dq, q, dq, 1e-3), 1e-3)
        np.testing.assert_allclose(Fn, _ns_flux(q, dq, muT), rtol=1e-11, atol=1e-12)


def test_power_law_with_zero_exponent_is_constant_viscosity():
    rng = np.random.default_rng(62)
    for mode in (0, 1):
        P3 = oracle.params_vec(flux_mode=mode, tau_model=3, mu=2e-3, T_ref=0.3, mu_pow=0.0)
        P2 = oracle.params_vec(flux_mode=mode, tau_model=2, mu=2e-3)
        for _ in range(3):
            ql, qr = _random_state(rng), _random_state(rng)
            dql, dqr = rng.normal(size=(3, 5)) * 0.2, rng.normal(size=(3, 5)) * 0.2
            np.testing.assert_array_equal(oracle.gp_flux(P3, ql, dql, qr, dqr, 1e-3),
                                          oracle.gp_flux(P2, ql, dql, qr, dqr, 1e-3))


def _conservative(rho, U, T, grho, gU, gT):
    """State and gradient [5][3] (d/dx_b) from primitives rho, U, T = p / rho and theirs."""
    p = rho * T
    q = np.array([rho, *(rho * U), p / (GAMMA - 1) + 0.5 * rho * U @ U])
    g = np.zeros((5, 3))
    gp = T * grho + rho * gT
    g[0] = grho
    for j in range(3):
        g[1 + j] = U[j] * grho + rho * gU[j]
    g[4] = gp / (GAMMA - 1) + 0.5 * (U @ U) * grho + rho * (U @ gU)
    return q, g


def _local(q, g, n1):
    """Rotate into a frame whose first axis is n1: state and dq[d][v] along n_d."""
    e = np.zeros(3)
    e[np.argmin(np.abs(n1))] = 1.0
    n2 = np.cross(n1, e)
    n2 /= np.linalg.norm(n2)
    n3 = np.cross(n1, n2)
    R = np.array([n1, n2, n3])
    ql = np.array([q[0], *(R @ q[1:4]), q[4]])
    gl = np.zeros((5, 3))
    gl[0], gl[4] = g[0], g[4]
    gl[1:4] = R @ g[1:4]       # rotate the momentum components
    return ql, (gl @ R.T).T    # derivatives along n_d


@pytest.mark.parametrize("kind,iso", [(1, False), (2, False), (2, True)])
@pytest.mark.parametrize("plane", [1, 3, 5])
def test_wall_ghost_of_continuable_data_gives_navier_stokes_flux(kind, iso, plane):
    """Data that satisfy the wall's conditions and continue smoothly through it (slip: U_n = 0
    with no normal derivative of rho, p and U_t and no tangential one of U_n; no-slip: U = U_w
    with no tangential derivative of U; adiabatic: no normal derivative of T; isothermal: T = T_w
    with no tangential derivative of T; no normal derivative of rho): the ghost continues them,
    so the Gauss-point flux along the outward normal is the Navier-Stokes flux."""
    rng = np.random.default_rng(70 + 10 * kind + plane + 5 * iso)
    ax, side = plane % 3, plane // 3
    n1 = np.zeros(3)
    n1[ax] = 1.0 if side else -1.0
    tang = [b for b in range(3) if b != ax]
    uw = np.zeros((6, 3))
    Tw = np.zeros(6)
    Uw = np.zeros(3)
    if kind == 2:
        Uw[tang] = rng.normal(size=2) * 0.4
        uw[plane] = Uw
    T = 0.5 + 0.5 * rng.random()
    if iso:
        Tw[plane] = T
    mu = 3e-3
    for _ in range(4):
        rho = 1.0 + 0.3 * rng.random()
        grho, gT, gU = rng.normal(size=3) * 0.3, rng.normal(size=3) * 0.3, np.zeros((3, 3))
        grho[ax] = 0.0
        if kind == 1:
            U = rng.normal(size=3) * 0.5
            U[ax] = 0.0
            gU[:, ax] = rng.normal(size=3) * 0.3   # d/dn of every component
            gU[tang, ax] = 0.0                     # ... but no normal derivative of U_t
            gU[ax, tang] = 0.0                     # no tangential derivative of U_n
            gU[np.ix_(tang, tang)] = rng.normal(size=(2, 2)) * 0.3
            gT[ax] = 0.0
        else:
            U = Uw.copy()
            gU[:, ax] = rng.normal(size=3) * 0.3   # only normal derivatives of U
            if iso:
                gT[tang] = 0.0
            else:
                gT[ax] = 0.0
        q, g = _conservative(rho, U, T, grho, gU, gT)
        P = oracle.params_vec(flux_mode=0, tau_model=2, mu=mu, wall_u=uw, wall_T=Tw)
        qg, gg = oracle.wall_ghost(P, kind, plane, q, g)
        ql, dql = _local(q, g, n1)
        qr, dqr = _local(qg, gg, n1)
        np.testing.assert_allclose(qr, ql, rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(dqr, dql, rtol=1e-12, atol=1e-13)
        Fn, _ = _fit(oracle.gp_flux(P, ql, dql, qr, dqr, 1e-3), 1e-3)
        np.testing.assert_allclose(Fn, _ns_flux(ql, dql, mu), rtol=1e-11, atol=1e-12)


def _box(bc, n=8, lo=(0, 0, 0), hi=(1, 1, 1), layers="hybrid8", jitter=0.1):
    m = I.layered_box_mesh(n, layers, lo=lo, hi=hi, bc=bc, jitter=jitter)
    return m, oracle.Mesh(m)


@pytest.fixture(scope="module")
def noslip_box():
    return _box((2, 2, 2), lo=(-1, -1, -1), hi=(1, 1, 1))


def test_noslip_box_rest_and_conservation(noslip_box):
    m, om = noslip_box
    vol = om.cell_info()["vol"]
    q0 = np.array([0.8, 0, 0, 0, 1.1 / 0.4])
    Qrest = np.tile(q0[:, None], (1, om.n_cells))
    T0 = 1.1 / 0.8
    for Tw in (0.0, T0):   # adiabatic, and isothermal at the gas temperature
        P = oracle.params_vec(flux_mode=1, tau_model=2, mu=1e-3, wall_T=np.full(6, Tw))
        L, Lt = om.residual(P, Qrest, 0.01)
        assert np.abs(L).max() < 1e-12 and np.abs(Lt).max() < 1e-10
    # stationary adiabatic walls: no mass and no energy crosses them
    Q = I.perturbed_state(Qrest, seed=6, amp=0.01)
    P = oracle.params_vec(flux_mode=1, tau_model=2, mu=1e-3)
    L, Lt = om.residual(P, Q, 0.002)
    assert abs(L[0] @ vol) < 1e-13 and abs(L[4] @ vol) < 1e-13
    assert abs(Lt[0] @ vol) < 1e-11 and abs(Lt[4] @ vol) < 1e-11


def test_isothermal_walls_heat_or_cool_and_keep_mass(noslip_box):
    m, om = noslip_box
    vol = om.cell_info()["vol"]
    Q = np.tile(np.array([0.8, 0, 0, 0, 1.1 / 0.4])[:, None], (1, om.n_cells))
    T0 = 1.1 / 0.8
    rates = []
    for Tw in (1.2 * T0, 0.8 * T0):
        P = oracle.params_vec(flux_mode=0, tau_model=2, mu=1e-2, wall_T=np.full(6, Tw))
        L, _ = om.residual(P, Q, 0.002)
        assert abs(L[0] @ vol) < 1e-13
        rates.append(L[4] @ vol)
    assert rates[0] > 0 > rates[1]


def test_walls_moving_with_the_gas_leave_it_unchanged():
    """Periodic in x and z, no-slip walls at both y planes moving with the gas: the ghost equals
    the gas, so a uniform moving state is steady (Galilean check of U_g = 2 U_w - U)."""
    m, om = _box((0, 2, 0))
    Uw = np.array([0.3, 0.0, -0.2])
    q = np.array([1.1, *(1.1 * Uw), 2.0 / 0.4 + 0.5 * 1.1 * Uw @ Uw])
    Q = np.tile(q[:, None], (1, om.n_cells))
    uw = np.zeros((6, 3))
    uw[1] = uw[4] = Uw
    for Tw in (0.0, 2.0 / 1.1):
        P = oracle.params_vec(flux_mode=1, tau_model=3, mu=1e-3, T_ref=1.0, wall_u=uw,
                              wall_T=np.full(6, Tw))
        L, _ = om.residual(P, Q, 0.01)
        assert np.abs(L).max() < 1e-12


def test_moving_lid_drags_the_gas():
    m, om = _box((2, 2, 2))
    vol = om.cell_info()["vol"]
    Q = np.tile(np.array([1.0, 0, 0, 0, 1.0 / 1.4 / 0.4])[:, None], (1, om.n_cells))
    uw = np.zeros((6, 3))
    uw[4] = (0.15, 0.0, 0.0)   # the upper y plane
    P = oracle.params_vec(flux_mode=1, tau_model=2, mu=1e-3, wall_u=uw)
    L, _ = om.residual(P, Q, 0.005)
    assert abs(L[0] @ vol) < 1e-13
    assert L[1] @ vol > 0 and L[4] @ vol > 0   # x momentum and the lid's work enter the gas


@pytest.mark.parametrize("tau_model", [2, 3])
@pytest.mark.parametrize("layers,jitter", [("hex", 0.0), ("tet", 0.1)])
def test_linear_shear_over_a_stationary_wall_has_the_exact_viscous_residual(tau_model, layers,
                                                                             jitter):
    """U = a (y - y0) over a no-slip wall at y0 with uniform rho and p (periodic in x and z, plain
    quadratic reconstruction): the reconstruction is exact (the ghosts continue U oddly and rho,
    E evenly), the wall pair is continuous and every flux is the Navier-Stokes one, so the cells
    away from the upper wall have L = (0, 0, 0, 0, mu a^2): no net force, viscous heating
    mu a^2. The convective energy flux (E + p) U . n is cubic along a face; the 2x2 Gauss rule
    integrates it exactly on the parallelogram faces of unjittered hexahedra only, so on
    jittered tetrahedra the energy check is loose and mass and momentum carry the pin."""
    m, om = _box((0, 2, 0), n=8, layers=layers, jitter=jitter)
    y = om.cell_info()["centroid"][:, 1]
    a, rho, p, mu, T_ref = 0.4, 1.0, 1.0, 2e-3, 0.8
    # cell averages (27-point quadrature, exact for these quadratics) of rho, m_x = rho a y and
    # E = p/(g-1) + rho a^2 y^2 / 2, the wall at y0 = 0; monomials 1 x y z xx yy zz xy xz yz
    c = np.zeros((5, 10))
    c[0, 0] = rho
    c[1, 2] = rho * a
    c[4, 0] = p / (GAMMA - 1)
    c[4, 5] = 0.5 * rho * a * a
    Q = om.cell_average(1, 0.0, c.ravel())
    muT = mu * (p / rho / T_ref) ** 0.7 if tau_model == 3 else mu
    P = oracle.params_vec(flux_mode=0, tau_model=tau_model, mu=mu, T_ref=T_ref, weno_linear=1)
    L, _ = om.residual(P, Q, 1e-3)
    sel = y < 0.45   # stencils reach about 2.5 cells, short of the upper wall
    assert sel.sum() > 100
    np.testing.assert_allclose(L[:4, sel], 0.0, atol=1e-12)
    np.testing.assert_allclose(L[4, sel], muT * a * a, rtol=1e-9 if jitter == 0 else 0.15)


# ------------------------------------------------------------------ far field (Riemann invariants)
def _prim(q, gamma=GAMMA):
    rho = q[0]
    U = q[1:4] / rho
    p = (gamma - 1) * (q[4] - 0.5 * rho * U @ U)
    return rho, U, p, np.sqrt(gamma * p / rho)


def _cons(rho, U, p, gamma=GAMMA):
    return np.array([rho, *(rho * U), p / (gamma - 1) + 0.5 * rho * U @ U])


FINF = (1.0, 0.3, -0.1, 0.05, 1.0 / GAMMA)   # rho, U, V, W, p: Mach 0.33


@pytest.mark.parametrize("plane", [0, 1, 3, 5])
def test_farfield_state_keeps_the_invariants(plane):
    """Subsonic boundaries: the ghost carries the interior's outgoing invariant
    R+ = u_n + 2c/(gamma-1) and the far field's incoming R- = u_n - 2c/(gamma-1) (n outward), and
    the entropy p/rho^gamma and tangential velocity of the side the flow comes from; supersonic
    outflow keeps the interior, supersonic inflow takes the far field; the far-field state is a
    fixed point; the ghost has no gradient."""
    rng = np.random.default_rng(90 + plane)
    ax = plane % 3
    n = np.zeros(3)
    n[ax] = 1.0 if plane >= 3 else -1.0
    P = oracle.params_vec(farfield=FINF)
    qinf = _cons(FINF[0], np.array(FINF[1:4]), FINF[4])
    g0 = rng.normal(size=(5, 3))
    qg, gg = oracle.wall_ghost(P, 3, plane, qinf, g0)
    np.testing.assert_allclose(qg, qinf, rtol=1e-14, atol=1e-15)
    assert not gg.any()
    ri, Ui, pi_, ci = _prim(qinf)
    k = 2 / (GAMMA - 1)
    for _ in range(6):
        rho = 0.8 + 0.4 * rng.random()
        p = 0.5 + 0.5 * rng.random()
        c = np.sqrt(GAMMA * p / rho)
        U = rng.normal(size=3) * 0.3
        un = rng.uniform(-0.9, 0.9) * c
        U += (un - U @ n) * n
        q = _cons(rho, U, p)
        qg, _ = oracle.wall_ghost(P, 3, plane, q, g0)
        rb, Ub, pb, cb = _prim(qg)
        unb = Ub @ n
        np.testing.assert_allclose(unb + k * cb, un + k * c, rtol=1e-13)
        np.testing.assert_allclose(unb - k * cb, Ui @ n - k * ci, rtol=1e-13, atol=1e-14)
        src_rho, src_U, src_p = (rho, U, p) if unb >= 0 else (ri, Ui, pi_)
        np.testing.assert_allclose(pb / rb ** GAMMA, src_p / src_rho ** GAMMA, rtol=1e-12)
        np.testing.assert_allclose(Ub - unb * n, src_U - (src_U @ n) * n, atol=1e-13)
    for sign in (1.0, -1.0):   # supersonic out- and inflow
        rho, p = 1.1, 0.6
        U = rng.normal(size=3) * 0.2
        U += (sign * 1.5 * np.sqrt(GAMMA * p / rho) - U @ n) * n
        q = _cons(rho, U, p)
        qg, _ = oracle.wall_ghost(P, 3, plane, q, g0)
        np.testing.assert_allclose(qg, q if sign > 0 else qinf, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("bc,finf", [((3, 3, 3), FINF), ((3, 3, 3), (1.0, 1.6, 0.3, -0.2, 1.0 / GAMMA)),
                                     ((3, 1, 0), (1.2, 0.4, 0.0, 0.1, 0.9))])
def test_farfield_box_preserves_the_free_stream(bc, finf):
    """A uniform flow equal to the far field (subsonic and supersonic through all six planes;
    with a slip wall along it) is a steady state: every ghost equals the flow."""
    m, om = _box(bc)
    q = _cons(finf[0], np.array(finf[1:4]), finf[4])
    Q = np.tile(q[:, None], (1, om.n_cells))
    for mode, tau in ((0, 0), (1, 2)):
        P = oracle.params_vec(flux_mode=mode, tau_model=tau, mu=1e-3, farfield=finf)
        L, Lt = om.residual(P, Q, 0.005)
        assert np.abs(L).max() < 1e-12 and np.abs(Lt).max() < 1e-9
