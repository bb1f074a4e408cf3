"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

FP64 mode must match to a relative L2 error of 1e-12 (the bar fixed for this path); mixed mode
(FP32 reconstruction and flux, FP64 sums and update) to the tolerances stated below, which
follow from FP32 rounding of the face states (relative 6e-8) amplified by the cancellation in
the face sums of a cell (flux / (h * dflux/dx), about 1e2-1e3 on these meshes).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL_L = 2e-4     # relative L2 of L in mixed mode
MIXED_TOL_STEP = 1e-7  # relative L2 of the state after steps in mixed mode

CASES = {
    "smooth_zero": dict(flux_mode=0, tau_model=0),
    "full_inviscid": dict(flux_mode=1, tau_model=1),
    "full_viscous": dict(flux_mode=1, tau_model=2, mu=1e-3),
    "smooth_viscous": dict(flux_mode=0, tau_model=2, mu=2e-3),
}


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


_mesh_cache = {}


def mesh_pair(n=8, layers="hybrid8", bc=(0, 0, 0), lo=(0, 0, 0), hi=(2, 2, 2), jitter=0.1):
    key = (n, layers, bc, lo, hi, jitter)
    if key not in _mesh_cache:
        m = I.layered_box_mesh(n, layers, lo=lo, hi=hi, bc=bc, jitter=jitter)
        _mesh_cache[key] = (m, oracle.Mesh(m))
    return _mesh_cache[key]


def smooth_state(m, om, seed=11, amp=0.02):
    return I.perturbed_state(om.advection_average(), seed=seed, amp=amp)


@pytest.mark.parametrize("case", list(CASES))
def test_residual_fp64_matches_oracle(case):
    m, om = mesh_pair()
    Q = smooth_state(m, om)
    dt = 0.01
    S = gks.Solver(m, **CASES[case])
    L, Lt = S.residual(Q, dt)
    Lo, Lto = om.residual(oracle.params_vec(**CASES[case]), Q, dt)
    assert rel(L.cpu(), Lo) < FP64_TOL
    assert rel(Lt.cpu(), Lto) < FP64_TOL


@pytest.mark.parametrize("layers", ["hex", "tet", "prism", ("trans", "transm") * 2])
def test_residual_fp64_single_kind_meshes(layers):
    m, om = mesh_pair(4, layers)
    Q = smooth_state(m, om, seed=12)
    p = CASES["full_viscous"]
    S = gks.Solver(m, **p)
    L, Lt = S.residual(Q, 0.01)
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.01)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL


def test_residual_fp64_reflecting_box():
    m, om = mesh_pair(8, "hybrid8", bc=(1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1))
    q = np.array([0.8, 0.0, 0.0, 0.0, 1.1 / 0.4])
    Q = I.perturbed_state(np.tile(q[:, None], (1, om.n_cells)), seed=13, amp=0.01)
    p = CASES["full_inviscid"]
    S = gks.Solver(m, **p)
    L, Lt = S.residual(Q, 0.004)
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.004)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL


def test_residual_fp64_taylor_green_prandtl():
    """Navier-Stokes with the Prandtl-number correction (Pr = 0.72) on the Taylor-Green layer
    pattern, [0, 2 pi]^3."""
    m, om = mesh_pair(8, "tgv48", lo=(0, 0, 0), hi=(2 * np.pi,) * 3)
    Q = I.perturbed_state(I.taylor_green_state(m), seed=15, amp=0.01)
    p = dict(flux_mode=0, tau_model=2, mu=1.0 / 1600.0, Pr=0.72)
    S = gks.Solver(m, **p)
    L, Lt = S.residual(Q, 0.02)
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.02)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL
    Sm = gks.Solver(m, precision=gks.GKS_PREC_MIXED, **p)
    Lm, _ = Sm.residual(Q, 0.02)
    assert rel(Lm.cpu(), Lo) < MIXED_TOL_L


def test_residual_fp64_mixed_boundaries():
    m, om = mesh_pair(8, "hybrid8", bc=(0, 1, 0))
    Q = smooth_state(m, om, seed=14)
    p = CASES["full_viscous"]
    S = gks.Solver(m, **p)
    L, Lt = S.residual(Q, 0.01)
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.01)
    assert rel(L.cpu(), Lo) < FP64_TOL and rel(Lt.cpu(), Lto) < FP64_TOL


@pytest.mark.parametrize("case", ["smooth_zero", "full_inviscid"])
def test_step_fp64_matches_oracle(case):
    m, om = mesh_pair()
    Q = om.advection_average()
    p = CASES[case]
    dt = om.max_dt(oracle.params_vec(**p), Q, 0.5)
    S = gks.Solver(m, **p)
    S.set_state(Q)
    assert abs(S.max_dt(0.5) - dt) <= 1e-14 * dt
    S.step(dt, 3)
    Qo = om.step(oracle.params_vec(**p), Q, dt, 3)
    assert rel(S.get_state().cpu(), Qo) < FP64_TOL


@pytest.mark.parametrize("case", ["smooth_zero", "full_viscous"])
def test_residual_mixed_within_stated_tolerance(case):
    m, om = mesh_pair()
    Q = smooth_state(m, om)
    p = CASES[case]
    S = gks.Solver(m, precision=gks.GKS_PREC_MIXED, **p)
    L, Lt = S.residual(Q, 0.01)
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.01)
    assert rel(L.cpu(), Lo) < MIXED_TOL_L
    assert rel(Lt.cpu(), Lto) < 10 * MIXED_TOL_L


def test_step_mixed_within_stated_tolerance():
    m, om = mesh_pair()
    Q = om.advection_average()
    p = CASES["smooth_zero"]
    dt = om.max_dt(oracle.params_vec(**p), Q, 0.5)
    S = gks.Solver(m, precision=gks.GKS_PREC_MIXED, **p)
    S.set_state(Q)
    S.step(dt, 3)
    Qo = om.step(oracle.params_vec(**p), Q, dt, 3)
    assert rel(S.get_state().cpu(), Qo) < MIXED_TOL_STEP


def test_deterministic_and_conservative():
    m, om = mesh_pair()
    Q = smooth_state(m, om)
    S = gks.Solver(m, **CASES["full_viscous"])
    L1, Lt1 = S.residual(Q, 0.01)
    L2, Lt2 = S.residual(Q, 0.01)
    assert torch.equal(L1, L2) and torch.equal(Lt1, Lt2)
    vol = om.cell_info()["vol"]
    assert np.abs(L1.cpu().numpy() @ vol).max() < 1e-13


def test_free_stream_on_gpu():
    m, om = mesh_pair()
    q = np.array([1.2, 0.3, -0.5, 0.7, 2.5 / 0.4 + 0.5 * (0.09 + 0.25 + 0.49) / 1.2])
    Q = np.tile(q[:, None], (1, om.n_cells))
    for prec in (gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED):
        S = gks.Solver(m, precision=prec, **CASES["full_inviscid"])
        S.set_state(Q)
        S.step(0.01, 2)
        tol = 1e-13 if prec == gks.GKS_PREC_FP64 else 1e-5
        assert np.abs(S.get_state().cpu().numpy() - Q).max() < tol


def test_nonphysical_state_reports_error():
    m, om = mesh_pair()
    Q = smooth_state(m, om)
    Q[0, 17] = -1.0
    S = gks.Solver(m)
    with pytest.raises(gks.GksError) as e:
        S.residual(Q, 0.01)
    assert e.value.status == gks.GKS_E_NONPHYSICAL
    # the solver stays usable afterwards
    L, _ = S.residual(smooth_state(m, om), 0.01)
    assert torch.isfinite(L).all()


def test_host_buffers_through_abi():
    """gks_residual takes host pointers as well (copies are part of the call)."""
    m, om = mesh_pair()
    Q = np.ascontiguousarray(smooth_state(m, om))
    S = gks.Solver(m)
    L = np.zeros_like(Q)
    Lt = np.zeros_like(Q)
    gks.gks_residual(S.h, Q, 0.01, L, Lt)
    Ld, Ltd = S.residual(Q, 0.01)
    assert np.array_equal(L, Ld.cpu().numpy()) and np.array_equal(Lt, Ltd.cpu().numpy())
