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


def test_step_mixed_fp64_update_mode():
    """GKS_PREC_MIXED_FP64UPD: FP32 reconstruction and flux, FP64 face sums and FP64 update of an
    FP64 state. Within the mixed step tolerance of the oracle, conservative to FP64 round-off,
    and an implicit step in between hands its state on to the explicit steps."""
    m, om = mesh_pair()
    Q = om.advection_average()
    p = CASES["smooth_zero"]
    dt = om.max_dt(oracle.params_vec(**p), Q, 0.5)
    S = gks.Solver(m, precision=gks.GKS_PREC_MIXED_FP64UPD, **p)
    S.set_state(Q)
    S.step(dt, 3)
    Qo = om.step(oracle.params_vec(**p), Q, dt, 3)
    Qg = S.get_state().cpu().numpy()
    assert rel(Qg, Qo) < MIXED_TOL_STEP
    vol = om.cell_info()["vol"]
    for v in range(5):
        assert abs(vol @ Qg[v] - vol @ Q[v]) <= 1e-14 * np.abs(vol @ np.abs(Q[v]))
    # an implicit step (it updates the float-pair copy) followed directly by an explicit step
    # must start the explicit step from the implicit step's result; R reads the state out in
    # between, which refreshes the FP64 state on the host call
    S.step_implicit(dt, 1, 3)
    S.step(dt, 1)
    R = gks.Solver(m, precision=gks.GKS_PREC_MIXED_FP64UPD, **p)
    R.set_state(torch.from_numpy(Qg).cuda())
    R.step_implicit(dt, 1, 3)
    R.get_state()
    R.step(dt, 1)
    assert torch.equal(S.get_state(), R.get_state())


def test_s2o4_stage_calls_match_oracle_and_transpose():
    """gks_s2o4_stage against the oracle's two-stage combinations (Section 3.3), and
    gks_s2o4_stage_vjp as its exact transpose (dot-product identity)."""
    rng = np.random.default_rng(51)
    n = 5 * 1000 + 7
    Q, L, Lt, Lts = (rng.normal(size=n) for _ in range(4))
    dt = 0.013
    Qs_o, Qn_o = oracle.s2o4(Q, L, Lt, Lts, dt)
    d = [torch.from_numpy(a).cuda() for a in (Q, L, Lt, Lts)]
    out1, out2 = torch.empty_like(d[0]), torch.empty_like(d[0])
    s = torch.cuda.current_stream().cuda_stream
    gks.gks_s2o4_stage(1, dt, d[0], d[1], d[2], None, out1, s)
    gks.gks_s2o4_stage(2, dt, d[0], d[1], d[2], d[3], out2, s)
    assert rel(out1.cpu(), Qs_o) < 1e-15 and rel(out2.cpu(), Qn_o) < 1e-15
    g = torch.from_numpy(rng.normal(size=n)).cuda()
    for stage, out in ((1, out1), (2, out2)):
        gs = [torch.empty_like(g) for _ in range(4)]
        gks.gks_s2o4_stage_vjp(stage, dt, g, gs[0], gs[1], gs[2], gs[3] if stage == 2 else None, s)
        lhs = float((g * out).sum())
        rhs = sum(float((gs[k] * d[k]).sum()) for k in range(3 if stage == 1 else 4))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    with pytest.raises(gks.GksError):
        gks.gks_s2o4_stage(3, dt, d[0], d[1], d[2], d[3], out1, s)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_enlarged_stencils_match_oracle(bc):
    """min_stencil = 18 (the third-ring reading of gks_mesh_options) on the hybrid generator:
    the GPU path and the oracle take the same members; FP64 at 1e-12, mixed at MIXED_TOL_L."""
    lo, hi = ((0, 0, 0), (2, 2, 2)) if bc[0] == 0 else ((-1, -1, -1), (1, 1, 1))
    m = I.layered_box_mesh(8, "hybrid8", lo=lo, hi=hi, bc=bc)
    om = oracle.Mesh(m, min_stencil=18)
    Q = I.perturbed_state(oracle.Mesh(m).advection_average() if bc[0] == 0 else
                          np.tile(np.array([[0.8], [0.0], [0.0], [0.0], [1.1 / 0.4]]),
                                  (1, om.n_cells)), seed=16, amp=0.02)
    p = CASES["full_viscous"]
    Lo, Lto = om.residual(oracle.params_vec(**p), Q, 0.01)
    for prec, tol in ((gks.GKS_PREC_FP64, FP64_TOL), (gks.GKS_PREC_MIXED, MIXED_TOL_L)):
        S = gks.Solver(m, min_stencil=18, precision=prec, **p)
        L, Lt = S.residual(Q, 0.01)
        assert rel(L.cpu(), Lo) < tol and rel(Lt.cpu(), Lto) < 10 * tol, (prec, rel(L.cpu(), Lo))
        S.close()


def test_cell_order_leaves_results_bitwise():
    """Every cell's arithmetic runs in its own fixed face and stencil order, so the internal
    cell order (caller order, Morton, reverse Cuthill-McKee) changes no bit of the results."""
    m, om = mesh_pair()
    Q = smooth_state(m, om, seed=17)
    p = CASES["full_viscous"]
    out = []
    for reorder in (gks.GKS_REORDER_NONE, gks.GKS_REORDER_MORTON, gks.GKS_REORDER_RCM):
        S = gks.Solver(m, reorder=reorder, **p)
        L, Lt = S.residual(Q, 0.01)
        S.set_state(Q)
        S.step(0.004, 2)
        out.append((L, Lt, S.get_state()))
        S.close()
    for k in (1, 2):
        assert all(torch.equal(a, b) for a, b in zip(out[0], out[k]))


@pytest.mark.parametrize("prec", [gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED, gks.GKS_PREC_MIXED_FP64UPD])
def test_checkpoint_and_resume(prec):
    """The state (Q, t, step) is the whole checkpoint: reading it out after k steps and setting
    it into a fresh solver continues bit for bit like the uninterrupted run when the state is
    FP64. The mixed path's float-float state has up to 48 significant bits spread over more than
    53 when the low part is small, so its FP64 form can round it: the resumed run then agrees to
    the mixed path's own step tolerance, and a checkpoint that round-trips exactly (set, get)
    resumes identically from there on."""
    m, om = mesh_pair()
    Q = smooth_state(m, om, seed=18)
    p = CASES["full_viscous"]
    dt = 0.004
    A = gks.Solver(m, precision=prec, **p)
    A.set_state(Q)
    A.step(dt, 5)
    ref = A.get_state()
    B = gks.Solver(m, precision=prec, **p)
    B.set_state(Q)
    B.step(dt, 2)
    ckpt = B.get_state().cpu().numpy()
    B.close()
    C = gks.Solver(m, precision=prec, **p)
    C.set_state(ckpt)
    C.step(dt, 3)
    if prec == gks.GKS_PREC_MIXED:
        assert rel(C.get_state().cpu(), ref.cpu()) < MIXED_TOL_STEP
        # from a state that is its own FP64 form, two solvers resume identically
        q1 = C.get_state().cpu().numpy()
        D, E = (gks.Solver(m, precision=prec, **p) for _ in range(2))
        for X in (D, E):
            X.set_state(q1)
            X.step(dt, 2)
        assert torch.equal(D.get_state(), E.get_state())
        D.close()
        E.close()
    else:
        assert torch.equal(C.get_state(), ref)
    A.close()
    C.close()
