"""The residual's vector-Jacobian product (gks_residual_vjp) on the GPU.

Checked by the dot-product identity <gQ, dQ> = <gL, dL> + <gLt, dLt> against the oracle's
forward-mode (dual-number) directional derivatives, against central differences of the GPU
residual, and through a checkpointed S2O4 rollout against central differences.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

CASES = {
    "smooth_zero": dict(flux_mode=0, tau_model=0),
    "full_zero": dict(flux_mode=1, tau_model=0),
    "full_inviscid": dict(flux_mode=1, tau_model=1),
    "full_viscous": dict(flux_mode=1, tau_model=2, mu=1e-3),
    "smooth_viscous": dict(flux_mode=0, tau_model=2, mu=2e-3),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()


_cache = {}


def mesh_pair(n=8, layers="hybrid8", bc=(0, 0, 0), lo=(0, 0, 0), hi=(2, 2, 2)):
    key = (n, layers, bc, lo, hi)
    if key not in _cache:
        m = I.layered_box_mesh(n, layers, lo=lo, hi=hi, bc=bc)
        _cache[key] = (m, oracle.Mesh(m))
    return _cache[key]


def _dot_test(m, om, Q, params, dt, seed):
    gL, gLt, dQ = I.normal_directions(Q.shape, 3, seed)
    S = gks.Solver(m, **params)
    gQ = S.residual_vjp(Q, dt, gL, gLt).cpu().numpy()
    _, _, dL, dLt = om.residual_jvp(oracle.params_vec(**params), Q, dQ, dt)
    lhs = (gQ * dQ).sum()
    rhs = (gL * dL).sum() + (gLt * dLt).sum()
    return lhs, rhs


@pytest.mark.parametrize("case", list(CASES))
def test_vjp_dot_product_with_oracle_jvp(case):
    m, om = mesh_pair()
    Q = I.perturbed_state(om.advection_average(), seed=31, amp=0.02)
    lhs, rhs = _dot_test(m, om, Q, CASES[case], 0.01, seed=32)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


def test_vjp_dot_product_reflecting_box():
    m, om = mesh_pair(8, "hybrid8", bc=(1, 1, 1), lo=(-1, -1, -1), hi=(1, 1, 1))
    q = np.array([0.8, 0.1, -0.05, 0.02, 1.1 / 0.4])
    Q = I.perturbed_state(np.tile(q[:, None], (1, om.n_cells)), seed=33, amp=0.02)
    lhs, rhs = _dot_test(m, om, Q, CASES["full_viscous"], 0.004, seed=34)
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs), (lhs, rhs)


def test_vjp_against_central_differences_and_deterministic():
    m, om = mesh_pair()
    Q = I.perturbed_state(om.advection_average(), seed=35, amp=0.02)
    p = CASES["full_viscous"]
    gL, gLt, d = I.normal_directions(Q.shape, 3, 36)
    S = gks.Solver(m, **p)
    gQ1 = S.residual_vjp(Q, 0.01, gL, gLt)
    gQ2 = S.residual_vjp(Q, 0.01, gL, gLt)
    assert torch.equal(gQ1, gQ2)
    eps = 1e-6
    Lp, Ltp = S.residual(Q + eps * d, 0.01)
    Lm, Ltm = S.residual(Q - eps * d, 0.01)
    fd = ((gL * (Lp - Lm).cpu().numpy()).sum() + (gLt * (Ltp - Ltm).cpu().numpy()).sum()) / (2 * eps)
    got = (gQ1.cpu().numpy() * d).sum()
    assert abs(got - fd) <= 1e-6 * abs(fd), (got, fd)


def test_vjp_of_mixed_solver_is_fp64():
    m, om = mesh_pair()
    Q = I.perturbed_state(om.advection_average(), seed=37, amp=0.02)
    p = CASES["smooth_zero"]
    gL, gLt, _ = I.normal_directions(Q.shape, 3, 38)
    g64 = gks.Solver(m, **p).residual_vjp(Q, 0.01, gL, gLt)
    gmx = gks.Solver(m, precision=gks.GKS_PREC_MIXED, **p).residual_vjp(Q, 0.01, gL, gLt)
    assert (g64 - gmx).norm() <= 1e-13 * g64.norm()


def test_checkpointed_s2o4_rollout_gradient():
    """Gradient of J = sum |Omega| rho^2 after 6 S2O4 steps (checkpoint every 2) through the
    autograd wrapper, against central differences and the oracle's forward-mode rollout."""
    from paper_2203_09047_gb300.autograd import s2o4_rollout
    m, om = mesh_pair()
    p = CASES["full_viscous"]
    Q0 = I.perturbed_state(om.advection_average(), seed=39, amp=0.01)
    vol = torch.from_numpy(om.cell_info()["vol"]).cuda()
    S = gks.Solver(m, **p)
    dt = 0.004
    nsteps = 6

    def J(Q):
        QT = s2o4_rollout(Q, S, dt, nsteps, checkpoint_every=2)
        return (vol * QT[0] ** 2).sum()

    Qt = torch.from_numpy(Q0).cuda().requires_grad_(True)
    J(Qt).backward()
    grad = Qt.grad.detach().cpu().numpy()
    dirs = I.normal_directions(Q0.shape, 3, 40)
    with torch.no_grad():
        J0 = abs(J(Qt).item())
        for d in dirs:
            eps = 1e-6
            dd = torch.from_numpy(d).cuda()
            fd = (J(Qt + eps * dd) - J(Qt - eps * dd)).item() / (2 * eps)
            # central differences carry O(eps^2) truncation and the FP64 rounding of the two
            # evaluations of J divided by 2 eps (a few eps_64 |J| / eps, about 1e-9 here)
            assert abs((grad * d).sum() - fd) <= 1e-6 * abs(fd) + 8 * 2.2e-16 * J0 / eps
    # the oracle's tangent rollout for one direction
    d = dirs[0]
    QTo, dQTo = om.step_jvp(oracle.params_vec(**p), Q0, d, dt, nsteps)
    jd = (2.0 * om.cell_info()["vol"] * QTo[0] * dQTo[0]).sum()
    assert abs((grad * d).sum() - jd) <= 1e-9 * abs(jd)


def _jacobian_columns(om, params, Q, dt, cols):
    """Columns of d(L, Lt)/dQ for the (variable, cell) pairs in cols, from the oracle's
    dual-number JVP: [len(cols)][2][5][n]."""
    out = []
    for v, c in cols:
        dQ = np.zeros_like(Q)
        dQ[v, c] = 1.0
        _, _, dL, dLt = om.residual_jvp(params, Q, dQ, dt)
        out.append(np.stack([dL, dLt]))
    return np.array(out)


def _vjp_rows(S, Q, dt, rows, n):
    """Rows of d(L, Lt)/dQ for the (output, variable, cell) triples in rows (output 0: L,
    1: Lt), from the GPU VJP with a unit cotangent: [len(rows)][5][n]."""
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    g0 = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    gQ = torch.empty_like(Qd)
    out = []
    for o, w, j in rows:
        gL, gLt = g0.clone(), g0.clone()
        (gL if o == 0 else gLt)[w, j] = 1.0
        gks.gks_residual_vjp(S.h, Qd, dt, gL, gLt, gQ)
        out.append(gQ.cpu().numpy())
    return np.array(out)


@pytest.mark.parametrize("case", ["full_viscous", "smooth_zero"])
def test_vjp_full_jacobian_elementwise_small_hex_mesh(case):
    """Every entry of the transposed Jacobian from the GPU VJP (one unit cotangent per row)
    against every column of the oracle's dual-number JVP, on 4^3 periodic hexahedra (64 cells,
    a 640 x 320 matrix), nonlinear weights active on a perturbed state."""
    m, om = mesh_pair(4, "hex")
    n = om.n_cells
    Q = I.perturbed_state(om.advection_average(), seed=71, amp=0.03)
    p = CASES[case]
    dt = 0.01
    J = _jacobian_columns(om, oracle.params_vec(**p), Q, dt,
                          [(v, c) for v in range(5) for c in range(n)])  # [(v,c)][o][w][j]
    S = gks.Solver(m, **p)
    rows = [(o, w, j) for o in range(2) for w in range(5) for j in range(n)]
    G = _vjp_rows(S, Q, dt, rows, n)  # [(o,w,j)][v][c]
    Jt = J.reshape(5 * n, 2 * 5 * n).T  # [(o,w,j)][(v,c)]
    Gm = G.reshape(2 * 5 * n, 5 * n)
    scale = np.abs(Jt).max()
    assert np.abs(Gm - Jt).max() <= 1e-10 * scale, np.abs(Gm - Jt).max() / scale
    S.close()


def test_vjp_jacobian_columns_elementwise_hybrid_mesh():
    """Entries of three full columns of the Jacobian (a split-pyramid tetrahedron, a pyramid and
    a prism of the 8^3 hybrid box with enlarged stencils, every variable) from GPU VJP rows over
    the columns' support, against the oracle's JVP columns; rows outside the support read 0."""
    m = I.layered_box_mesh(8, "hybrid8")
    om = oracle.Mesh(m, min_stencil=18)
    n = om.n_cells
    Q = I.perturbed_state(oracle.Mesh(m).advection_average(), seed=72, amp=0.03)
    p = CASES["full_viscous"]
    dt = 0.01
    types = m["cell_type"]
    cells = [int(np.nonzero(types == t)[0][len(np.nonzero(types == t)[0]) // 2]) for t in (4, 5, 6)]
    cols = [(v, c) for c in cells for v in range(5)]
    J = _jacobian_columns(om, oracle.params_vec(**p), Q, dt, cols)  # [col][o][w][j]
    support = np.nonzero(np.abs(J).max(axis=(0, 1, 2)) > 0)[0]
    outside = np.setdiff1d(np.arange(n), support)[:8]
    S = gks.Solver(m, min_stencil=18, **p)
    rows = [(o, w, j) for j in np.concatenate([support, outside]) for o in range(2)
            for w in range(5)]
    G = _vjp_rows(S, Q, dt, rows, n)
    scale = np.abs(J).max()
    worst = 0.0
    for r, (o, w, j) in enumerate(rows):
        for k, (v, c) in enumerate(cols):
            worst = max(worst, abs(G[r, v, c] - J[k, o, w, j]))
    assert worst <= 1e-10 * scale, worst / scale
    S.close()
