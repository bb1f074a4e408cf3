"""The benchmark workload at full size: the 64^3-cube hybrid advection mesh (1,048,576 cells),
the solvers built as bench.py builds them. Sampled cells are checked against the oracle one by
one (its stencils are built only where needed); conservation, free-stream preservation and
determinism are checked on the whole mesh."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

MIXED_TOL_L = 2e-4


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()
    m = I.layered_box_mesh(64, "hybrid8")
    mesh = gks.Mesh(m)
    om = oracle.Mesh(m, lazy=True)
    return m, mesh, om


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("params", [dict(flux_mode=0, tau_model=0),
                                    dict(flux_mode=1, tau_model=2, mu=1e-3)])
def test_sampled_residual_matches_oracle(full, params):
    m, mesh, om = full
    assert mesh.n_cells == 1048576 and mesh.n_faces == 2392064
    Q = I.perturbed_state(I.advection_state(m), seed=41, amp=0.01)
    dt = 2e-3
    rng = np.random.default_rng(42)
    cells = np.sort(rng.choice(mesh.n_cells, 96, replace=False))
    Lo, Lto = om.residual_cells(oracle.params_vec(**params), Q, dt, cells)
    S64 = gks.Solver(mesh, **params)
    L, Lt = S64.residual(Q, dt)
    L, Lt = L.cpu().numpy()[:, cells].T, Lt.cpu().numpy()[:, cells].T
    assert _rel(L, Lo) < 1e-12 and _rel(Lt, Lto) < 1e-12
    S32 = gks.Solver(mesh, precision=gks.GKS_PREC_MIXED, **params)
    Lm, _ = S32.residual(Q, dt)
    assert _rel(Lm.cpu().numpy()[:, cells].T, Lo) < MIXED_TOL_L


def test_full_size_steps_conserve_and_repeat(full):
    m, mesh, om = full
    Q0 = I.advection_state(m)
    vol = torch.from_numpy(om.cell_info()["vol"]).cuda()
    for prec in (gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED):
        S = gks.Solver(mesh, precision=prec)
        S.set_state(Q0)
        dt = S.max_dt(0.5)
        S.step(dt, 3)
        Q1 = S.get_state()
        S.set_state(Q0)
        S.step(dt, 3)
        assert torch.equal(Q1, S.get_state())  # bitwise repeatable
        tot0 = (torch.from_numpy(Q0).cuda() * vol).sum(dim=1)
        tot1 = (Q1 * vol).sum(dim=1)
        assert ((tot1 - tot0).abs() <= 1e-12 * tot0.abs().clamp(min=1.0)).all()


def test_full_size_free_stream(full):
    m, mesh, om = full
    q = np.array([1.2, 0.3, -0.5, 0.7, 2.5 / 0.4 + 0.5 * (0.09 + 0.25 + 0.49) / 1.2])
    Q = np.tile(q[:, None], (1, mesh.n_cells))
    S = gks.Solver(mesh, precision=gks.GKS_PREC_MIXED, flux_mode=1, tau_model=1)
    S.set_state(Q)
    S.step(1e-3, 2)
    # FP32 fluxes: the free-stream residual of a cell is FP32 rounding of its face fluxes,
    # |dQ| ~ eps32 t |F| A/|Omega|; the largest values sit in the smallest tetrahedra (|Omega|
    # about 0.4 of the median), the bulk is two orders lower
    err = np.abs(S.get_state().cpu().numpy() - Q).max(axis=0)
    assert err.max() < 3e-5 and np.quantile(err, 0.999) < 2e-6


def test_full_size_implicit_steps_repeat_and_conserve_when_converged(full):
    """Implicit Jacobi steps (Section 4) on the benchmark mesh: bitwise repeatable (concurrent
    reconstruction ranges, fixed-order gathers); with the iteration converged the update is
    conservative (the flux-split operator sums to zero over the closed periodic mesh)."""
    m, mesh, om = full
    Q0 = I.advection_state(m)
    vol = torch.from_numpy(om.cell_info()["vol"]).cuda()
    tot0 = (torch.from_numpy(Q0).cuda() * vol).sum(dim=1)
    for prec in (gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED):
        S = gks.Solver(mesh, precision=prec)
        S.set_state(Q0)
        dt = S.max_dt(1.0)
        S.step_implicit(dt, 2, 3)
        Q1 = S.get_state()
        S.set_state(Q0)
        S.step_implicit(dt, 2, 3)
        assert torch.equal(Q1, S.get_state())
        if prec == gks.GKS_PREC_FP64:
            S.set_state(Q0)
            S.step_implicit(dt, 1, 60)
            tot1 = (S.get_state() * vol).sum(dim=1)
            assert ((tot1 - tot0).abs() <= 1e-12 * tot0.abs().clamp(min=1.0)).all()
        S.close()
