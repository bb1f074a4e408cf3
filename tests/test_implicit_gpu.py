"""Parity of the implicit Jacobi step (Section 4, gks_step_implicit through the C ABI) with the
FP64 oracle's implicit step on the same seeded inputs: FP64 to 1e-12 relative L2 of the state
change, mixed precision (FP32 reconstruction, flux and Jacobi sweeps, float-float state) to the
residual tolerance of the parity tests relative to the state change. Also on the GPU: zero
residual states stay put and the converged iteration conserves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL = 2e-4  # relative L2 of the state change in mixed mode

CASES = {
    "smooth_zero": dict(flux_mode=0, tau_model=0),
    "full_inviscid": dict(flux_mode=1, tau_model=1),
    "smooth_viscous": dict(flux_mode=0, tau_model=2, mu=2e-3),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()


_cache = {}


def setup(kind):
    if kind not in _cache:
        if kind == "periodic":
            m = I.layered_box_mesh(8, "hybrid8")
            om = oracle.Mesh(m)
            Q = I.perturbed_state(om.advection_average(), seed=21, amp=0.02)
        else:  # reflecting walls, a perturbed gas at rest
            m = I.layered_box_mesh(8, "hybrid8", lo=(-1, -1, -1), hi=(1, 1, 1), bc=(1, 1, 1))
            om = oracle.Mesh(m)
            rest = np.tile(np.array([1.0, 0.0, 0.0, 0.0, 2.5])[:, None], (1, om.n_cells))
            Q = I.perturbed_state(rest, seed=22, amp=0.02)
        _cache[kind] = (m, om, Q)
    return _cache[kind]


def run(m, Q, params, precision, dt, nsteps, kmax):
    S = gks.Solver(gks.Mesh(m), precision=precision, **params)
    S.set_state(Q)
    S.step_implicit(dt, nsteps, kmax)
    out = S.get_state().cpu().numpy()
    S.close()
    return out


@pytest.mark.parametrize("kind", ["periodic", "walls"])
@pytest.mark.parametrize("case", list(CASES))
def test_implicit_step_matches_oracle(kind, case):
    m, om, Q = setup(kind)
    p = CASES[case]
    P = oracle.params_vec(**p)
    dt = 2.0 * om.max_dt(P, Q, 0.5)  # CFL 1
    Qo = om.step_implicit(P, Q, dt, 2, 3)
    d = np.linalg.norm(Qo - Q)
    Q64 = run(m, Q, p, gks.GKS_PREC_FP64, dt, 2, 3)
    assert np.linalg.norm(Q64 - Qo) <= FP64_TOL * d
    Qmx = run(m, Q, p, gks.GKS_PREC_MIXED, dt, 2, 3)
    assert np.linalg.norm(Qmx - Qo) <= MIXED_TOL * d


def test_implicit_single_sweep_and_many_sweeps_match_oracle():
    m, om, Q = setup("periodic")
    p = CASES["smooth_zero"]
    P = oracle.params_vec(**p)
    dt = om.max_dt(P, Q, 0.5)
    for kmax in (1, 8):
        Qo = om.step_implicit(P, Q, dt, 1, kmax)
        Q64 = run(m, Q, p, gks.GKS_PREC_FP64, dt, 1, kmax)
        assert np.linalg.norm(Q64 - Qo) <= FP64_TOL * np.linalg.norm(Qo - Q)


def test_implicit_free_stream_and_conservation_on_gpu():
    m, om, Q = setup("periodic")
    q = np.array([1.2, 0.3, -0.5, 0.7, 2.5 / 0.4 + 0.5 * (0.09 + 0.25 + 0.49) / 1.2])
    U = np.tile(q[:, None], (1, om.n_cells))
    for prec in (gks.GKS_PREC_FP64, gks.GKS_PREC_MIXED):
        out = run(m, U, {}, prec, 5e-3, 2, 3)
        assert np.abs(out - U).max() < (1e-13 if prec == gks.GKS_PREC_FP64 else 1e-6)
    vol = om.cell_info()["vol"]
    P = oracle.params_vec()
    dt = om.max_dt(P, Q, 0.5)
    tot0 = (Q * vol).sum(axis=1)
    out = run(m, Q, {}, gks.GKS_PREC_FP64, dt, 1, 60)
    assert np.all(np.abs((out * vol).sum(axis=1) - tot0) <= 1e-13 * np.abs(tot0).clip(min=1.0))


def test_implicit_rejects_bad_arguments():
    m, om, Q = setup("periodic")
    S = gks.Solver(gks.Mesh(m))
    S.set_state(Q)
    for args in ((0.0, 1, 3), (1e-3, -1, 3), (1e-3, 1, 0)):
        with pytest.raises(gks.GksError) as e:
            gks.gks_step_implicit(S.h, *args)
        assert e.value.status == gks.GKS_E_INVAL
    S.close()
