"""The allocation-free CFL time-step call, gks_cfl_dt_noalloc.

It serves callers that cannot call cudaMalloc (a framework pool owns the device memory, or a
latency-critical loop must not pay for cudaMalloc's implicit synchronisation): its scratch is a
fixed array inside the library. These checks call it through the C ABI and compare it with the
allocating gks_max_dt of a solver on the same state, on two calls in a row (the second reuses
the scratch the first one filled). This file is collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402

TOL = 1e-12  # relative, as in the FP64 parity tests


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()
    m = I.layered_box_mesh(8, "hybrid8")
    om = oracle.Mesh(m)
    vol = om.cell_info()["vol"]
    fi = om.face_info()
    area = fi["w"].sum(axis=1)
    amax = np.zeros(om.n_cells)
    np.maximum.at(amax, fi["owner"], area)
    np.maximum.at(amax, fi["nb"][fi["nb"] >= 0], area[fi["nb"] >= 0])
    h = vol / amax  # cell length used by the time-step bound
    return m, om, h


def _noalloc(Q, h, gamma, mu, cfl):
    stream = torch.cuda.current_stream()
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    hd = torch.from_numpy(np.ascontiguousarray(h)).cuda()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    gks.gks_cfl_dt_noalloc(Q.shape[1], Qd, hd, gamma, mu, cfl, out, stream.cuda_stream)
    stream.synchronize()
    return float(out.item())


def test_noalloc_dt_matches_max_dt_twice(setup):
    m, om, h = setup
    Q1 = I.perturbed_state(om.advection_average(), seed=21, amp=0.02)
    S1 = gks.Solver(m)
    S1.set_state(Q1)
    ref1 = S1.max_dt(0.5)
    got1 = _noalloc(Q1, h, 1.4, 0.0, 0.5)
    assert abs(got1 - ref1) <= TOL * ref1
    # second call in a row: another state, viscosity and CFL number
    Q2 = I.perturbed_state(I.taylor_green_state(m), seed=22, amp=0.05)
    S2 = gks.Solver(m, mu=2e-2, tau_model=2)
    S2.set_state(Q2)
    ref2 = S2.max_dt(0.3)
    got2 = _noalloc(Q2, h, 1.4, 2e-2, 0.3)
    assert abs(got2 - ref2) <= TOL * ref2
    assert got1 != got2


def test_noalloc_dt_flags_nonphysical_and_rejects_oversize(setup):
    m, om, h = setup
    Q0 = om.advection_average()
    Q = Q0.copy()
    Q[4, 5] = 0.0  # negative pressure in one cell
    assert _noalloc(Q, h, 1.4, 0.0, 0.5) == -1.0
    # zero pressure: the sound speed is 0 and the bound alone would stay positive
    Q = Q0.copy()
    Q[4, 7] = 0.5 * (Q[1, 7] ** 2 + Q[2, 7] ** 2 + Q[3, 7] ** 2) / Q[0, 7]
    assert _noalloc(Q, h, 1.4, 0.0, 0.5) == -1.0
    # negative density and negative pressure: gamma p / rho is positive, c is real
    Q = Q0.copy()
    Q[:, 9] = [-1.0, 0.0, 0.0, 0.0, -1.0]
    assert _noalloc(Q, h, 1.4, 0.0, 0.5) == -1.0
    # a NaN anywhere in a cell
    Q = Q0.copy()
    Q[2, 11] = float("nan")
    assert _noalloc(Q, h, 1.4, 0.0, 0.5) == -1.0
    # the physical state itself stays positive after those calls reused the scratch
    assert _noalloc(Q0, h, 1.4, 0.0, 0.5) > 0.0
    tiny = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GksError) as e:
        # rejected on the host before any launch
        gks.gks_cfl_dt_noalloc(16_777_217, tiny, tiny, 1.4, 0.0, 0.5, tiny, 0)
    assert e.value.status == gks.GKS_E_INVAL and "limit" in str(e.value)
