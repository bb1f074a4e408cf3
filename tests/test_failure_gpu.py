"""Failure detection on the GPU without faulting it.

Every reconstruction block waits on an mbarrier (completed by the bulk copy of its sub-stencil
entries into shared memory, where the range stages them) with a bounded number of tries; when
the wait runs out, the block sets the timeout bit of the solver's status word and returns. The
test hook gks_debug_recon_wait withholds the copy and expects more bytes than any copy brings
(nothing is in flight, so the barrier simply never completes) with a limit of a few dozen
tries: the status check must report GKS_E_TIMEOUT, and the same solver must then compute a
normal residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2203_09047_gb300 as gks  # noqa: E402
from paper_2203_09047_gb300 import build, inputs as I  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gks.load_library()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("prec", [gks.GKS_PREC_MIXED, gks.GKS_PREC_FP64])
def test_bounded_wait_times_out_and_the_solver_recovers(prec):
    m = I.layered_box_mesh(3, "hex")  # 27 cells: one 32-cell tile
    om = oracle.Mesh(m)
    Q = I.perturbed_state(om.advection_average(), seed=61, amp=0.02)
    S = gks.Solver(m, precision=prec)
    L0, Lt0 = S.residual(Q, 0.01)
    gks.gks_debug_recon_wait(S.h, 32, True)
    with pytest.raises(gks.GksError) as e:
        S.residual(Q, 0.01)
    assert e.value.status == gks.GKS_E_TIMEOUT
    # a step reports it through gks_check as well
    S.set_state(Q)
    with pytest.raises(gks.GksError) as e:
        S.step(1e-3, 1)
    assert e.value.status == gks.GKS_E_TIMEOUT
    # back to normal: the same solver gives the same residual as before, and the oracle's
    gks.gks_debug_recon_wait(S.h, 0, False)
    L1, Lt1 = S.residual(Q, 0.01)
    assert torch.equal(L0, L1) and torch.equal(Lt0, Lt1)
    Lo, _ = om.residual(oracle.params_vec(), Q, 0.01)
    tol = 2e-4 if prec == gks.GKS_PREC_MIXED else 1e-12  # the path's residual tolerance
    assert rel(L1.cpu().numpy(), Lo) < tol
    # a short limit that the copies meet in time changes nothing
    gks.gks_debug_recon_wait(S.h, 1 << 16, False)
    L2, _ = S.residual(Q, 0.01)
    assert torch.equal(L0, L2)
    S.close()
