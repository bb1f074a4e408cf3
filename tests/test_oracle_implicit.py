"""Pins of the oracle's implicit Jacobi step (Section 4) against properties the method fixes:
a state with zero residual does not move (free stream, and a gas at rest in a walled box); for
small dt the step agrees with explicit Euler on the step-averaged residual to O(dt^2); with the
Jacobi iteration converged the update is conservative (the flux-split operator sums to zero over
a closed periodic mesh)."""
import numpy as np
import pytest

import oracle
from paper_2203_09047_gb300 import inputs as I


@pytest.fixture(scope="module")
def meshes():
    per = I.layered_box_mesh(8, "hybrid8")
    wall = I.layered_box_mesh(8, "hybrid8", lo=(-1, -1, -1), hi=(1, 1, 1), bc=(1, 1, 1))
    return oracle.Mesh(per), oracle.Mesh(wall)


def test_free_stream_and_rest_state_do_not_move(meshes):
    per, wall = meshes
    P = oracle.params_vec()
    q = np.array([1.2, 0.3, -0.5, 0.7, 2.5 / 0.4 + 0.5 * (0.09 + 0.25 + 0.49) / 1.2])
    Q = np.tile(q[:, None], (1, per.n_cells))
    Q1 = per.step_implicit(P, Q, 5e-3, 2, 3)
    assert np.abs(Q1 - Q).max() < 1e-12
    rest = np.tile(np.array([1.0, 0.0, 0.0, 0.0, 2.5])[:, None], (1, wall.n_cells))
    R1 = wall.step_implicit(P, rest, 5e-3, 2, 3)
    assert np.abs(R1 - rest).max() < 1e-12


@pytest.mark.parametrize("which", [0, 1])
def test_small_dt_agrees_with_explicit_euler_to_second_order(meshes, which):
    om = meshes[which]
    P = oracle.params_vec(flux_mode=1, tau_model=1)
    if which == 0:
        Q = om.advection_average()
    else:  # smooth perturbation of a gas at rest in the walled box
        rest = np.tile(np.array([1.0, 0.0, 0.0, 0.0, 2.5])[:, None], (1, om.n_cells))
        Q = I.perturbed_state(rest, seed=5, amp=0.01)

    def err(dt):
        L, Lt = om.residual(P, Q, dt)
        return np.abs(om.step_implicit(P, Q, dt, 1, 3) - (Q + dt * (L + 0.5 * dt * Lt))).max()

    e1, e2 = err(2e-3), err(1e-3)
    assert 3.4 < e1 / e2 < 4.6


def test_converged_jacobi_update_is_conservative(meshes):
    per = meshes[0]
    P = oracle.params_vec()
    Q = I.perturbed_state(per.advection_average(), seed=6, amp=0.02)
    vol = per.cell_info()["vol"]
    dt = per.max_dt(P, Q, 0.5)
    tot0 = (Q * vol).sum(axis=1)
    Q60 = per.step_implicit(P, Q, dt, 1, 60)
    assert np.all(np.abs((Q60 * vol).sum(axis=1) - tot0) <= 1e-13 * np.abs(tot0).clip(min=1.0))
    # the iteration has converged: more sweeps do not change the update
    Q80 = per.step_implicit(P, Q, dt, 1, 80)
    assert np.abs(Q80 - Q60).max() < 1e-13
