"""The exact Riemann solver that validates the Sod case, checked against the laws it must obey:
Rankine-Hugoniot conditions across its shock, the isentropic relation across its rarefaction,
continuity of pressure and velocity at the contact."""
import numpy as np

from paper_2203_09047_gb300.cases import exact_riemann

G = 1.4


def _E(r, u, p):
    return p / (G - 1) + 0.5 * r * u * u


def test_sod_jump_conditions_and_rarefaction():
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    x = np.linspace(0.0, 1.0, 4001)
    r, u, p, ps, us = exact_riemann(L, R, x, 0.2)
    # star region right of the contact: density just behind the shock
    rs = r[(x > 0.5 + us * 0.2 + 1e-3) & (p > 0.9 * ps) & (p < 1.1 * ps)][0]
    # shock speed from mass conservation; momentum and energy must then balance
    S = (rs * us - R[0] * R[1]) / (rs - R[0])
    mom = (rs * us * us + ps) - (R[0] * R[1] ** 2 + R[2])
    ene = us * (_E(rs, us, ps) + ps) - R[1] * (_E(*R) + R[2])
    assert abs(mom - S * (rs * us - R[0] * R[1])) < 1e-12
    assert abs(ene - S * (_E(rs, us, ps) - _E(*R))) < 1e-12
    # the computed profile has its jump where S puts it
    xs = x[np.argmax(r < 0.5 * (rs + R[0]))]
    assert abs(xs - (0.5 + S * 0.2)) < 1e-3
    # left rarefaction: entropy p / rho^gamma unchanged through the fan and the left star state
    fan = (p < L[2]) & (p > ps) & (x < 0.5 + us * 0.2)
    assert fan.sum() > 10
    assert np.allclose(p[fan] / r[fan] ** G, L[2] / L[0] ** G, rtol=1e-12)
    rsl = r[(x < 0.5 + us * 0.2 - 1e-3) & (np.abs(p - ps) < 1e-14)][0]
    assert abs(ps / rsl ** G - L[2] / L[0] ** G) < 1e-12
    # Riemann invariant u + 2c/(gamma - 1) constant through the fan
    c = np.sqrt(G * p[fan] / r[fan])
    assert np.allclose(u[fan] + 2 * c / (G - 1), 2 * np.sqrt(G) / (G - 1), rtol=1e-12)
