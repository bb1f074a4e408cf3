"""Pins of the oracle's smoothness indicators and nonlinear weights (Section 2, Eqs. weno and
indicator), each checked against a value that does not come from the oracle's own formulas:

- beta_0 of an exact quadratic on an unjittered cube, against the closed-form integrals of its
  first and second derivatives over the cube (each multi-index l once, weight |Omega|^(2|l|/3-1));
- beta_m of linear data on any cell kind: |Omega|^(-1/3) |Omega| |grad P|^2;
- tau and the normalised weights for indicator values chosen so the result is a fraction worked
  out by hand (gamma_m = 0.0125, gamma_0 = 1 - 0.0125 M);
- a step profile, where the weights must gather on the candidates that do not cross the jump.

Each of these mistakes fails at least one test: a wrong |Omega| exponent in beta; the mixed second
derivatives counted twice or not at all; tau without its 1/M; epsilon added in the wrong place;
gamma_0 and gamma_m swapped; the exponent of tau/(beta + eps) other than the one asked for.
"""
import numpy as np
import pytest

import oracle
from paper_2203_09047_gb300 import inputs as I


@pytest.fixture(scope="module")
def cube8():
    m = I.layered_box_mesh(8, "hex", jitter=0.0)
    return m, oracle.Mesh(m)


def _interior_cells(om):
    """Cells whose stencils do not reach across the periodic boundary."""
    return np.nonzero(om.cell_info()["plain"])[0]


def _quadratic(rng):
    """Coefficients (1, x, y, z, xx, yy, zz, xy, xz, yz) of a quadratic for each variable, with
    every mixed term present and a physical state."""
    coef = rng.normal(size=(5, 10)) * 0.3
    coef[:, 0] += np.array([3.0, 0.0, 0.0, 0.0, 20.0])
    return coef


def _gradient_hessian(c, x):
    """Gradient and Hessian of one quadratic c[10] at x."""
    g = np.array([c[1] + 2 * c[4] * x[0] + c[7] * x[1] + c[8] * x[2],
                  c[2] + 2 * c[5] * x[1] + c[7] * x[0] + c[9] * x[2],
                  c[3] + 2 * c[6] * x[2] + c[8] * x[0] + c[9] * x[1]])
    H = np.array([[2 * c[4], c[7], c[8]], [c[7], 2 * c[5], c[9]], [c[8], c[9], 2 * c[6]]])
    return g, H


def _beta0_on_cube(c, centre, s):
    """Eq. indicator for P0 = the quadratic c on the cube of side s about centre, integrated in
    closed form. With xi = x - centre, d_a P = g_a + (H xi)_a, and over the cube the odd moments
    vanish and int xi_b^2 dV = s^5 / 12, so
        sum_{|l|=1} int (d^l P)^2 = s^3 |g|^2 + s^5/12 ||H||_F^2,
        sum_{|l|=2} int (d^l P)^2 = s^3 (H_xx^2 + H_yy^2 + H_zz^2 + H_xy^2 + H_xz^2 + H_yz^2)
    (the six second-order multi-indices (2,0,0) .. (0,1,1), each once). The weights are
    |Omega|^(2/3 - 1) = 1/s for |l| = 1 and |Omega|^(4/3 - 1) = s for |l| = 2."""
    g, H = _gradient_hessian(c, centre)
    first = s ** 3 * g @ g + s ** 5 / 12.0 * np.sum(H * H)
    second = s ** 3 * (np.sum(np.diag(H) ** 2) + H[0, 1] ** 2 + H[0, 2] ** 2 + H[1, 2] ** 2)
    return first / s + second * s


def test_beta0_of_a_quadratic_on_a_cube(cube8):
    m, om = cube8
    rng = np.random.default_rng(31)
    coef = _quadratic(rng)
    Q = om.cell_average(1, 0.0, coef.ravel())
    info = om.cell_info()
    s = 2.0 / 8  # side of every cell: |Omega| = 1/64, so every |Omega| power differs from 1
    cells = rng.choice(_interior_cells(om), 10, replace=False)
    P = oracle.params_vec()
    for c in cells:
        d = om.weno_detail(P, Q, c)
        assert d["M"] == 8
        assert abs(info["vol"][c] - s ** 3) < 1e-15
        for v in range(5):
            ref = _beta0_on_cube(coef[v], info["centroid"][c], s)
            assert d["beta"][v, 0] == pytest.approx(ref, rel=1e-11), (c, v)


def test_beta0_distinguishes_the_mixed_second_derivative(cube8):
    """A field whose only second-order term is xy: the |l| = 2 part of beta_0 is s |Omega| H_xy^2
    with H_xy = 1, exactly once."""
    m, om = cube8
    s = 0.25
    coef = np.zeros((5, 10))
    coef[:, 0] = [3.0, 0.0, 0.0, 0.0, 20.0]
    coef[0, 7] = 1.0  # rho = 3 + xy
    Q = om.cell_average(1, 0.0, coef.ravel())
    info = om.cell_info()
    c = _interior_cells(om)[0]
    d = om.weno_detail(oracle.params_vec(), Q, c)
    x0, y0, _ = info["centroid"][c]
    # first derivatives y, x: s^3 (y0^2 + x0^2) + s^5/12 (1 + 1); weight 1/s
    first = (s ** 3 * (x0 ** 2 + y0 ** 2) + s ** 5 / 6.0) / s
    second = s ** 3 * 1.0 * s
    assert d["beta"][0, 0] == pytest.approx(first + second, rel=1e-11)
    # the other variables are constant: every indicator vanishes
    assert np.max(np.abs(d["beta"][1:])) < 1e-20


@pytest.mark.parametrize("layers", ["hex", "tet", "prism", "hybrid8"])
def test_beta_of_linear_data_on_every_cell_kind(layers):
    """Linear data: every candidate reproduces it, so beta_0 = beta_m = |Omega|^(2/3) |grad P|^2
    (|l| = 1 only; the second derivatives of P0 vanish), tau = 0 and the weights are linear."""
    m = I.layered_box_mesh(16 if layers == "hybrid8" else 8, layers)
    om = oracle.Mesh(m)
    rng = np.random.default_rng(32)
    coef = np.zeros((5, 10))
    coef[:, :4] = rng.normal(size=(5, 4)) * 0.2
    coef[:, 0] += [3.0, 0.0, 0.0, 0.0, 20.0]
    Q = om.cell_average(1, 0.0, coef.ravel())
    vol = om.cell_info()["vol"]
    inner = _interior_cells(om)
    kinds = m["cell_type"][inner]
    cells = np.concatenate([rng.choice(inner[kinds == k], 3, replace=False) for k in np.unique(kinds)])
    assert layers != "hybrid8" or len(np.unique(kinds)) == 4  # pyramids included
    for c in cells:
        d = om.weno_detail(oracle.params_vec(), Q, c)
        M = d["M"]
        for v in range(5):
            ref = vol[c] ** (2.0 / 3.0) * np.sum(coef[v, 1:4] ** 2)
            np.testing.assert_allclose(d["beta"][v], np.full(M + 1, ref), rtol=1e-9)
        gam = np.r_[1 - 0.0125 * M, np.full(M, 0.0125)]
        np.testing.assert_allclose(d["wbar"], np.tile(gam, (5, 1)), rtol=0, atol=1e-7)


def test_weights_from_hand_worked_indicators():
    """M = 8, beta_0 = 1, beta_1..7 = 1, beta_8 = 3: tau = |1 - 3| / 8 = 1/4.
    eps = 0:  omega_0 = 0.9 (1 + 1/4) = 1.125, omega_1..7 = 0.0125 (5/4) = 1/64,
              omega_8 = 0.0125 (1 + 1/12) = 13/960; the sum is 1198/960, so
              wbar = (1080, 15 x 7, 13) / 1198.
    eps = 1:  ratios 1/8 and 1/16: omega_0 = 0.9 (9/8), omega_1..7 = 0.0125 (9/8),
              omega_8 = 0.0125 (17/16); in units of 0.0125/16: 1296, 18 x 7, 17, sum 1439.
    eps = 0, exponent 2: ratios squared 1/16 and 1/144: omega_0 = 0.9 (17/16),
              omega_1..7 = 0.0125 (17/16), omega_8 = 0.0125 (145/144); in units of 0.0125/144:
              11016, 153 x 7, 145, sum 12232."""
    beta = np.array([1.0, 1, 1, 1, 1, 1, 1, 1, 3])
    w, tau = oracle.weno_weights(oracle.params_vec(weno_eps=0.0), beta)
    assert tau == pytest.approx(0.25, rel=1e-15)
    np.testing.assert_allclose(w, np.r_[1080, [15] * 7, 13] / 1198.0, rtol=1e-14)
    w, tau = oracle.weno_weights(oracle.params_vec(weno_eps=1.0), beta)
    np.testing.assert_allclose(w, np.r_[1296, [18] * 7, 17] / 1439.0, rtol=1e-14)
    w, _ = oracle.weno_weights(oracle.params_vec(weno_eps=0.0, weno_pow=2), beta)
    np.testing.assert_allclose(w, np.r_[11016, [153] * 7, 145] / 12232.0, rtol=1e-14)


def test_weights_of_a_tetrahedron_count():
    """M = 4 (a tetrahedron): gamma_0 = 0.95. beta = (2, 0, 2, 2, 4): tau = (2 + 0 + 0 + 2)/4 = 1.
    eps = 1: ratios 1/3, 1, 1/3, 1/3, 1/5: omega = 0.95 (4/3), 0.0125 (2), 0.0125 (4/3) x 2,
    0.0125 (6/5); in units of 0.0125/15: 1520, 30, 20, 20, 18, sum 1608."""
    beta = np.array([2.0, 0.0, 2.0, 2.0, 4.0])
    w, tau = oracle.weno_weights(oracle.params_vec(weno_eps=1.0), beta)
    assert tau == pytest.approx(1.0, rel=1e-15)
    np.testing.assert_allclose(w, np.array([1520, 30, 20, 20, 18]) / 1608.0, rtol=1e-14)


def test_weights_gather_on_the_smooth_side_of_a_jump(cube8):
    """A density step at x = 1 seen from the cell just left of it: the candidates that stay on
    the left see constant data (beta_m = 0) and take all the weight as tau / eps grows; the
    candidates across the jump and P0 keep a weight of order eps / tau."""
    m, om = cube8
    cen = om.cell_info()["centroid"]
    rho = np.where(cen[:, 0] < 1.0, 1.0, 2.0)
    Q = np.stack([rho, 0 * rho, 0 * rho, 0 * rho, np.full_like(rho, 2.5)])
    target = np.nonzero((np.abs(cen[:, 0] - 0.875) < 1e-9) & (np.abs(cen[:, 1] - 0.875) < 1e-9)
                        & (np.abs(cen[:, 2] - 0.875) < 1e-9))[0][0]
    d = om.weno_detail(oracle.params_vec(), Q, target)
    beta, w = d["beta"][0], d["wbar"][0]
    smooth = np.nonzero(beta[1:] < 1e-24)[0] + 1
    rough = np.setdiff1d(np.arange(1, 9), smooth)
    # two of the four side neighbours of a hexahedron lie in each candidate, so the one across
    # the jump belongs to half of the eight candidates
    assert len(smooth) == 4 and len(rough) == 4
    assert beta[0] > 0.01 and np.all(beta[rough] > 0.01)
    assert w[smooth].sum() > 1.0 - 1e-6
    np.testing.assert_allclose(w[smooth], 0.25, rtol=1e-6)
    assert w[0] < 1e-6 and np.all(w[rough] < 1e-6)
    # the energy is uniform: every indicator vanishes and the weights stay linear
    np.testing.assert_allclose(d["wbar"][4], np.r_[0.9, [0.0125] * 8], rtol=1e-12)
