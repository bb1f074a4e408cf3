"""The C-ABI library builds, loads, exports every symbol include/gks.h declares, and its
host-side mesh construction (faces, stencils) agrees with the oracle's. No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2203_09047_gb300 as gks
from paper_2203_09047_gb300 import build, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gks.load_library()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_params_default(lib):
    p = gks.gks_params_default()
    assert p.gamma == 1.4 and p.weno_gamma == 0.0125 and p.weno_eps == 1e-8 and p.weno_pow == 1
    assert p.tau_eps == 0.01 and p.tau_C == 1.0 and p.Pr == 1.0


@pytest.mark.parametrize("n,layers,bc", [(8, "hybrid8", (0, 0, 0)), (4, "hex", (0, 0, 0)),
                                         (4, "tet", (0, 0, 0)), (8, "hybrid8", (1, 1, 1)),
                                         (8, "hybrid8", (0, 1, 0)), (8, "hybrid8", (2, 2, 2)),
                                         (4, "tet", (3, 1, 2)), (4, "hex", (3, 3, 3))])
def test_mesh_counts_match_oracle(lib, n, layers, bc):
    m = I.layered_box_mesh(n, layers, bc=bc)
    h = gks.gks_mesh_create(m["xyz"], m["cell_type"], m["cell_nodes"], m["bc"], m["lo"], m["hi"])
    try:
        nc, nf, nst = gks.gks_mesh_counts(h)
    finally:
        gks.gks_mesh_destroy(h)
    om = oracle.Mesh(m)
    info = om.cell_info()
    assert nc == om.n_cells and nf == om.n_faces
    assert nst == int(info["K"].sum())


@pytest.mark.parametrize("n,layers,bc", [(8, "hybrid8", (0, 0, 0)), (8, "hybrid8", (1, 1, 1)),
                                         (4, "tet", (3, 1, 2))])
@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_enlarged_stencils_match_oracle(lib, n, layers, bc, reorder):
    """min_stencil = 18: both sides take the same third-ring members, for every cell order; the
    stencils that already had 18 or more members are unchanged."""
    m = I.layered_box_mesh(n, layers, bc=bc)
    h = gks.gks_mesh_create(m["xyz"], m["cell_type"], m["cell_nodes"], m["bc"], m["lo"], m["hi"],
                            reorder=reorder, min_stencil=18)
    try:
        nc, nf, nst = gks.gks_mesh_counts(h)
    finally:
        gks.gks_mesh_destroy(h)
    K = oracle.Mesh(m, min_stencil=18).cell_info()["K"]
    K0 = oracle.Mesh(m).cell_info()["K"]
    assert nst == int(K.sum())
    assert np.all(K >= np.minimum(18, K0)) and np.all(K[K0 >= 18] == K0[K0 >= 18])
    assert K.min() >= 18 or layers == "tet"  # tetrahedra at walls may run out of candidates


def test_mesh_options_rejected(lib):
    m = I.layered_box_mesh(4, "hex")
    for kw in (dict(reorder=3), dict(min_stencil=-1), dict(min_stencil=65)):
        with pytest.raises(gks.GksError) as e:
            gks.gks_mesh_create(m["xyz"], m["cell_type"], m["cell_nodes"], m["bc"], m["lo"],
                                m["hi"], **kw)
        assert e.value.status == gks.GKS_E_INVAL


def test_mesh_errors(lib):
    m = I.layered_box_mesh(4, "hex")
    bad = dict(m)
    bad["cell_type"] = m["cell_type"].copy()
    bad["cell_type"][3] = 7
    with pytest.raises(gks.GksError) as e:
        gks.gks_mesh_create(bad["xyz"], bad["cell_type"], bad["cell_nodes"], bad["bc"], bad["lo"], bad["hi"])
    assert e.value.status == gks.GKS_E_INVAL
    # drop one cell: its neighbours' faces become unmatched inside a periodic box
    with pytest.raises(gks.GksError) as e:
        gks.gks_mesh_create(m["xyz"], m["cell_type"][1:], m["cell_nodes"][1:], m["bc"], m["lo"], m["hi"])
    assert e.value.status == gks.GKS_E_MESH
    nodes = m["cell_nodes"].copy()
    nodes[0, 0] = len(m["xyz"])
    with pytest.raises(gks.GksError) as e:
        gks.gks_mesh_create(m["xyz"], m["cell_type"], nodes, m["bc"], m["lo"], m["hi"])
    assert e.value.status == gks.GKS_E_INVAL


def test_invalid_parameters_are_rejected_before_any_device_work(lib):
    """gks_init validates its parameters first (no CUDA call is made for a rejected set)."""
    m = I.layered_box_mesh(4, "hex", bc=(3, 2, 1))
    h = gks.gks_mesh_create(m["xyz"], m["cell_type"], m["cell_nodes"], m["bc"], m["lo"], m["hi"])
    try:
        far_bad = np.tile([1.0, 0.0, 0.0, 0.0, 1.0], (6, 1))
        far_bad[3, 4] = -1.0
        wall_bad = np.zeros((6, 3))
        wall_bad[4, 0] = np.nan
        for bad in (dict(tau_model=3, T_ref=0.0), dict(tau_model=4), dict(farfield=far_bad),
                    dict(wall_u=wall_bad), dict(wall_T=[0, 0, 0, 0, np.inf, 0])):
            with pytest.raises(gks.GksError) as e:
                gks.gks_init(h, gks.gks_params_default(**bad))
            assert e.value.status == gks.GKS_E_INVAL, bad
    finally:
        gks.gks_mesh_destroy(h)


def test_wall_and_farfield_parameter_defaults(lib):
    p = gks.gks_params_default()
    assert p.T_ref == 1.0 and p.mu_pow == 0.7
    assert all(p.wall_T[w] == 0.0 and list(p.wall_u[w]) == [0.0, 0.0, 0.0] for w in range(6))
    assert all(list(p.farfield[w]) == [1.0, 0.0, 0.0, 0.0, 1.0 / 1.4] for w in range(6))
    q = gks.gks_params_default(farfield=(1.2, 0.1, 0.0, 0.0, 0.9))
    assert all(list(q.farfield[w]) == [1.2, 0.1, 0.0, 0.0, 0.9] for w in range(6))
