"""Seeded synthetic inputs: hybrid hexahedral/prismatic/pyramidal/tetrahedral meshes of a box
and conserved-variable states on them.

This module is shared by the CUDA path, the tests and the CPU oracle. It holds none of the
scheme's arithmetic: it only lays out nodes and cell connectivity and draws seeded numbers.

Cell connectivity uses eight slots per cell, the degenerate-hexahedron labelling of Section 2:
    tetrahedron  {p1 p2 p3 p3 p4 p4 p4 p4}
    pyramid      {p1 p2 p3 p4 p5 p5 p5 p5}
    prism        {p1 p2 p3 p3 p4 p5 p6 p6}
    hexahedron   {p1 p2 p3 p4 p5 p6 p7 p8}
with the bottom face p1 p2 p3 (p4) counter-clockwise seen from the top (the apex p4 of a
tetrahedron, the apex p5 of a pyramid, the second triangle of a prism, the top quad of a hex),
so every cell has positive volume.

Mesh recipe (the layered hybrid box): N x N x N cubes of side h = (hi - lo) / N. Each z-layer of
cubes is one of
    'hex'    one hexahedron per cube
    'prism'  two prisms per cube, axis along x, cut by the plane through the (y0,z0)-(y1,z1)
             diagonal of the yz square
    'trans'  six pyramids apexed at a node near the cube centre; the top one is cut into two
             tetrahedra along the (x0,y0)-(x1,y1) diagonal of the top face
    'transm' the same mirrored in z: the bottom pyramid is cut into two tetrahedra
    'tet'    six Kuhn tetrahedra around the (0,0,0)-(1,1,1) cube diagonal
Adjacent layers conform: quad faces meet quad faces and the triangulated faces of 'trans',
'transm' and 'tet' layers all use the (x0,y0)-(x1,y1) diagonal.
Nodes off the boundary planes (lattice nodes and cube-centre nodes) are displaced by
(2u - 1) * jitter * h per component, u from splitmix64 over (seed, 3 * node_id + component).
Boundary-plane nodes are not moved, so periodic faces match by translation.
"""
from __future__ import annotations

import numpy as np

TET, PYR, PRI, HEX = 4, 5, 6, 8
BC_PERIODIC, BC_REFLECT = 0, 1

# z-layer pattern of the 8-layer hybrid recipe (2 hex, prism, transition, 2 tet, mirrored
# transition, prism), repeated every 8 layers.
HYBRID8 = ("hex", "hex", "prism", "trans", "tet", "tet", "transm", "prism")

_MASK64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(_MASK64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(_MASK64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(_MASK64)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter: np.ndarray) -> np.ndarray:
    """U[0,1) from the top 53 bits of splitmix64(seed * 2^32 + counter)."""
    c = np.asarray(counter, dtype=np.uint64) + np.uint64((int(seed) << 32) & _MASK64)
    return (splitmix64(c) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def layer_pattern(name: str, n: int) -> tuple:
    """Named z-layer patterns.

    'hybrid8' : the 8-layer hybrid pattern repeated (n must be a multiple of 8)
    'tgv48'   : for n = 48: 12 hex, 6 prism, 1 trans, 22 tet, 1 transm, 6 prism; other n keep the
                same proportions (25 % hex, 12.5 % prism on each side of the tetrahedra)
    'hex' / 'tet' / 'prism' / 'trans' / 'transm' : every layer of one kind
    """
    if name == "hybrid8":
        if n % 8:
            raise ValueError("hybrid8 needs n divisible by 8")
        return HYBRID8 * (n // 8)
    if name == "tgv48":
        nh, npr = n // 4, n // 8
        nt = n - nh - 2 * npr - 2
        if nt < 1:
            raise ValueError("tgv48 needs n >= 8")
        return ("hex",) * nh + ("prism",) * npr + ("trans",) + ("tet",) * nt + ("transm",) + ("prism",) * npr
    if name in ("hex", "tet", "prism", "trans", "transm"):
        return (name,) * n
    raise ValueError(f"unknown layer pattern {name!r}")


def _kuhn_paths():
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    out = []
    for p in perms:
        v = [0, 0, 0]
        path = [tuple(v)]
        for ax in p:
            v[ax] = 1
            path.append(tuple(v))
        out.append(path)
    return out


def _signed_vol(x, a, b, c, d):
    return float(np.dot(np.cross(x[b] - x[a], x[c] - x[a]), x[d] - x[a]))


def layered_box_mesh(n: int, layers="hybrid8", lo=(0.0, 0.0, 0.0), hi=(2.0, 2.0, 2.0),
                     jitter: float = 0.1, seed: int = 1, bc=(BC_PERIODIC,) * 3, shape=None):
    """The layered hybrid box mesh described in the module docstring: n z-layers of n x n
    cubes, or of shape = (nx, ny) cubes.

    Returns a dict with
        xyz        float64 [n_nodes, 3]
        cell_type  int8    [n_cells]      4 tet, 5 pyramid, 6 prism, 8 hex
        cell_nodes int64   [n_cells, 8]   degenerate-hexahedron slots
        bc, lo, hi the box description passed to the mesh constructors
    Cells are numbered cube by cube (x fastest, then y, then z), in a fixed order within a cube.
    """
    if isinstance(layers, str):
        layers = layer_pattern(layers, n)
    if len(layers) != n:
        raise ValueError("need one layer kind per z-layer")
    nx, ny = (n, n) if shape is None else (int(shape[0]), int(shape[1]))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    counts = np.array([nx, ny, n])
    h = (hi - lo) / counts
    mx, my, mz = nx + 1, ny + 1, n + 1
    ii, jj, kk = np.meshgrid(np.arange(mx), np.arange(my), np.arange(mz), indexing="ij")
    lat = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                    kk.transpose(2, 1, 0).ravel()], axis=1)  # id = i + mx*(j + my*k)
    xyz = [lo[None, :] + lat * h[None, :]]
    interior = np.all((lat > 0) & (lat < counts[None, :]), axis=1)

    def lid(i, j, k):
        return i + mx * (j + my * k)

    n_lat = mx * my * mz
    centre = {}
    centres = []
    for k, kind in enumerate(layers):
        if kind in ("trans", "transm"):
            for j in range(ny):
                for i in range(nx):
                    centre[(i, j, k)] = n_lat + len(centres)
                    centres.append(lo + (np.array([i, j, k]) + 0.5) * h)
    if centres:
        xyz.append(np.array(centres))
    xyz = np.concatenate(xyz, axis=0)
    movable = np.concatenate([interior, np.ones(len(centres), dtype=bool)])
    ids = np.nonzero(movable)[0].astype(np.uint64)
    if jitter != 0.0 and len(ids):
        u = uniform01(seed, (3 * ids[:, None] + np.arange(3, dtype=np.uint64)[None, :]).ravel())
        xyz[ids] += ((2.0 * u - 1.0) * jitter).reshape(-1, 3) * h[None, :]

    # vectorised over the nx x ny cubes of each layer (x fastest, then y)
    jj2, ii2 = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ii2, jj2 = ii2.ravel(), jj2.ravel()
    kuhn = _kuhn_paths()
    blocks_t, blocks_n = [], []

    def emit(t, slots_list):
        """slots_list: list over the cells of one cube of [8] node-id arrays (one per cube);
        cells are interleaved cube by cube."""
        arr = np.stack([np.stack(sl, axis=1) for sl in slots_list], axis=1)  # [cubes, cells, 8]
        blocks_n.append(arr.reshape(-1, 8))
        blocks_t.append(np.broadcast_to(np.asarray(t, dtype=np.int8)[None, :], arr.shape[:2]).reshape(-1))

    def oriented_tet(a, b, c, d):
        vol = np.einsum("ij,ij->i", np.cross(xyz[b] - xyz[a], xyz[c] - xyz[a]), xyz[d] - xyz[a])
        flip = vol < 0.0
        b2 = np.where(flip, c, b)
        c2 = np.where(flip, b, c)
        return [a, b2, c2, c2, d, d, d, d]

    for k, kind in enumerate(layers):
        def V(a, b, c):
            return lid(ii2 + a, jj2 + b, k + c)
        if kind == "hex":
            emit([HEX], [[V(0, 0, 0), V(1, 0, 0), V(1, 1, 0), V(0, 1, 0),
                          V(0, 0, 1), V(1, 0, 1), V(1, 1, 1), V(0, 1, 1)]])
        elif kind == "prism":
            # triangles in the yz planes x = x0 (p1 p2 p3) and x = x1 (p4 p5 p6)
            cells = []
            for tri in (((0, 0), (1, 0), (1, 1)), ((0, 0), (1, 1), (0, 1))):
                b0 = [V(0, y, z) for (y, z) in tri]
                t0 = [V(1, y, z) for (y, z) in tri]
                cells.append([b0[0], b0[1], b0[2], b0[2], t0[0], t0[1], t0[2], t0[2]])
            emit([PRI, PRI], cells)
        elif kind in ("trans", "transm"):
            c = np.array([centre[(i, j, k)] for j, i in zip(jj2, ii2)], dtype=np.int64)
            bottom = [V(0, 0, 0), V(1, 0, 0), V(1, 1, 0), V(0, 1, 0)]
            top = [V(0, 0, 1), V(0, 1, 1), V(1, 1, 1), V(1, 0, 1)]
            sides = [[V(0, 0, 0), V(0, 1, 0), V(0, 1, 1), V(0, 0, 1)],   # x = x0
                     [V(1, 0, 0), V(1, 0, 1), V(1, 1, 1), V(1, 1, 0)],   # x = x1
                     [V(0, 0, 0), V(0, 0, 1), V(1, 0, 1), V(1, 0, 0)],   # y = y0
                     [V(0, 1, 0), V(1, 1, 0), V(1, 1, 1), V(0, 1, 1)]]   # y = y1
            quads = list(sides)
            if kind == "trans":
                quads.insert(0, bottom)
                split_z = 1
            else:
                quads.append(top)
                split_z = 0
            cells = [[q[0], q[1], q[2], q[3], c, c, c, c] for q in quads]
            a0, a1 = V(0, 0, split_z), V(1, 1, split_z)
            cells.append(oriented_tet(a0, V(1, 0, split_z), a1, c))
            cells.append(oriented_tet(a0, a1, V(0, 1, split_z), c))
            emit([PYR] * 5 + [TET, TET], cells)
        elif kind == "tet":
            emit([TET] * 6, [oriented_tet(*[V(*p) for p in path]) for path in kuhn])
        else:
            raise ValueError(kind)
    types = np.concatenate(blocks_t)
    nodes = np.concatenate(blocks_n)
    cell_type = np.ascontiguousarray(types, dtype=np.int8)
    cell_nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    return {"xyz": np.ascontiguousarray(xyz), "cell_type": cell_type, "cell_nodes": cell_nodes,
            "bc": tuple(int(b) for b in bc), "lo": tuple(float(v) for v in lo),
            "hi": tuple(float(v) for v in hi), "n": n, "shape": (nx, ny), "layers": tuple(layers)}


def mesh_summary(mesh) -> dict:
    t = mesh["cell_type"]
    return {"cells": int(len(t)), "hex": int((t == HEX).sum()), "prism": int((t == PRI).sum()),
            "pyramid": int((t == PYR).sum()), "tet": int((t == TET).sum()),
            "nodes": int(len(mesh["xyz"]))}


def vertex_mean(mesh) -> np.ndarray:
    """Mean of each cell's distinct vertices (a cheap cell location for synthetic states)."""
    cn = mesh["cell_nodes"]
    x = mesh["xyz"]
    out = np.empty((len(cn), 3))
    for t, nv, slots in ((TET, 4, [0, 1, 2, 4]), (PYR, 5, [0, 1, 2, 3, 4]),
                         (PRI, 6, [0, 1, 2, 4, 5, 6]), (HEX, 8, list(range(8)))):
        sel = mesh["cell_type"] == t
        if sel.any():
            out[sel] = x[cn[sel][:, slots]].mean(axis=1)
    return out


def advection_primitive(x: np.ndarray, t: float = 0.0):
    """Density sine wave of the accuracy test (Section 5.1): rho = 1 + 0.2 sin(pi(x+y+z-3t)),
    U = V = W = 1, p = 1 (the profile moves with the velocity (1,1,1)). Returns
    (rho, u[...,3], p) at points x[..., 3]."""
    s = x[..., 0] + x[..., 1] + x[..., 2] - 3.0 * t
    rho = 1.0 + 0.2 * np.sin(np.pi * s)
    u = np.ones(x.shape[:-1] + (3,))
    p = np.ones(x.shape[:-1])
    return rho, u, p


def primitive_to_conserved(rho, u, p, gamma=1.4) -> np.ndarray:
    """[5, ...] conserved (rho, rho U, rho V, rho W, rho E) from primitives."""
    ke = 0.5 * rho * (u * u).sum(axis=-1)
    return np.stack([rho, rho * u[..., 0], rho * u[..., 1], rho * u[..., 2],
                     p / (gamma - 1.0) + ke], axis=0)


def advection_state(mesh, gamma=1.4) -> np.ndarray:
    """Synthetic smooth state [5, n_cells] SoA: the advection field sampled at vertex means.
    (Not exact cell averages; it is a realistic smooth input for throughput and parity runs.)"""
    rho, u, p = advection_primitive(vertex_mean(mesh))
    return np.ascontiguousarray(primitive_to_conserved(rho, u, p, gamma))


def taylor_green_state(mesh, mach=0.1, gamma=1.4) -> np.ndarray:
    """Taylor-Green vortex state [5, n_cells] at vertex means: u = sin x cos y cos z,
    v = -cos x sin y cos z, w = 0, rho = 1, p = 1/(gamma Ma^2) + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    x = vertex_mean(mesh)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    u = np.stack([np.sin(X) * np.cos(Y) * np.cos(Z), -np.cos(X) * np.sin(Y) * np.cos(Z),
                  np.zeros_like(X)], axis=1)
    p = 1.0 / (gamma * mach * mach) + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    return np.ascontiguousarray(primitive_to_conserved(np.ones_like(X), u, p, gamma))


def explosion_state(mesh, gamma=1.4) -> np.ndarray:
    """Spherical explosion: rho = 1, p = 1 inside r < 0.4 (tested at the vertex mean), else
    rho = 0.125, p = 0.1; zero velocity."""
    x = vertex_mean(mesh)
    inside = (x * x).sum(axis=1) < 0.16
    rho = np.where(inside, 1.0, 0.125)
    p = np.where(inside, 1.0, 0.1)
    return np.ascontiguousarray(primitive_to_conserved(rho, np.zeros_like(x), p, gamma))


def rest_bump_state(mesh, amp=0.02, width2=0.02, centre=(0.5, 0.5, 0.5), gamma=1.4) -> np.ndarray:
    """Gas at rest (rho = 1, p = 1) with a smooth bump amp exp(-|x - centre|^2 / width2) added
    to density and pressure, sampled at vertex means."""
    x = vertex_mean(mesh)
    b = amp * np.exp(-((x - np.asarray(centre)) ** 2).sum(axis=1) / width2)
    return np.ascontiguousarray(primitive_to_conserved(1.0 + b, np.zeros_like(x), 1.0 + b, gamma))


def perturbed_state(q: np.ndarray, seed: int, amp: float = 0.01) -> np.ndarray:
    """q + U(-amp, amp) on every entry, u from splitmix64 over (seed, flat index)."""
    u = uniform01(seed, np.arange(q.size, dtype=np.uint64)).reshape(q.shape)
    return np.ascontiguousarray(q + (2.0 * u - 1.0) * amp)


def normal_directions(shape, count: int, seed: int) -> np.ndarray:
    """`count` unit directions of the given shape, N(0,1) entries by Box-Muller over splitmix64."""
    size = int(np.prod(shape))
    u1 = uniform01(seed, np.arange(count * size, dtype=np.uint64) * np.uint64(2))
    u2 = uniform01(seed, np.arange(count * size, dtype=np.uint64) * np.uint64(2) + np.uint64(1))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    z = z.reshape((count,) + tuple(shape))
    norms = np.sqrt((z.reshape(count, -1) ** 2).sum(axis=1))
    return z / norms.reshape((count,) + (1,) * len(shape))
