"""Surface meshes of quadratic 6-node triangles for the test bodies.

Element node order: v0 v1 v2 m01 m12 m20 (three vertices, then the mid-edge nodes of
edges 0-1, 1-2, 2-0), counter-clockwise when seen from the fluid, so that the cross
product of the parametric tangents points out of the body into the fluid.  Vertices and
mid-edge nodes lie on the exact surface; node normals are the exact surface normals
(unit, into the fluid).  Boundary-condition codes per node: 0 = sound-hard, 1 = sound-soft.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    nodes: np.ndarray          # float64 [N, 3]
    elems: np.ndarray          # int32   [E, 6]
    normals: np.ndarray        # float64 [N, 3], unit, pointing into the fluid
    bc: np.ndarray             # uint8   [N], 0 = hard, 1 = soft
    body: np.ndarray = field(default=None)  # int32 [N], body index of each node

    @property
    def N(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def E(self) -> int:
        return int(self.elems.shape[0])

    def contiguous(self) -> "Mesh":
        return Mesh(np.ascontiguousarray(self.nodes, dtype=np.float64),
                    np.ascontiguousarray(self.elems, dtype=np.int32),
                    np.ascontiguousarray(self.normals, dtype=np.float64),
                    np.ascontiguousarray(self.bc, dtype=np.uint8),
                    None if self.body is None else np.ascontiguousarray(self.body, dtype=np.int32))


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _quadratic_from_flat(verts: np.ndarray, tris: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Add one mid-edge node per unique edge, projected onto the unit sphere."""
    edge_id: dict[tuple[int, int], int] = {}
    mids: list[np.ndarray] = []
    nv = verts.shape[0]
    elems = np.empty((tris.shape[0], 6), dtype=np.int64)
    for t, (a, b, c) in enumerate(tris):
        ids = []
        for p, q in ((a, b), (b, c), (c, a)):
            key = (min(p, q), max(p, q))
            if key not in edge_id:
                edge_id[key] = nv + len(mids)
                mids.append(_unit(verts[p] + verts[q]))
            ids.append(edge_id[key])
        elems[t] = (a, b, c, ids[0], ids[1], ids[2])
    nodes = np.concatenate([verts, np.array(mids).reshape(-1, 3)], axis=0)
    return nodes, elems


def _orient_outward(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    tris = tris.copy()
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(v1 - v0, v2 - v0)
    flip = np.einsum("ij,ij->i", n, v0 + v1 + v2) < 0
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return tris


def _dedupe(points: list[np.ndarray]) -> tuple[np.ndarray, dict]:
    index: dict[tuple, int] = {}
    out: list[np.ndarray] = []
    for p in points:
        key = tuple(np.round(p, 9))
        if key not in index:
            index[key] = len(out)
            out.append(p)
    return np.array(out), index


def octa_sphere(levels: int, radius: float = 1.0, bc: int = 0) -> Mesh:
    """Unit octahedron refined `levels` times (each triangle into four), projected onto the
    sphere: 8*4**levels quadratic elements, 2*E + 2 nodes (levels=2: 128 elements, 258 nodes)."""
    verts = [np.array(v, dtype=np.float64) for v in
             ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
    tris = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4), (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    verts_arr = np.array(verts)
    for _ in range(levels):
        cache: dict[tuple[int, int], int] = {}
        vl = list(verts_arr)

        def mid(p: int, q: int) -> int:
            key = (min(p, q), max(p, q))
            if key not in cache:
                cache[key] = len(vl)
                vl.append(_unit(vl[p] + vl[q]))
            return cache[key]

        new = []
        for a, b, c in tris:
            ab, bc_, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [(a, ab, ca), (ab, b, bc_), (ca, bc_, c), (ab, bc_, ca)]
        tris, verts_arr = new, np.array(vl)
    tri = _orient_outward(verts_arr, np.array(tris, dtype=np.int64))
    nodes, elems = _quadratic_from_flat(verts_arr, tri)
    normals = _unit(nodes)
    return Mesh(nodes * radius, elems.astype(np.int32), normals,
                np.full(nodes.shape[0], bc, dtype=np.uint8), np.zeros(nodes.shape[0], np.int32))


def ico_sphere(freq: int, radius: float = 1.0, bc: int = 0) -> Mesh:
    """Icosahedron with every face split into freq**2 triangles (geodesic grid), projected
    onto the sphere: E = 20*freq**2 quadratic elements, N = 40*freq**2 + 2 nodes
    (freq 4: 642, 5: 1002, 6: 1442, 8: 2562)."""
    t = (1.0 + 5 ** 0.5) / 2.0
    ico = _unit(np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
                          (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)],
                         dtype=np.float64))
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    pts: list[np.ndarray] = []
    face_grid = []
    for a, b, c in faces:
        A, B, C = ico[a], ico[b], ico[c]
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                p = _unit((A * (freq - i - j) + B * i + C * j) / freq)
                grid[(i, j)] = len(pts)
                pts.append(p)
        face_grid.append(grid)
    verts, index = _dedupe(pts)
    remap = np.array([index[tuple(np.round(p, 9))] for p in pts])
    tris = []
    for grid in face_grid:
        for i in range(freq):
            for j in range(freq - i):
                tris.append((remap[grid[(i, j)]], remap[grid[(i + 1, j)]], remap[grid[(i, j + 1)]]))
                if i + j + 1 < freq:
                    tris.append((remap[grid[(i + 1, j)]], remap[grid[(i + 1, j + 1)]],
                                 remap[grid[(i, j + 1)]]))
    tri = _orient_outward(verts, np.array(tris, dtype=np.int64))
    nodes, elems = _quadratic_from_flat(verts, tri)
    normals = _unit(nodes)
    return Mesh(nodes * radius, elems.astype(np.int32), normals,
                np.full(nodes.shape[0], bc, dtype=np.uint8), np.zeros(nodes.shape[0], np.int32))


def ellipsoid_from_sphere(m: Mesh, axes: tuple[float, float, float]) -> Mesh:
    """Map a unit-sphere mesh onto the ellipsoid x^2/a^2 + y^2/b^2 + z^2/c^2 = 1 (nodes stay on
    the exact surface); normals are the exact ellipsoid normals."""
    ax = np.asarray(axes, dtype=np.float64)
    unit = m.nodes / np.linalg.norm(m.nodes, axis=1, keepdims=True)
    nodes = unit * ax
    normals = _unit(nodes / ax ** 2)
    return Mesh(nodes, m.elems.copy(), normals, m.bc.copy(), None if m.body is None else m.body.copy())


def scale_translate(m: Mesh, scale: float = 1.0, shift=(0.0, 0.0, 0.0), rot: np.ndarray | None = None,
                    bc: int | None = None) -> Mesh:
    nodes = m.nodes * scale
    normals = m.normals.copy()
    if rot is not None:
        nodes = nodes @ rot.T
        normals = normals @ rot.T
    nodes = nodes + np.asarray(shift, dtype=np.float64)
    bcs = m.bc.copy() if bc is None else np.full(m.N, bc, dtype=np.uint8)
    return Mesh(nodes, m.elems.copy(), normals, bcs, None if m.body is None else m.body.copy())


def merge_meshes(meshes: list[Mesh]) -> Mesh:
    nodes, elems, normals, bcs, body = [], [], [], [], []
    off = 0
    for b, m in enumerate(meshes):
        nodes.append(m.nodes)
        elems.append(m.elems.astype(np.int64) + off)
        normals.append(m.normals)
        bcs.append(m.bc)
        body.append(np.full(m.N, b, dtype=np.int32))
        off += m.N
    return Mesh(np.concatenate(nodes), np.concatenate(elems).astype(np.int32), np.concatenate(normals),
                np.concatenate(bcs), np.concatenate(body))
