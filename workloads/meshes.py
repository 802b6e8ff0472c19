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


def revolution_mesh(profile, n_theta: int, n_phi: int, bc: int = 0) -> Mesh:
    """Closed surface of revolution about the z axis from a profile curve.

    profile(theta) -> (rho, z, drho, dz) for theta in [0, pi]: distance from the axis, height, and
    their derivatives; rho(0) = rho(pi) = 0 (the poles) and rho > 0 in between.  The surface point
    is (rho cos phi, rho sin phi, z).  Rings at theta_i = i pi / n_theta (i = 1 .. n_theta - 1) with
    n_phi vertices each, fans of triangles at the two poles, quads between rings split in two.  Every
    mid-edge node is the surface point at the middle of its edge in the (theta, phi) parameters, so
    all nodes lie on the exact surface; node normals are the exact unit normals t_theta x t_phi
    (pointing away from the enclosed body when the profile runs from the top pole down).
    N = 2 E + 2 with E = 2 (n_theta - 1) n_phi."""
    if n_theta < 2 or n_phi < 3:
        raise ValueError("need n_theta >= 2 and n_phi >= 3")
    index: dict[tuple[int, int], int] = {}
    pts: list[np.ndarray] = []
    nrm: list[np.ndarray] = []

    def node(it2: int, ip2: int) -> int:
        """Node at theta = it2 * pi / (2 n_theta), phi = ip2 * pi / n_phi (half-steps)."""
        if it2 == 0 or it2 == 2 * n_theta:
            key = (it2, 0)
        else:
            key = (it2, ip2 % (2 * n_phi))
        if key not in index:
            th = key[0] * np.pi / (2 * n_theta)
            ph = key[1] * np.pi / n_phi
            rho, z, drho, dz = profile(th)
            if key[0] in (0, 2 * n_theta):
                rho = 0.0
            c, s = np.cos(ph), np.sin(ph)
            p = np.array([rho * c, rho * s, z])
            t_th = np.array([drho * c, drho * s, dz])
            if key[0] in (0, 2 * n_theta):  # the normal on the axis: along +-z
                n = np.array([0.0, 0.0, 1.0 if key[0] == 0 else -1.0])
            else:
                t_ph = np.array([-rho * s, rho * c, 0.0])
                n = np.cross(t_th, t_ph)
            index[key] = len(pts)
            pts.append(p)
            nrm.append(n / np.linalg.norm(n))
        return index[key]

    elems = []

    poles = (0, 2 * n_theta)

    def tri(a, b, c):  # vertices at even half-step coordinates; mid nodes at parametric midpoints
        mids = []
        for p, q in ((a, b), (b, c), (c, a)):
            if p[0] in poles:    # an edge from a pole runs along the ring vertex's meridian
                ip2 = q[1]
            elif q[0] in poles:
                ip2 = p[1]
            else:
                ip2 = (p[1] + q[1]) // 2
            mids.append(node((p[0] + q[0]) // 2, ip2))
        return [node(*a), node(*b), node(*c)] + mids

    for j in range(n_phi):
        j2, j3 = 2 * j, 2 * (j + 1)
        elems.append(tri((0, j2), (2, j2), (2, j3)))                                  # top fan
        elems.append(tri((2 * n_theta, j2), (2 * n_theta - 2, j3), (2 * n_theta - 2, j2)))  # bottom fan
        for i in range(1, n_theta - 1):
            a, b = (2 * i, j2), (2 * i, j3)
            c, d = (2 * i + 2, j2), (2 * i + 2, j3)
            elems.append(tri(a, c, d))
            elems.append(tri(a, d, b))
    nodes = np.array(pts)
    normals = np.array(nrm)
    el = np.array(elems, dtype=np.int64)
    # orient every element so that its geometric normal agrees with the exact normal
    v0, v1, v2 = nodes[el[:, 0]], nodes[el[:, 1]], nodes[el[:, 2]]
    gn = np.cross(v1 - v0, v2 - v0)
    ref = normals[el[:, 0]] + normals[el[:, 1]] + normals[el[:, 2]]
    flip = np.einsum("ij,ij->i", gn, ref) < 0
    el[flip] = el[flip][:, [0, 2, 1, 5, 4, 3]]
    return Mesh(nodes, el.astype(np.int32), normals, np.full(nodes.shape[0], bc, dtype=np.uint8),
                np.zeros(nodes.shape[0], np.int32))


def bowl_profile(theta):
    """The closed generating curve of the paper's acoustic bowl, Eq. (dish), for a = 1:
    xi = sin(theta), eta = 0.2 cos(theta) - 0.6 sin(theta)^2, as (rho, z, drho, dz)."""
    s, c = np.sin(theta), np.cos(theta)
    return s, 0.2 * c - 0.6 * s * s, c, -0.2 * s - 1.2 * s * c


def bowl_mesh(n_theta: int = 48, n_phi: int = 48, tilt: float = 0.15 * np.pi, bc: int = 0) -> Mesh:
    """The hard bowl of Sec. 4.2: the curve of Eq. (dish) rotated about its eta axis, with that axis
    turned by `tilt` (radians, about the x axis) away from the propagation direction +z."""
    m = revolution_mesh(bowl_profile, n_theta, n_phi, bc)
    c, s = np.cos(tilt), np.sin(tilt)
    rot = np.array([[1.0, 0.0, 0.0], [0.0, c, s], [0.0, -s, c]])  # e_z -> (0, sin tilt, cos tilt)
    return scale_translate(m, 1.0, (0.0, 0.0, 0.0), rot=rot)


def linear_from_quadratic(m: Mesh) -> Mesh:
    """The linear 3-node mesh on the vertices of a quadratic mesh (flat triangles between the same
    vertices, mid-edge nodes dropped, node numbering compacted in order of first use)."""
    tri = m.elems[:, :3]
    used = np.unique(tri)
    remap = -np.ones(m.N, np.int64)
    remap[used] = np.arange(used.size)
    return Mesh(m.nodes[used].copy(), remap[tri].astype(np.int32), m.normals[used].copy(), m.bc[used].copy(),
                None if m.body is None else m.body[used].copy())


def sphere_profile(theta):
    """The unit sphere as a profile for revolution_mesh: rho = sin t, z = cos t."""
    return np.sin(theta), np.cos(theta), np.cos(theta), -np.sin(theta)


def uv_sphere_linear(n_theta: int = 10, n_phi: int = 43, radius: float = 1.0, bc: int = 0) -> Mesh:
    """Linear 3-node sphere mesh on a latitude-longitude grid: n_theta - 1 rings of n_phi vertices
    and the two poles, E = 2 (n_theta - 1) n_phi flat triangles; the defaults give the 774 linear
    elements and 389 nodes of the paper's cross-check (Sec. 4)."""
    m = linear_from_quadratic(revolution_mesh(sphere_profile, n_theta, n_phi, bc))
    return Mesh(m.nodes * radius, m.elems, m.normals, m.bc, m.body)

