"""Writes point_source_residuals_lattice.txt: the oracle's residual of the row equation of
Eq. BRIEF (App. B's +4 pi P term included) for the nodal values of two interior point sources on
the 32-sphere lattice (N = 20 544), per body, at k = 0, 6 and 24.

A point source inside a body radiates into the whole exterior, so its nodal values (P, dP/dnu)
satisfy every row equation up to the discretisation error of the method: the residual
r = H u - (4 pi + alpha) u - Gm du - beta du measures that error, and the CUDA path's assembly must
give the same residual at full size over all rows.  Only oracle/ computes here (the sources and the
mesh are inputs); a run takes a few minutes and about 15 GB of host memory.

    python tests/golden/make_point_source_residuals.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SOURCES = [(-1.8 + 0.05, -1.8 - 0.03, -0.6 + 0.08), (1.8 - 0.06, 1.8 + 0.04, 0.6 - 0.05)]
KS = (0.0, 6.0, 24.0)
NODES_PER_BODY = 642


def point_sources(nodes, normals, k, sources):
    """P and dP/dnu at the nodes of the field of unit point sources: sum of e^{ikR}/R."""
    u = np.zeros(nodes.shape[0], complex)
    du = np.zeros(nodes.shape[0], complex)
    for s in sources:
        r = nodes - np.asarray(s)
        R = np.linalg.norm(r, axis=1)
        e = np.exp(1j * k * R)
        u += e / R
        du += e * (1j * k * R - 1.0) * np.einsum("ij,ij->i", r, normals) / R ** 3
    return u, du


def main():
    m = W.config_lattice_large(Nk=2048, grid=16).mesh
    assert m.N == 32 * NODES_PER_BODY
    lines = ["# Oracle residual of the row equation of Eq. BRIEF (with App. B's +4 pi P term) for two",
             "# interior unit point sources on the 32-sphere lattice (N = 20544), written by",
             "# make_point_source_residuals.py (oracle only).  Sources: " + repr(SOURCES) + ".",
             "# columns: k  body  |r_body| / (4 pi |u|)   (body -1: all rows; u over all nodes)"]
    for k in KS:
        H, Gm, al, be = oracle.assemble_raw(m, k)
        u, du = point_sources(m.nodes, m.normals, k, SOURCES)
        r = H @ u - (4 * np.pi + al) * u - Gm @ du - be * du
        del H, Gm
        scale = 4 * np.pi * np.linalg.norm(u)
        lines.append(f"{k:g} -1 {np.linalg.norm(r) / scale:.12e}")
        for b in range(32):
            rb = r[b * NODES_PER_BODY:(b + 1) * NODES_PER_BODY]
            lines.append(f"{k:g} {b} {np.linalg.norm(rb) / scale:.12e}")
        print(lines[-33], flush=True)
    with open(os.path.join(HERE, "point_source_residuals_lattice.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
