"""The mixed path at the lattice workload's full size (32 sound-soft spheres, N = 20 544): the
CPU oracle cannot solve a system of this size in a test, so it checks what it can compute one by
one -- sampled rows of the system, against which the GPU solution's per-row backward error must
stay within the mixed path's bar, and the field at sampled points from the GPU's surface solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def lattice():
    return W.config_lattice_large(Nk=2048, grid=16)


def test_large_lattice_rows_and_field(lattice):
    from paper_1706_07919_gb300 import Solver
    from paper_1706_07919_gb300 import binding as B
    w = lattice
    m = w.mesh
    assert m.N == 20544
    ks = w.k[[255, 640, 1023]]  # ka = 1.5, 3.75, 6; three: the two-wavenumber assembly's last group is ragged
    s = Solver(0)
    s.set_geometry(m.nodes, m.elems, m.normals, m.bc)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    pts = w.xobs[np.random.default_rng(5002).choice(w.xobs.shape[0], 4, replace=False)]
    T = s.eval_field(torch.tensor(pts, device="cuda"), ks, surf, B.BIE_MODE_MIXED).cpu().numpy()
    surf = surf.cpu().numpy()
    s.close()
    rows = np.sort(np.random.default_rng(5001).choice(m.N, 6, replace=False))
    for i, k in enumerate(ks):
        assert rep[i].backward_err <= 1e-10
        A, b = oracle.assemble_rows(m, k, [0.0, 0.0, 1.0], rows)
        x = surf[i, 1]  # all nodes soft: the unknown is dP/dnu
        r = A @ x - b
        berr = np.abs(r) / (np.abs(A) @ np.abs(x) + np.abs(b))
        assert berr.max() <= 1e-6, (k, berr)
        # the known boundary values: P = -exp(i k d.x) on every node
        assert np.allclose(surf[i, 0], -np.exp(1j * k * m.nodes[:, 2]), rtol=0, atol=1e-12)
        Tr = oracle.field(m, k, surf[i, 0], surf[i, 1], pts)
        assert np.linalg.norm(T[i] - Tr) / np.linalg.norm(Tr) <= 1e-6
