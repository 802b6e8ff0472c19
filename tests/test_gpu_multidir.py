"""Several incident directions on one factor per wavenumber (Sec. 5: the solution matrix is kept
and only the incident wave changes), through bie_solve_frequencies_multi, against the CPU FP64
oracle solved separately for each direction.  Bars: FP64 path 1e-10, mixed path 1e-6."""
import numpy as np
import pytest
import torch

import oracle
from workloads import octa_sphere, ico_sphere, merge_meshes, scale_translate

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_1706_07919_gb300 import binding
    return binding


def _dirs():
    d = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.3, -0.5, 0.8], [0.0, -1.0, -1.0]])
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _meshes():
    s0 = ico_sphere(2)
    mixed = merge_meshes([scale_translate(s0, 0.8, (0, 0, -1.0), bc=1), scale_translate(s0, 1.1, (0.3, 0, 1.3), bc=0)])
    return [octa_sphere(2, bc=0), octa_sphere(2, bc=1), mixed]


@pytest.mark.parametrize("mode,tol", [(0, 1e-10), (1, 1e-6)])
def test_directions_share_the_factor(B, mode, tol):
    from paper_1706_07919_gb300 import Solver
    dirs = _dirs()
    ks = np.array([0.0, 0.7, 2.3, 4.1, 5.6])
    for m in _meshes():
        s = Solver(0)
        s.set_geometry(m.nodes, m.elems, m.normals, m.bc)
        surf, rep = s.solve_frequencies_multi(ks, dirs, mode)
        single, _ = s.solve_frequencies(ks, mode)  # the context's direction: +z, dirs[0]
        surf, single = surf.cpu().numpy(), single.cpu().numpy()
        s.close()
        assert len(rep) == len(ks) * len(dirs)
        for i, k in enumerate(ks):
            if np.abs(single[i]).max() == 0.0:  # a hard body at k = 0 scatters nothing
                assert np.abs(surf[i]).max() == 0.0
                continue
            assert rel(surf[i, 0], single[i]) <= tol
            for d, dv in enumerate(dirs):
                P, Pn = oracle.solve_frequency(m, k, dv)
                got = np.concatenate([surf[i, d, 0], surf[i, d, 1]])
                assert rel(got, np.concatenate([P, Pn])) <= tol, (k, d, rep[i * len(dirs) + d].flags)


def test_directions_with_reassembled_wavenumbers(B):
    """Every wavenumber flagged (tiny threshold): the FP64 re-assembly runs per direction."""
    from paper_1706_07919_gb300 import Solver
    dirs = _dirs()[:3]
    m = _meshes()[2]
    ks = np.array([1.1, 3.3])
    s = Solver(0)
    s.set_geometry(m.nodes, m.elems, m.normals, m.bc)
    s.set_option("mixed.fallback_err_est", 1e-30)
    surf, rep = s.solve_frequencies_multi(ks, dirs, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    s.close()
    for i, k in enumerate(ks):
        for d, dv in enumerate(dirs):
            assert rep[i * len(dirs) + d].flags & B.BIE_FLAG_FP64_ASSEMBLY
            P, Pn = oracle.solve_frequency(m, k, dv)
            assert rel(np.concatenate([surf[i, d, 0], surf[i, d, 1]]), np.concatenate([P, Pn])) <= 1e-8
