"""Linear 3-node elements (Sec. 4's cross-check: 774 linear elements, 389 nodes) on the CUDA path,
against the oracle's own linear-element discretisation: the reduced system's entries (1e-12 of
max|A|), FP64 solves and fields (1e-10), the mixed field (1e-6); and the paper's statement that
the linear and quadratic results agree to about two significant figures."""
import numpy as np
import pytest
import torch

import oracle
from workloads import uv_sphere_linear, ico_sphere, shell_points, merge_meshes, scale_translate, linear_from_quadratic

pytestmark = pytest.mark.gpu
D = np.array([0.0, 0.0, 1.0])


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_1706_07919_gb300 import binding
    return binding


def _solver(m):
    from paper_1706_07919_gb300 import Solver
    s = Solver(0)
    s.set_geometry_linear(m.nodes, m.elems, m.normals, m.bc)
    s.set_incident_plane_wave(D)
    return s


def test_linear_assembly_matches_oracle(B):
    two = linear_from_quadratic(merge_meshes([scale_translate(ico_sphere(2), 0.8, (0, 0, -1.0), bc=1),
                                              scale_translate(ico_sphere(2), 1.1, (0.3, 0, 1.3), bc=0)]))
    for m in (uv_sphere_linear(8, 16, bc=0), uv_sphere_linear(8, 16, bc=1), two):
        s = _solver(m)
        for k in (0.0, 0.9, 3.7):
            A, b = s.assemble(k)
            Ar, br = oracle.assemble_system_linear(m, k, D)
            assert A.shape == (m.N, m.N)
            assert np.abs(A.cpu().numpy() - Ar).max() <= 1e-12 * np.abs(Ar).max(), k
            if np.abs(br).max() > 0:
                assert rel(b.cpu().numpy(), br) <= 1e-12
            else:
                assert np.abs(b.cpu().numpy()).max() == 0.0
        s.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_linear_solves_and_fields_match_oracle(B, bc):
    m = uv_sphere_linear(bc=bc)  # the paper's 774 elements / 389 nodes
    assert (m.N, m.E) == (389, 774)
    ks = np.array([0.0, 1.25, 2.5, 5.0])
    pts = shell_points(16, 1.2, 3.0, seed=41)
    s = _solver(m)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
    T64 = s.eval_field(xo, ks, surf, B.BIE_MODE_FP64).cpu().numpy()
    T32 = s.eval_field(xo, ks, surf, B.BIE_MODE_MIXED).cpu().numpy()
    sc = surf.cpu().numpy()
    with pytest.raises(B.BieError):
        s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    s.close()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency_linear(m, k, D)
        if bc == 0 and k == 0.0:
            assert np.abs(sc[i]).max() == 0.0
            continue
        assert rel(np.concatenate(sc[i]), np.concatenate([P, Pn])) <= 1e-10, k
        Tr = oracle.field_linear(m, k, P, Pn, pts)
        assert rel(T64[i], Tr) <= 1e-10 and rel(T32[i], Tr) <= 1e-6, k


def test_linear_and_quadratic_agree_to_two_figures(B):
    """The paper's cross-check on the soft sphere: 389-node linear against 1002-node quadratic,
    scattered field at (0,0,-1.1a) and (0,0,-4a) for the pulse's wavenumbers m = 4, 8, 12
    (k_m a = 2 pi m / 20.1): within 5 % (measured 1.0 - 3.1 %)."""
    from paper_1706_07919_gb300 import Solver
    ks = 2 * np.pi * np.array([4, 8, 12]) / 20.1
    pts = torch.tensor([[0.0, 0.0, -1.1], [0.0, 0.0, -4.0]], dtype=torch.float64, device="cuda:0")
    ml = uv_sphere_linear(bc=1)
    s = _solver(ml)
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    Tl = s.eval_field(pts, ks, surf, B.BIE_MODE_FP64).cpu().numpy()
    s.close()
    mq = ico_sphere(5, bc=1)
    s = Solver(0)
    s.set_geometry(mq.nodes, mq.elems, mq.normals, mq.bc)
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    Tq = s.eval_field(pts, ks, surf, B.BIE_MODE_MIXED).cpu().numpy()
    s.close()
    d = np.abs(Tl - Tq) / np.abs(Tq)
    print("linear vs quadratic, relative difference:", d.ravel())
    assert d.max() < 5e-2
