"""Empty and degenerate inputs through every call of the path (Sec. 4's pipeline: frequency solves,
field, spectra, synthesis): nothing is launched for an empty dimension, the outputs keep their
shapes, and a synthesis without frequencies is exactly zero.  Then the smallest non-empty cases:
one wavenumber on a tiny mesh through each solve entry point, one observation point, one pulse of
two samples, each checked against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from workloads import octa_sphere

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


@pytest.fixture(scope="module")
def Solver(B):
    from paper_1706_07919_gb300 import Solver as S
    return S


@pytest.fixture(scope="module")
def mesh():
    return octa_sphere(1)


def _solver(Solver, m):
    s = Solver(0)
    s.set_geometry(m.nodes, m.elems, m.normals, m.bc)
    s.set_incident_plane_wave(D)
    return s


def test_empty_dimensions(Solver, B, mesh):
    s = _solver(Solver, mesh)
    k0 = np.zeros(0)
    for mode in (B.BIE_MODE_FP64, B.BIE_MODE_MIXED):
        surf, rep = s.solve_frequencies(k0, mode)
        assert tuple(surf.shape) == (0, 2, mesh.N) and rep == []
    surf, pending = s.solve_frequencies_async(k0)
    assert tuple(surf.shape) == (0, 2, mesh.N) and pending.reports() == []
    sm, rm = s.solve_frequencies_multi(k0, np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]]), B.BIE_MODE_MIXED)
    assert tuple(sm.shape) == (0, 2, 2, mesh.N) and rm == []
    # field: no points, or no wavenumbers
    ks = np.array([1.3])
    surf1, _ = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    for mode in (B.BIE_MODE_FP64, B.BIE_MODE_MIXED):
        T = s.eval_field(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), ks, surf1, mode)
        assert tuple(T.shape) == (1, 0)
        xo = torch.tensor([[0.0, 0.0, 3.0]], dtype=torch.float64, device="cuda")
        T = s.eval_field(xo, k0, torch.zeros((0, 2, mesh.N), dtype=torch.complex128, device="cuda"), mode)
        assert tuple(T.shape) == (0, 1)
    # spectra of no pulses; a synthesis without frequencies is zero; no points gives no samples
    Nt = 16
    S0 = s.pulse_spectrum(torch.zeros((0, Nt), dtype=torch.float64, device="cuda"))
    assert tuple(S0.shape) == (0, Nt // 2 + 1)
    S = s.pulse_spectrum(torch.ones((2, Nt), dtype=torch.float64, device="cuda"))
    M = 3
    for dt in (torch.float64, torch.float32):
        out = s.synthesize(torch.zeros((0, M), dtype=torch.complex128, device="cuda"), np.zeros(0, np.int64), S, Nt, dt)
        assert tuple(out.shape) == (2, M, Nt) and not out.abs().max().item()
    out = s.synthesize(torch.zeros((1, 0), dtype=torch.complex128, device="cuda"), np.array([1]), S, Nt)
    assert tuple(out.shape) == (2, 0, Nt)
    assert s.top_frequencies(S, Nt, 0).shape[0] == 0
    s.close()


def test_smallest_cases_against_oracle(Solver, B, mesh):
    """One wavenumber through each solve call, one observation point, one two-sample pulse."""
    s = _solver(Solver, mesh)
    k = np.array([2.2])
    P, Pn = oracle.solve_frequency(mesh, k[0], D)
    a, _ = s.solve_frequencies(k, B.BIE_MODE_FP64)
    b, _ = s.solve_frequencies(k, B.BIE_MODE_MIXED)
    c, pending = s.solve_frequencies_async(k)
    rep = pending.reports()
    d, _ = s.solve_frequencies_multi(k, D[None, :], B.BIE_MODE_MIXED)
    assert rel(a.cpu().numpy()[0, 0], P) <= 1e-10
    for x in (b.cpu().numpy()[0, 0], c.cpu().numpy()[0, 0], d.cpu().numpy()[0, 0, 0]):
        assert rel(x, P) <= 1e-6
    assert rep[0].path == B.BIE_MODE_MIXED and not rep[0].flags & B.BIE_FLAG_NOT_CONVERGED
    xs = np.array([[0.3, -0.2, 2.5]])
    T = s.eval_field(torch.tensor(xs, device="cuda"), k, a, B.BIE_MODE_FP64).cpu().numpy()
    Tr = oracle.field(mesh, k[0], P, Pn, xs)
    assert rel(T[0], Tr) <= 1e-10
    # Nt = 2: the spectrum is (s0 + s1, s0 - s1); the synthesis of m = 1 alone is S_1 T (-1)^t / 2
    sig = torch.tensor([[0.7, -0.1]], dtype=torch.float64, device="cuda")
    S = s.pulse_spectrum(sig)
    assert np.allclose(S.cpu().numpy(), [[0.6, 0.8]], atol=1e-15)
    Tm = torch.tensor([[0.5 - 0.25j]], dtype=torch.complex128, device="cuda")
    out = s.synthesize(Tm, np.array([1]), S, 2).cpu().numpy()
    want = np.real(0.8 * (0.5 - 0.25j)) * np.array([1.0, -1.0]) / 2.0
    ref = oracle.synthesize(np.array([[0.5 - 0.25j]]), np.array([1]), oracle.dft(np.array([0.7, -0.1]))[None, :], 2)
    assert np.allclose(ref[0, 0], want, atol=1e-15)
    assert np.allclose(out[0, 0], want, atol=1e-15), (out, want)
    s.close()
