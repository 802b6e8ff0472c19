"""Parity of the FP64 CUDA path (through the C ABI) with the CPU FP64 oracle on the same seeded
inputs.  Bar: relative L2 <= 1e-10 (the FP64 path's tolerance); assembly entries <= 1e-12."""
import numpy as np
import pytest
import torch

import oracle
from workloads import (octa_sphere, ico_sphere, merge_meshes, scale_translate, shell_points, gaussian_pulse,
                       config_sphere_fp64)

pytestmark = pytest.mark.gpu
D = np.array([0.0, 0.0, 1.0])
TOL = 1e-10


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


def _solver(Solver, mesh, d=D, ng=None):
    s = Solver(0)
    if ng is not None:
        s.set_quadrature(*ng)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    s.set_incident_plane_wave(d)
    return s


@pytest.mark.parametrize("L,k", [(1, 0.5), (2, 3.0), (2, 7.875)])
def test_assembly_matches_oracle(Solver, L, k):
    m = octa_sphere(L)
    s = _solver(Solver, m)
    A, b = s.assemble(k)
    Ar, br = oracle.assemble_system(m, k, D)
    assert np.abs(A.cpu().numpy() - Ar).max() <= 1e-12 * np.abs(Ar).max()
    assert rel(b.cpu().numpy(), br) <= 1e-12


@pytest.mark.parametrize("L,k", [(1, 0.5), (2, 7.875), (3, 15.9)])
def test_float_float_bulk_assembly_matches_oracle(Solver, L, k):
    """The float-float bulk assembly (used to re-assemble flagged wavenumbers) meets the FP64 bar."""
    m = octa_sphere(L)
    s = _solver(Solver, m)
    s.set_option("assemble.bulk_ff", 1)
    A, b = s.assemble(k)
    s.set_option("assemble.bulk_ff", 0)
    A64, b64 = s.assemble(k)
    Ar, br = oracle.assemble_system(m, k, D)
    A, A64 = A.cpu().numpy(), A64.cpu().numpy()
    assert np.abs(A - Ar).max() <= 1e-12 * np.abs(Ar).max()
    assert rel(b.cpu().numpy(), br) <= 1e-12
    assert np.abs(A - A64).max() <= 1e-12 * np.abs(Ar).max()


def test_assembly_mixed_bc_two_bodies_and_custom_rule(Solver):
    s0 = ico_sphere(2)
    m = merge_meshes([scale_translate(s0, 0.8, (0, 0, -1.0), bc=1), scale_translate(s0, 1.1, (0.3, 0, 1.3), bc=0)])
    d = np.array([0.3, -0.2, 1.0]); d /= np.linalg.norm(d)
    s = _solver(Solver, m, d, ng=(3, 5))
    for k in (0.9, 4.2):
        A, b = s.assemble(k)
        Ar, br = oracle.assemble_system(m, k, d, ng=3, ng_near=5)
        assert np.abs(A.cpu().numpy() - Ar).max() <= 1e-12 * np.abs(Ar).max()
        assert rel(b.cpu().numpy(), br) <= 1e-12


def test_fp64_solves_all_sphere_wavenumbers(Solver, B):
    w = config_sphere_fp64()
    s = _solver(Solver, w.mesh)
    surf, rep = s.solve_frequencies(w.k, B.BIE_MODE_FP64)
    surf = surf.cpu().numpy()
    worst = 0.0
    for i, k in enumerate(w.k):
        P, Pn = oracle.solve_frequency(w.mesh, k, D)
        worst = max(worst, rel(surf[i, 0], P))
        assert rep[i].flags == 0
    assert worst <= TOL, worst


def test_fp64_solve_soft_and_ragged(Solver, B):
    # 66 nodes (ragged against every tile size), soft body, tiny and large k in one call
    m = octa_sphere(1, bc=1)
    ks = np.array([1e-3, 0.37, 5.1])
    s = _solver(Solver, m)
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(m, k, D)
        assert rel(surf[i, 1], Pn) <= TOL
        np.testing.assert_allclose(surf[i, 0], P, rtol=0, atol=1e-14)


def test_default_normals_match_oracle_with_same_normals(Solver, B):
    m = octa_sphere(1)
    s = Solver(0)
    s.set_geometry(m.nodes, m.elems, None, m.bc)
    A, b = s.assemble(1.3)
    # the library's averaged normals are not returned; the solve must still be accurate vs series
    import analytic_sphere as an
    surf, _ = s.solve_frequencies(np.array([1.0]), B.BIE_MODE_FP64)
    ex = an.scattered(m.nodes, 1.0, hard=True)
    assert rel(surf.cpu().numpy()[0, 0], ex) < 0.05


def test_field_matches_oracle(Solver, B):
    w = config_sphere_fp64()
    s = _solver(Solver, w.mesh)
    ks = w.k[[0, 17, 35, 63]]
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    xo = torch.tensor(w.xobs, dtype=torch.float64, device="cuda")
    T = s.eval_field(xo, ks, surf, B.BIE_MODE_FP64).cpu().numpy()
    sn = surf.cpu().numpy()
    for i, k in enumerate(ks):
        Tr = oracle.field(w.mesh, k, sn[i, 0], sn[i, 1], w.xobs)
        assert rel(T[i], Tr) <= TOL


def test_foot_points_edge_cases(Solver, B):
    # points very close to nodes, on the axis and far away
    m = octa_sphere(2)
    pts = np.concatenate([m.nodes[:5] * 1.0001, np.array([[0, 0, 7.0], [0, 0, -1.05], [3.0, -2.0, 0.5]])])
    s = _solver(Solver, m)
    surf, _ = s.solve_frequencies(np.array([2.0]), B.BIE_MODE_FP64)
    T = s.eval_field(torch.tensor(pts, device="cuda"), np.array([2.0]), surf, B.BIE_MODE_FP64).cpu().numpy()
    sn = surf.cpu().numpy()
    Tr = oracle.field(m, 2.0, sn[0, 0], sn[0, 1], pts)
    assert rel(T[0], Tr) <= 1e-9


def test_pulse_spectrum_and_synthesis(Solver, B):
    s = Solver(0)
    for Nt in (2, 64, 256, 1024):
        T = 2 * np.pi / 0.125
        pulses = np.stack([gaussian_pulse(Nt, T, 0.5, 8.0), np.random.default_rng(Nt).standard_normal(Nt)])
        S = s.pulse_spectrum(torch.tensor(pulses, device="cuda")).cpu().numpy()
        for p in range(2):
            Sr = oracle.dft(pulses[p])[: Nt // 2 + 1]
            assert np.abs(S[p] - Sr).max() <= 1e-12 * np.abs(Sr).max()
    Nt, M = 256, 37
    rng = np.random.default_rng(5)
    midx = np.array([0, 1, 5, 64, 127, 128])
    Tm = rng.standard_normal((len(midx), M)) + 1j * rng.standard_normal((len(midx), M))
    sig = rng.standard_normal((3, Nt))
    Sfull = np.stack([oracle.dft(x) for x in sig])
    ref = oracle.synthesize(Tm, midx, Sfull, Nt)
    Sd = torch.tensor(Sfull[:, : Nt // 2 + 1], device="cuda")
    Td = torch.tensor(Tm, device="cuda")
    out64 = s.synthesize(Td, midx, Sd, Nt, torch.float64).cpu().numpy()
    assert np.abs(out64 - ref).max() <= 1e-12 * np.abs(ref).max()
    out32 = s.synthesize(Td, midx, Sd, Nt, torch.float32).cpu().numpy()
    assert np.abs(out32 - ref).max() <= 1e-5 * np.abs(ref).max()


def test_end_to_end_sphere_space_time(Solver, B):
    """The whole FP64 path on the 258-node sphere (64 k, 256 time steps) on 200 of its points."""
    w = config_sphere_fp64()
    xsub = w.xobs[::5]
    s = _solver(Solver, w.mesh)
    surf, _ = s.solve_frequencies(w.k, B.BIE_MODE_FP64)
    xo = torch.tensor(xsub, device="cuda")
    T = s.eval_field(xo, w.k, surf, B.BIE_MODE_FP64)
    S = s.pulse_spectrum(torch.tensor(w.pulses, device="cuda"))
    midx = np.arange(1, len(w.k) + 1)
    p = s.synthesize(T, midx, S, w.Nt, torch.float64).cpu().numpy()
    sn = surf.cpu().numpy()
    Tr = np.stack([oracle.field(w.mesh, k, sn[i, 0], sn[i, 1], xsub) for i, k in enumerate(w.k)])
    pr = oracle.synthesize(Tr, midx, oracle.dft(w.pulses[0])[None, :], w.Nt)
    assert rel(p, pr) <= TOL


def test_errors_are_reported(Solver, B):
    s = Solver(0)
    with pytest.raises(B.BieError) as e:
        s.solve_frequencies(np.array([1.0]))
    assert e.value.code == B.BIE_ERR_STATE
    m = octa_sphere(1)
    bad = m.elems.copy()
    bad[3, 2] = m.N + 5
    with pytest.raises(B.BieError) as e:
        s.set_geometry(m.nodes, bad, m.normals, m.bc)
    assert e.value.code == B.BIE_ERR_INVALID_ARG
    s.set_geometry(m.nodes, m.elems, m.normals, m.bc)
    with pytest.raises(B.BieError) as e:
        s.solve_frequencies(np.array([1.0, -2.0]))
    assert e.value.code == B.BIE_ERR_INVALID_ARG and "k[1]" in str(e.value)
    nodes = m.nodes.copy()
    nodes[0, 0] = np.nan
    with pytest.raises(B.BieError):
        s.set_geometry(nodes, m.elems, m.normals, m.bc)
