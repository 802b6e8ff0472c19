"""Parity of the mixed-precision CUDA path (FP32 assembly with float-float phases, FP32/TF32 LU,
float-float iterative refinement) with the CPU FP64 oracle.  Bar: relative L2 <= 1e-6 per
wavenumber for surface solutions and for fields (the mixed path's tolerance)."""
import numpy as np
import pytest
import torch

import oracle
from workloads import octa_sphere, ico_sphere, merge_meshes, scale_translate, config_sphere_fp64, plane_grid_points

pytestmark = pytest.mark.gpu
D = np.array([0.0, 0.0, 1.0])
TOL = 1e-6


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


def _solver(Solver, mesh, d=D, tc=None):
    s = Solver(0)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    s.set_incident_plane_wave(d)
    if tc is not None:
        s.set_option("mixed.tcgen05", tc)
    return s


@pytest.fixture(scope="module")
def two_spheres():
    s0 = ico_sphere(4)
    return merge_meshes([scale_translate(s0, 1.0, (0, 0, -1.05)), scale_translate(s0, 1.0, (0, 0, 1.05))])


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_mixed_sphere_all_wavenumbers(Solver, B, tc):
    w = config_sphere_fp64()
    s = _solver(Solver, w.mesh, tc=tc)
    surf, rep = s.solve_frequencies(w.k, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    errs = []
    for i, k in enumerate(w.k):
        P, Pn = oracle.solve_frequency(w.mesh, k, D)
        errs.append(rel(surf[i, 0], P))
        assert rep[i].backward_err <= 1e-10 or rep[i].flags & B.BIE_FLAG_FALLBACK_FP64, (k, rep[i].backward_err)
    assert max(errs) <= TOL, (max(errs), int(np.argmax(errs)))
    # only the wavenumbers next to interior resonances (j_n zeros near 3.14, 4.49, 5.76, 6.99, 7.73)
    # may leave the mixed path, and never because the refinement failed
    fell = [i for i in range(len(w.k)) if rep[i].flags & B.BIE_FLAG_FP64_ASSEMBLY]
    assert len(fell) <= 6, [(w.k[i], rep[i].err_est) for i in fell]
    assert all(not (rep[i].flags & (B.BIE_FLAG_NOT_CONVERGED | B.BIE_FLAG_FALLBACK_FP64)) for i in range(len(w.k)))


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_mixed_two_spheres_high_k(Solver, B, two_spheres, tc):
    ks = np.array([0.5, 4.0, 9.3, 16.0])
    s = _solver(Solver, two_spheres, tc=tc)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(two_spheres, k, D)
        assert rel(surf[i, 0], P) <= TOL, (k, rel(surf[i, 0], P), rep[i].iters)
        assert rep[i].iters <= 8 and rep[i].flags == 0, (k, rep[i].iters, rep[i].flags, rep[i].err_est)


@pytest.mark.parametrize("tc", [0, 1, 2, 3])
def test_unrefined_lu_accuracy(Solver, B, two_spheres, tc):
    """With refinement switched off the answer is the low-precision factor's: FP32 (SIMT) or
    TF32 (tensor cores) rounding times the condition number -- a broken update would be O(1)."""
    ks = np.array([2.0, 11.0])
    s = _solver(Solver, two_spheres, tc=tc)
    s.set_option("refine.it_max", 0)
    s.set_option("mixed.fallback_err_est", 1.0)
    s.set_option("refine.tol", 0.5)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(two_spheres, k, D)
        e = rel(surf[i, 0], P)
        assert e <= (1e-5 if tc == 0 else 2e-2), (k, e)


def test_mixed_soft_ragged_and_batch_edges(Solver, B):
    m = octa_sphere(1, bc=1)
    ks = np.array([0.01, 0.6, 2.2, 6.1, 7.7])
    s = _solver(Solver, m)
    s.set_option("mixed.batch", 2)  # ragged last batch
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(m, k, D)
        assert rel(surf[i, 1], Pn) <= TOL


@pytest.mark.parametrize("variant", [2, 1, 0])
def test_mixed_field_uniform_groups_match_oracle(Solver, B, two_spheres, variant):
    """Uniformly spaced wavenumbers (groups of 16 and a ragged remainder of 8) take the phase
    recurrence of the field kernel; smooth synthetic surface data isolates the field evaluation."""
    xs = plane_grid_points(7, 5.0, 0.0)
    ks = 12.0 + 0.03125 * np.arange(40)
    s = _solver(Solver, two_spheres)
    s.set_option("field.variant", variant)
    x = two_spheres.nodes
    surf = np.zeros((len(ks), 2, two_spheres.N), complex)
    for i, k in enumerate(ks):
        surf[i, 0] = np.exp(1j * k * x[:, 2]) * (1.0 + 0.3 * np.sin(2.0 * x[:, 0]))
        surf[i, 1] = 1j * k * np.exp(1j * k * x[:, 2]) * (0.5 + 0.2 * np.cos(x[:, 1]))
    T = s.eval_field(torch.tensor(xs, device="cuda"), ks, torch.tensor(surf, device="cuda"), B.BIE_MODE_MIXED)
    T = T.cpu().numpy()
    for i in (0, 7, 15, 16, 19, 31, 32, 39):
        Tr = oracle.field(two_spheres, ks[i], surf[i, 0], surf[i, 1], xs)
        assert rel(T[i], Tr) <= 1e-6, (ks[i], rel(T[i], Tr))


@pytest.mark.parametrize("accurate,bound", [(1, 1e-6), (0, 2e-5)])
def test_mixed_field_matches_oracle(Solver, B, two_spheres, accurate, bound):
    xs = plane_grid_points(9, 5.0, 0.0)
    ks = np.array([1.0, 8.0, 16.0])
    s = _solver(Solver, two_spheres)
    s.set_option("field.accurate_phase", accurate)
    # identical surface data for both sides isolates the field evaluation
    surf = np.zeros((len(ks), 2, two_spheres.N), complex)
    for i, k in enumerate(ks):
        surf[i] = oracle.solve_frequency(two_spheres, k, D)
    T = s.eval_field(torch.tensor(xs, device="cuda"), ks, torch.tensor(surf, device="cuda"), B.BIE_MODE_MIXED)
    T = T.cpu().numpy()
    for i, k in enumerate(ks):
        Tr = oracle.field(two_spheres, k, surf[i, 0], surf[i, 1], xs)
        assert rel(T[i], Tr) <= bound, (k, rel(T[i], Tr))


@pytest.mark.parametrize("ff", [0, 1])
def test_fp64_reassembly_path_reaches_fp64_accuracy(Solver, B, ff):
    """Forcing every wavenumber through the FP64 re-assembly (threshold below any estimate):
    refinement with the TF32 factor against the FP64 system must reach the FP64 path's answer to
    the refinement's FP64 stop (backward error 1e-13) times the condition number."""
    w = config_sphere_fp64()
    ks = w.k[[3, 30, 35, 60]]
    s = _solver(Solver, w.mesh, tc=1)
    s.set_option("mixed.fallback_err_est", 1e-15)
    s.set_option("mixed.reassembly", ff)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        assert rep[i].flags & B.BIE_FLAG_FP64_ASSEMBLY and not rep[i].flags & B.BIE_FLAG_FALLBACK_FP64
        P, Pn = oracle.solve_frequency(w.mesh, k, D)
        assert rel(surf[i, 0], P) <= 1e-8, (k, rel(surf[i, 0], P))


def test_full_fp64_last_resort_reports(Solver, B):
    """Every wavenumber flagged and no correction allowed against its FP64 re-assembly: each one
    ends on the full FP64 path, whose report describes that solve (FALLBACK_FP64, path FP64,
    NOT_CONVERGED cleared), and whose surface values are the FP64 path's."""
    w = config_sphere_fp64()
    ks = w.k[[5, 21, 40]]
    s = _solver(Solver, w.mesh)
    s.set_option("mixed.fallback_err_est", 1e-30)
    s.set_option("mixed.refine64_it_max", 0)
    s.set_option("mixed.refactor32", 0)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    ref, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    surf, ref = surf.cpu().numpy(), ref.cpu().numpy()
    for i in range(len(ks)):
        assert rep[i].flags & B.BIE_FLAG_FALLBACK_FP64 and rep[i].flags & B.BIE_FLAG_FP64_ASSEMBLY, rep[i].flags
        assert not rep[i].flags & B.BIE_FLAG_NOT_CONVERGED and rep[i].path == B.BIE_MODE_FP64, rep[i].flags
        assert rel(surf[i], ref[i]) <= 1e-12, (ks[i], rel(surf[i], ref[i]))
    with pytest.raises(B.BieError):
        s.set_option("mixed.refine64_it_max", 65)


@pytest.mark.parametrize("mesh", ["sphere", "two_spheres"])
def test_fp32_refactorisation_before_the_fp64_path(Solver, B, two_spheres, mesh):
    """Every wavenumber flagged and no correction allowed with the TF32 factor against the FP64
    re-assembly: the FP64 system is factored again in FP32 on the CUDA cores (64-column panels,
    cooperative ones for the two spheres' N = 2884) and refined against itself with that factor.
    Each report carries FP32_REFACTOR on the mixed path (no full FP64 solve), a backward error at
    the FP64 refinement's tolerance, and surface values equal to the FP64 path's within 1e-9; two
    incident directions take the same step per direction."""
    m = config_sphere_fp64().mesh if mesh == "sphere" else two_spheres
    ks = np.array([1.5, 4.49, 7.0])
    s = _solver(Solver, m)
    s.set_option("mixed.fallback_err_est", 1e-30)
    s.set_option("mixed.refine64_it_max", 0)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    ref, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    surf, ref = surf.cpu().numpy(), ref.cpu().numpy()
    for i in range(len(ks)):
        f = rep[i].flags
        assert f & B.BIE_FLAG_FP32_REFACTOR and f & B.BIE_FLAG_FP64_ASSEMBLY, (ks[i], f)
        assert not f & (B.BIE_FLAG_FALLBACK_FP64 | B.BIE_FLAG_NOT_CONVERGED) and rep[i].path == B.BIE_MODE_MIXED, (ks[i], f)
        assert rep[i].backward_err <= 1e-12, (ks[i], rep[i].backward_err)
        assert rel(surf[i], ref[i]) <= 1e-9, (ks[i], rel(surf[i], ref[i]))
    if mesh == "sphere":
        dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
        sd, rd = s.solve_frequencies_multi(ks, dirs, B.BIE_MODE_MIXED)
        sr, _ = s.solve_frequencies_multi(ks, dirs, B.BIE_MODE_FP64)
        sd, sr = sd.cpu().numpy(), sr.cpu().numpy()
        assert all(r.flags & B.BIE_FLAG_FP32_REFACTOR and not r.flags & B.BIE_FLAG_FALLBACK_FP64 for r in rd), [r.flags for r in rd]
        assert rel(sd, sr) <= 1e-9, rel(sd, sr)
    s.close()


def test_pooled_reassembly_across_batches(Solver, B):
    """Every wavenumber flagged, 70 wavenumbers in batches of 8: the flagged systems of all batches
    are pooled (factors, permutations, solutions copied aside) and re-assembled and refined in
    groups when the pool fills and after the last batch; each surface solution must match the FP64
    path's to the FP64 refinement's accuracy and carry the re-assembly flag."""
    w = config_sphere_fp64()
    ks = np.linspace(0.5, 9.5, 70)
    s = _solver(Solver, w.mesh)
    s.set_option("mixed.fallback_err_est", 1e-30)
    s.set_option("mixed.batch", 8)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    ref, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    surf, ref = surf.cpu().numpy(), ref.cpu().numpy()
    for i in range(len(ks)):
        assert rep[i].flags & B.BIE_FLAG_FP64_ASSEMBLY and not rep[i].flags & B.BIE_FLAG_NOT_CONVERGED, i
        assert rel(surf[i, 0], ref[i, 0]) <= 1e-8 and rel(surf[i, 1], ref[i, 1]) <= 1e-8, (ks[i], rel(surf[i, 0], ref[i, 0]))


@pytest.mark.parametrize("kb", [0, 1, 2])
def test_bulk_assembly_variants_match_oracle(Solver, B, two_spheres, kb):
    """The FP32 bulk assembly with one (general kernel, kb 0) or several wavenumbers per thread
    (uniform-condition kernel, kb 1 and 2) gives the oracle's solution; five wavenumbers leave a
    ragged last group of the two-wavenumber kernel, and soft and hard bodies are mixed."""
    m = merge_meshes([scale_translate(ico_sphere(3, bc=1), 0.8, (0, 0, -1.0)),
                      scale_translate(ico_sphere(3), 1.0, (0.1, 0, 1.2))])
    ks = np.array([0.7, 3.3, 6.2, 9.1, 12.5])
    s = _solver(Solver, m)
    s.set_option("mixed.asm_kb", kb)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(m, k, D)
        assert rel(surf[i, 0], P) <= TOL and rel(surf[i, 1], Pn) <= TOL, (k, rep[i].flags)
        assert not (rep[i].flags & (B.BIE_FLAG_NOT_CONVERGED | B.BIE_FLAG_FALLBACK_FP64))


def test_bulk_assembly_element_with_mixed_conditions(Solver, B):
    """An element whose nodes carry different boundary conditions sends the assembly to the
    general kernel even when the multi-wavenumber kernel is selected."""
    m = octa_sphere(2)
    bc = m.bc.copy()
    bc[m.elems[0, :3]] = 1  # the three vertices of element 0 soft, its mid-edge nodes hard
    m.bc = bc
    ks = np.array([1.1, 4.4, 7.3])
    s = _solver(Solver, m)
    s.set_option("mixed.asm_kb", 2)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(m, k, D)
        assert rel(surf[i, 0], P) <= TOL and rel(surf[i, 1], Pn) <= TOL, k


def test_mixed_large_batch_matches_oracle(Solver, B):
    """A batch of 70 systems (at least 64: the LU leaf kernel then updates the panel itself instead
    of a separate launch) gives the oracle's solutions."""
    m = octa_sphere(2)
    ks = 0.11 * np.arange(1, 71)
    s = _solver(Solver, m)
    s.set_option("mixed.batch", 128)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i in range(0, 70, 3):
        P, Pn = oracle.solve_frequency(m, ks[i], D)
        assert rel(surf[i, 0], P) <= TOL, (ks[i], rel(surf[i, 0], P))
    assert all(not (r.flags & B.BIE_FLAG_NOT_CONVERGED) for r in rep)


@pytest.mark.parametrize("block", [128, 512])
def test_mixed_lu_block_variants(Solver, B, two_spheres, block):
    """The deferred tensor-core update over 128- or 512-column blocks (N = 1284: whole blocks and a
    ragged last one) gives the oracle's solutions with few refinement corrections."""
    ks = np.array([1.5, 8.0])
    s = _solver(Solver, two_spheres, tc=3)
    s.set_option("mixed.lu_block", block)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(two_spheres, k, D)
        assert rel(surf[i, 0], P) <= TOL, (k, rel(surf[i, 0], P))
        assert rep[i].iters <= 8 and not (rep[i].flags & B.BIE_FLAG_NOT_CONVERGED), (k, rep[i].iters)
    with pytest.raises(B.BieError):
        s.set_option("mixed.lu_block", 192)


@pytest.mark.parametrize("tc", [3, 2])
def test_mixed_lu_tile128(Solver, B, two_spheres, tc):
    """Update tiles of 128 x 128 real columns (MMA N = 128) in the deferred (3) and per-panel (2)
    tensor-core updates give the oracle's solutions with few refinement corrections."""
    ks = np.array([1.5, 8.0])
    s = _solver(Solver, two_spheres, tc=tc)
    s.set_option("mixed.lu_tile", 128)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(two_spheres, k, D)
        assert rel(surf[i, 0], P) <= TOL, (k, rel(surf[i, 0], P))
        assert rep[i].iters <= 8 and not (rep[i].flags & B.BIE_FLAG_NOT_CONVERGED), (k, rep[i].iters)
    with pytest.raises(B.BieError):
        s.set_option("mixed.lu_tile", 64)


@pytest.mark.parametrize("block", [128, 256])
def test_mixed_lu_panel32(Solver, B, two_spheres, block):
    """32-column panels in the deferred update (N = 1284: a ragged last panel and block) give the
    oracle's solutions with few refinement corrections."""
    ks = np.array([1.5, 8.0])
    s = _solver(Solver, two_spheres, tc=3)
    s.set_option("mixed.lu_block", block)
    s.set_option("mixed.lu_panel", 32)
    surf, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf = surf.cpu().numpy()
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(two_spheres, k, D)
        assert rel(surf[i, 0], P) <= TOL, (k, rel(surf[i, 0], P))
        assert rep[i].iters <= 8 and not (rep[i].flags & B.BIE_FLAG_NOT_CONVERGED), (k, rep[i].iters)
    with pytest.raises(B.BieError):
        s.set_option("mixed.lu_panel", 48)
