"""The zero-frequency term of Eq. (inverseFourier) on the CUDA path, against the CPU FP64 oracle:
k = 0 is solved by the k -> 0 limit of the same kernels (G = 1/R, g = 1, f = nu.r), in every
kernel variant that can meet it, and the space-time synthesis of a soft body then includes m = 0.
Also the rejection of observation points that lie inside a body (Eq. BRIEFdmn holds in the fluid).
Bars as in the other GPU tests: FP64 path 1e-10 (entries 1e-12 of max|A|), mixed path 1e-6."""
import numpy as np
import pytest
import torch

import oracle
from workloads import octa_sphere, ico_sphere, merge_meshes, scale_translate, shell_points, gaussian_pulse

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


def _solver(Solver, mesh, d=D):
    s = Solver(0)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    s.set_incident_plane_wave(d)
    return s


def _mixed_bodies():
    s0 = ico_sphere(2)
    return merge_meshes([scale_translate(s0, 0.8, (0, 0, -1.0), bc=1), scale_translate(s0, 1.1, (0.3, 0, 1.3), bc=0)])


@pytest.mark.parametrize("bulk_ff", [0, 1])
def test_zero_frequency_assembly_matches_oracle(Solver, bulk_ff):
    for m in (octa_sphere(2, bc=1), octa_sphere(2, bc=0), _mixed_bodies()):
        s = _solver(Solver, m)
        s.set_option("assemble.bulk_ff", bulk_ff)
        A, b = s.assemble(0.0)
        Ar, br = oracle.assemble_system(m, 0.0, D)
        assert np.abs(A.cpu().numpy() - Ar).max() <= 1e-12 * np.abs(Ar).max()
        if np.abs(br).max() > 0:
            assert rel(b.cpu().numpy(), br) <= 1e-12
        else:
            assert np.abs(b.cpu().numpy()).max() == 0.0


@pytest.mark.parametrize("asm_kb", [0, 1, 2])
def test_zero_frequency_solves_and_fields(Solver, B, asm_kb):
    """k = 0 inside a batch with k > 0 (so the two-wavenumber assembly pairs it with another k),
    soft sphere and a mixed hard/soft pair; FP64 and mixed solves and fields against the oracle."""
    ks = np.array([0.0, 0.5, 1.25])
    for m in (octa_sphere(2, bc=1), _mixed_bodies()):
        pts = shell_points(40, 2.6, 4.0, seed=11)
        s = _solver(Solver, m)
        s.set_option("mixed.asm_kb", asm_kb)
        xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
        s64, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
        s32, rep = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
        T64 = s.eval_field(xo, ks, s64, B.BIE_MODE_FP64).cpu().numpy()
        T32 = s.eval_field(xo, ks, s32, B.BIE_MODE_MIXED).cpu().numpy()
        g64, g32 = s64.cpu().numpy(), s32.cpu().numpy()
        for i, k in enumerate(ks):
            P, Pn = oracle.solve_frequency(m, k, D)
            Tr = oracle.field(m, k, P, Pn, pts)
            assert rel(g64[i, 0], P) <= 1e-10 and rel(g64[i, 1], Pn) <= 1e-10, k
            assert rel(T64[i], Tr) <= 1e-10, k
            assert rel(g32[i, 0], P) <= 1e-6 and rel(g32[i, 1], Pn) <= 1e-6, (k, rep[i].flags)
            assert rel(T32[i], Tr) <= 1e-6, k
        assert rep[0].backward_err <= 1e-10


def test_zero_frequency_reassembly_path(Solver, B):
    """k = 0 through the float-float and FP64 re-assembly of flagged wavenumbers (forced by a tiny
    sensitivity threshold)."""
    m = octa_sphere(2, bc=1)
    P, Pn = oracle.solve_frequency(m, 0.0, D)
    for reas in (1, 0):
        s = _solver(Solver, m)
        s.set_option("mixed.fallback_err_est", 1e-30)
        s.set_option("mixed.reassembly", reas)
        surf, rep = s.solve_frequencies(np.array([0.0, 0.75]), B.BIE_MODE_MIXED)
        assert rep[0].flags & B.BIE_FLAG_FP64_ASSEMBLY
        assert rel(surf[0, 1].cpu().numpy(), Pn) <= 1e-8


def test_zero_frequency_uniform_field_group(Solver, B):
    """A uniform wavenumber group that starts at k = 0 (the field kernels step e^{ikR} from k_0 by
    rotations): 16 wavenumbers k_m = m dk, m = 0..15, mixed field against the oracle's."""
    m = octa_sphere(2, bc=1)
    dk = 0.25
    ks = dk * np.arange(16)
    pts = shell_points(32, 1.2, 3.0, seed=12)
    s = _solver(Solver, m)
    xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    sc = surf.cpu().numpy()
    for variant in (0, 1, 2):
        s.set_option("field.variant", variant)
        T = s.eval_field(xo, ks, surf, B.BIE_MODE_MIXED).cpu().numpy()
        for i in (0, 1, 7, 15):
            Tr = oracle.field(m, ks[i], sc[i, 0], sc[i, 1], pts)
            assert rel(T[i], Tr) <= 1e-6, (variant, ks[i])


def test_field_segments_zero_term_and_uniform_run(Solver, B):
    """k = 0 in front of a uniform run, a non-uniform stretch and another uniform run (the field
    launch is cut into segments: runs of at least 4 equally spaced wavenumbers keep the phase
    recurrence): one call gives the same mixed fields as the segments called one by one, and the
    oracle's fields."""
    m = octa_sphere(2, bc=1)
    ks = np.concatenate([[0.0], 0.5 + 0.125 * np.arange(19), [3.3, 4.1], 5.0 + 0.2 * np.arange(6)])
    pts = shell_points(32, 1.2, 3.0, seed=13)
    s = _solver(Solver, m)
    xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    sc = surf.cpu().numpy()
    for variant in (0, 2):
        s.set_option("field.variant", variant)
        T = s.eval_field(xo, ks, surf, B.BIE_MODE_MIXED).cpu().numpy()
        parts = [s.eval_field(xo, ks[a:b], surf[a:b], B.BIE_MODE_MIXED).cpu().numpy()
                 for a, b in ((0, 1), (1, 20), (20, 22), (22, 28))]
        assert np.array_equal(T, np.concatenate(parts)), variant
        for i in (0, 1, 16, 19, 20, 21, 22, 27):
            Tr = oracle.field(m, ks[i], sc[i, 0], sc[i, 1], pts)
            assert rel(T[i], Tr) <= 1e-6, (variant, ks[i], rel(T[i], Tr))
    s.close()


def test_soft_body_space_time_field_includes_zero_frequency(Solver, B):
    """A Gaussian pulse has a non-zero mean; for a soft sphere T(x, 0) = -a/r is not zero, so the
    synthesis over m = 0..Nt/2 must include the k = 0 solve.  FP64 path against the oracle's
    solves, fields, DFT and synthesis at 1e-10."""
    m = scale_translate(octa_sphere(1, bc=1), 0.7, (0.0, 0.0, 0.0))
    Nt, dk = 32, 0.375
    T = 2 * np.pi / dk
    sig = gaussian_pulse(Nt, T, 0.8, T / 2)[None, :]
    midx = np.arange(0, Nt // 2 + 1)
    ks = dk * midx
    pts = shell_points(12, 1.2, 2.5, seed=13)
    s = _solver(Solver, m)
    xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    Tk = s.eval_field(xo, ks, surf, B.BIE_MODE_FP64)
    S = s.pulse_spectrum(torch.tensor(sig, device="cuda:0"))
    p = s.synthesize(Tk, midx, S, Nt).cpu().numpy()
    Tref = np.zeros((len(ks), len(pts)), complex)
    for i, k in enumerate(ks):
        P, Pn = oracle.solve_frequency(m, k, D)
        Tref[i] = oracle.field(m, k, P, Pn, pts)
    pref = oracle.synthesize(Tref, midx, oracle.dft(sig[0])[None, :], Nt)
    assert np.abs(p - pref).max() <= 1e-10 * np.abs(pref).max()
    # the m = 0 term is not negligible here: dropping it moves the field by more than 1 %
    pnodc = oracle.synthesize(Tref[1:], midx[1:], oracle.dft(sig[0])[None, :], Nt)
    assert np.abs(pnodc - pref).max() > 1e-2 * np.abs(pref).max()


def test_hard_body_zero_frequency_is_exactly_zero(Solver, B):
    m = octa_sphere(2, bc=0)
    s = _solver(Solver, m)
    for mode in (B.BIE_MODE_FP64, B.BIE_MODE_MIXED):
        surf, rep = s.solve_frequencies(np.array([0.0]), mode)
        assert torch.count_nonzero(surf).item() == 0
        if mode == B.BIE_MODE_MIXED:
            assert rep[0].backward_err == 0.0 and not rep[0].flags


def test_wavenumber_and_observation_point_checks(Solver, B):
    m = octa_sphere(2, bc=1)
    s = _solver(Solver, m)
    for bad in (-0.5, 1e-31, float("nan")):
        with pytest.raises(B.BieError) as e:
            s.solve_frequencies(np.array([1.0, bad]), B.BIE_MODE_MIXED)
        assert e.value.code == B.BIE_ERR_INVALID_ARG and "k[1]" in str(e.value)
    with pytest.raises(B.BieError) as e:
        s.solve_frequencies(np.array([0.0, 1.0]), B.BIE_MODE_LEARNED)
    assert e.value.code == B.BIE_ERR_INVALID_ARG
    ks = np.array([0.0, 1.0])
    surf, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    pts = shell_points(20, 1.5, 3.0, seed=14)
    pts[7] = [0.1, 0.2, -0.3]   # inside the unit sphere
    pts[13] = [0.0, 0.0, 0.95]  # inside, next to the surface
    xo = torch.tensor(pts, dtype=torch.float64, device="cuda:0")
    for mode in (B.BIE_MODE_FP64, B.BIE_MODE_MIXED):
        with pytest.raises(B.BieError) as e:
            s.eval_field(xo, ks, surf, mode)
        assert e.value.code == B.BIE_ERR_INVALID_ARG and "observation point 7 " in str(e.value)
    # points on the surface itself (the nodes) and just outside are accepted
    pts2 = np.concatenate([m.nodes[:5], 1.001 * m.nodes[5:10]])
    T = s.eval_field(torch.tensor(pts2, dtype=torch.float64, device="cuda:0"), ks, surf, B.BIE_MODE_FP64)
    assert torch.isfinite(torch.view_as_real(T)).all()
