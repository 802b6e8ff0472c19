"""The stream-ordered mixed-precision solves (bie_solve_frequencies_async) against the synchronous
call and the CPU FP64 oracle, and their overlap across two contexts on two streams.

* Parity: the same wavenumbers through both calls give the same surface solutions (relative L2
  <= 1e-9 of each other; the unflagged ones run the same kernels) and flags, and the oracle's
  solutions within the mixed path's 1e-6.
* Device-side re-assembly rounds: with every wavenumber flagged, batches of 8 and rounds of 3 slots
  (three rounds per batch, the last with an idle slot), each solution matches the FP64 path's to
  the FP64 refinement's accuracy.
* Stream order: the call returns before its work has run (a pending event right after it), the
  reports arrive once the stream has completed, and two contexts on two streams finish together
  sooner than one after the other.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from workloads import config_sphere_fp64, ico_sphere, merge_meshes, scale_translate

pytestmark = pytest.mark.gpu
D = np.array([0.0, 0.0, 1.0])


def rel(a, b):
    nb = np.linalg.norm(np.asarray(b))
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    return d / nb if nb > 0 else d  # a hard body scatters nothing at k = 0


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


def _solver(Solver, mesh, stream=None):
    s = Solver(0, stream)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    s.set_incident_plane_wave(D)
    return s


@pytest.fixture(scope="module")
def two_spheres():
    s0 = ico_sphere(4)
    return merge_meshes([scale_translate(s0, 1.0, (0, 0, -1.05)), scale_translate(s0, 1.0, (0, 0, 1.05))])


def test_async_matches_sync_and_oracle(Solver, B, two_spheres):
    ks = np.array([0.0, 1.5, 3.1, 4.49, 8.0, 11.0])  # k = 0, and 4.49 next to the zero 4.4934 of j_1
    s = _solver(Solver, two_spheres)
    ref, rep_ref = s.solve_frequencies(ks, B.BIE_MODE_MIXED)
    surf, pending = s.solve_frequencies_async(ks)
    torch.cuda.synchronize()
    rep = pending.reports()
    s.close()
    ref, surf = ref.cpu().numpy(), surf.cpu().numpy()
    assert any(r.flags & B.BIE_FLAG_FP64_ASSEMBLY for r in rep), [r.flags for r in rep]
    for i, k in enumerate(ks):
        assert rel(surf[i], ref[i]) <= 1e-9, (k, rel(surf[i], ref[i]))
        assert rep[i].flags == rep_ref[i].flags and rep[i].path == B.BIE_MODE_MIXED, (k, rep[i].flags, rep_ref[i].flags)
        assert rep[i].backward_err <= 1e-10, (k, rep[i].backward_err)
    for i in (1, 3, 5):
        P, _ = oracle.solve_frequency(two_spheres, ks[i], D)
        assert rel(surf[i, 0], P) <= 1e-6, (ks[i], rel(surf[i, 0], P))


def test_async_reassembly_rounds(Solver, B):
    w = config_sphere_fp64()
    ks = np.linspace(0.5, 9.5, 21)  # batches of 8, 8, 5
    s = _solver(Solver, w.mesh)
    s.set_option("mixed.fallback_err_est", 1e-30)  # every wavenumber flagged
    s.set_option("mixed.batch", 8)
    s.set_option("mixed.reassembly_group", 3)  # rounds of 3 slots: 3 per batch, idle slots in the last
    surf, pending = s.solve_frequencies_async(ks)
    ref, _ = s.solve_frequencies(ks, B.BIE_MODE_FP64)
    torch.cuda.synchronize()
    rep = pending.reports()
    s.close()
    surf, ref = surf.cpu().numpy(), ref.cpu().numpy()
    for i in range(len(ks)):
        assert rep[i].flags & B.BIE_FLAG_FP64_ASSEMBLY and not rep[i].flags & B.BIE_FLAG_NOT_CONVERGED, (i, rep[i].flags)
        assert rep[i].backward_err <= 1e-12, (i, rep[i].backward_err)
        assert rel(surf[i, 0], ref[i, 0]) <= 1e-8 and rel(surf[i, 1], ref[i, 1]) <= 1e-8, (ks[i], rel(surf[i, 0], ref[i, 0]))


def test_async_returns_before_the_work_and_overlaps(Solver, B, two_spheres):
    ks = np.linspace(1.0, 10.0, 8)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sols = [_solver(Solver, two_spheres, st) for st in streams]
    for s in sols:
        s.set_option("mixed.batch", 8)
    warm = [s.solve_frequencies_async(ks) for s in sols]  # first calls: geometry tables, workspace
    torch.cuda.synchronize()
    # the call returns while its work is still queued (32 wavenumbers: four batches of GPU work,
    # far longer than enqueuing them)
    surf, pending = sols[0].solve_frequencies_async(np.linspace(1.0, 10.0, 32))
    pending_at_return = not pending.done()
    rep = pending.reports()
    assert pending_at_return
    assert all(r.path == B.BIE_MODE_MIXED and r.backward_err <= 1e-10 for r in rep)
    # one after the other, then both at once (best of three each)
    seq, par = [], []
    for _ in range(3):
        t = time.perf_counter()
        for s in sols:
            out = s.solve_frequencies_async(ks)
            torch.cuda.synchronize()
        seq.append(time.perf_counter() - t)
        t = time.perf_counter()
        outs = [s.solve_frequencies_async(ks) for s in sols]
        torch.cuda.synchronize()
        par.append(time.perf_counter() - t)
    del warm, out
    for s in sols:
        s.close()
    print(f"two contexts: one after the other {min(seq) * 1e3:.1f} ms, together {min(par) * 1e3:.1f} ms")
    assert min(par) < 0.9 * min(seq), (seq, par)
    a, b = outs[0][0].cpu().numpy(), outs[1][0].cpu().numpy()
    assert rel(a, b) <= 1e-12
