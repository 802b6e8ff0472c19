"""GPU tests of the batching machinery around the mixed path: CUDA-graph replay of full batches,
the autotuner and its JSON cache, and the multi-configuration scheduler (uneven N)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def _solver(mesh):
    from paper_1706_07919_gb300 import Solver
    s = Solver(0)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_graph_replay_matches_direct_launches():
    from paper_1706_07919_gb300 import binding as B
    mesh = W.octa_sphere(2, 1.0, bc=0)
    k = 0.125 * np.arange(1, 50)  # 49 wavenumbers: three full batches of 16 and one of 1
    out = {}
    for g in (0, 1):
        s = _solver(mesh)
        s.set_option("mixed.batch", 16)
        s.set_option("mixed.graph", g)
        n0 = B.bie_kernel_launches()
        surf, rep = s.solve_frequencies(k, B.BIE_MODE_MIXED)
        out[g] = (surf.cpu().numpy(), B.bie_kernel_launches() - n0, [r.iters for r in rep])
        s.close()
    assert _rel(out[1][0], out[0][0]) <= 1e-13
    assert out[1][2] == out[0][2]
    assert out[1][1] == out[0][1]  # replayed kernels are counted like launched ones
    P, _ = oracle.solve_frequency(mesh, k[40], [0.0, 0.0, 1.0])
    assert _rel(out[1][0][40, 0], P) <= 1e-6


def test_autotune_cache(tmp_path):
    from paper_1706_07919_gb300 import binding as B
    mesh = W.octa_sphere(2, 1.0, bc=0)
    cache = str(tmp_path / "tune.json")
    s = _solver(mesh)
    r1 = B.bie_autotune(s.ctx, [1.0, 2.5, 4.0], cache)
    assert r1["from_cache"] == 0 and r1["n_bucket"] == 320
    assert r1["batch"] in (8, 16, 32, 64, 128, 256) and r1["tcgen05"] in (2, 3) and r1["us_per_k"] > 0
    assert r1["lu_block"] in (128, 256, 512) and r1["lu_panel"] in (32, 64) and r1["lu_tile"] in (128, 256)
    data = json.load(open(cache))
    assert data["entries"]["320"]["batch"] == r1["batch"]
    s.close()
    s = _solver(mesh)
    r2 = B.bie_autotune(s.ctx, [1.0], cache)
    assert r2["from_cache"] == 1 and r2["batch"] == r1["batch"] and r2["tcgen05"] == r1["tcgen05"]
    assert r2["lu_block"] == r1["lu_block"] and r2["lu_panel"] == r1["lu_panel"] and r2["lu_tile"] == r1["lu_tile"]
    surf, rep = s.solve_frequencies([2.25], B.BIE_MODE_MIXED)
    P, _ = oracle.solve_frequency(mesh, 2.25, [0.0, 0.0, 1.0])
    assert _rel(surf.cpu().numpy()[0, 0], P) <= 1e-6
    s.close()


def test_scheduler_uneven_configurations(tmp_path):
    from paper_1706_07919_gb300 import binding as B
    picks = []
    for i in range(64):
        mesh, _ = W.uneven_configuration(i)
        if mesh.N <= 1100:
            picks.append(mesh)
        if len(picks) == 5:
            break
    assert len(picks) == 5
    k = np.linspace(0.5, 6.0, 6)
    sched = B.bie_sched_create(0, 3, str(tmp_path / "tune.json"))
    surfs, jobs = [], []
    for m in picks:
        surf = torch.empty((len(k), 2, m.N), dtype=torch.complex128, device="cuda")
        surfs.append(surf)
        jobs.append(B.bie_sched_add(sched, m.nodes, m.elems, m.normals, m.bc, [0.0, 0.0, 1.0], k,
                                    B.BIE_MODE_MIXED, surf))
    st = B.bie_sched_run(sched)
    B.bie_sched_destroy(sched)
    assert st["jobs"] == 5 and st["workers"] == 3 and st["wall_ms"] > 0
    for m, surf, job in zip(picks, surfs, jobs):
        s = _solver(m)
        ref, _ = s.solve_frequencies(k, B.BIE_MODE_MIXED)
        s.close()
        assert _rel(surf.cpu().numpy(), ref.cpu().numpy()) <= 1e-7
        assert all(r.backward_err <= 1e-10 for r in job.reports())
    i = int(np.argmin([x.N for x in picks]))
    m = picks[i]
    P, _ = oracle.solve_frequency(m, k[3], [0.0, 0.0, 1.0])
    assert _rel(surfs[i].cpu().numpy()[3, 0], P) <= 1e-6


def test_scheduler_reports_a_failing_job(tmp_path):
    from paper_1706_07919_gb300 import binding as B
    good = W.octa_sphere(1)
    bad = W.octa_sphere(1)
    bad_elems = bad.elems.copy()
    bad_elems[3, 2] = bad.N + 5  # node index out of range
    sched = B.bie_sched_create(0, 2, None)
    k = np.array([1.0, 2.0])
    o1 = torch.empty((2, 2, good.N), dtype=torch.complex128, device="cuda")
    o2 = torch.empty((2, 2, bad.N), dtype=torch.complex128, device="cuda")
    B.bie_sched_add(sched, good.nodes, good.elems, good.normals, good.bc, None, k, B.BIE_MODE_MIXED, o1)
    B.bie_sched_add(sched, bad.nodes, bad_elems, bad.normals, bad.bc, None, k, B.BIE_MODE_MIXED, o2)
    with pytest.raises(B.BieError) as e:
        B.bie_sched_run(sched)
    assert e.value.code == B.BIE_ERR_INVALID_ARG and "scheduler job failed" in str(e.value)
    B.bie_sched_destroy(sched)


def test_autotune_ignores_a_corrupt_cache(tmp_path):
    from paper_1706_07919_gb300 import binding as B
    cache = tmp_path / "tune.json"
    cache.write_text('{"bie_autotune": 1, "entries": {"320": {"batch": -4, "tcgen05": 9}, garbage')
    s = _solver(W.octa_sphere(2))
    r = B.bie_autotune(s.ctx, [2.0], str(cache))
    assert r["from_cache"] == 0 and r["batch"] >= 8
    assert json.load(open(cache))["entries"]["320"]["batch"] == r["batch"]
    s.close()
