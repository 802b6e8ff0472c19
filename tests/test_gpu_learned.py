"""GPU tests of the learned warm start (network kernels) and of BIE_MODE_LEARNED (GMRES solves),
through the C ABI, against the CPU oracle.

Tolerances of the network kernels come from their arithmetic: the hidden layers multiply BF16
operands (unit roundoff u = 2^-9) with FP32 accumulation and round every activation and every
backward product to BF16 again, so each layer adds a relative error of a few u; over three layers
the outputs and gradients stay within 1.5e-2 and 4e-2 (relative L2) of the FP64 oracle on the
random networks used here, the test parameters and inputs being BF16-representable so that the
operand rounding is exact.  The optimiser step runs in FP32 (relative 1e-6).  The frequency solves
of the learned mode must meet the mixed path's bar: relative L2 <= 1e-6 against the FP64 oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def _bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16-representable value (ties to even), kept as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    sl = oracle.mlp_param_slices()
    th = np.zeros(oracle.mlp_param_count(), np.float32)
    for name, (off, shp) in sl.items():
        n = int(np.prod(shp))
        if len(shp) == 2:
            a = np.sqrt(6.0 / (shp[0] + shp[1]))
            th[off:off + n] = rng.uniform(-a, a, n)
        else:
            th[off:off + n] = rng.uniform(-0.2, 0.2, n)
    return _bf16(th)


def _solver(mesh):
    from paper_1706_07919_gb300 import Solver
    s = Solver(0)
    s.set_geometry(mesh.nodes, mesh.elems, mesh.normals, mesh.bc)
    return s


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small_spheroid():
    return W.ellipsoid_from_sphere(W.ico_sphere(3, 1.0, bc=0), (1.0, 1.0, 2.0))


def test_features_match_oracle(small_spheroid):
    m = small_spheroid
    s = _solver(m)
    s.set_option("learned.kmax", 10.0)
    kv = np.array([0.37, 4.1, 9.5])
    phi = s.mlp_features(kv).cpu().numpy()
    c = m.nodes.mean(axis=0)
    sc = np.max(np.linalg.norm(m.nodes - c, axis=1))
    ref = oracle.mlp_features(m.nodes, m.normals, kv, [0.0, 0.0, 1.0], c, sc, 10.0)
    # GPU features are rounded to BF16: half an ulp of values up to ~1.5, plus FP32 phases
    assert np.max(np.abs(phi - ref)) <= 4e-3
    assert np.array_equal(phi, _bf16(phi))
    s.close()


@pytest.mark.parametrize("B", [128, 300, 1000])
def test_forward_matches_oracle(small_spheroid, B):
    s = _solver(small_spheroid)
    th = _params(7)
    s.mlp_set_params(th)
    rng = np.random.default_rng(B)
    X = _bf16(rng.uniform(-1, 1, (B, 64)))
    Y = s.mlp_forward(torch.tensor(X, device="cuda")).cpu().numpy()
    ref = oracle.mlp_forward(th.astype(np.float64), X.astype(np.float64))
    assert _rel(Y, ref) <= 1.5e-2
    assert np.allclose(s.mlp_get_params(), th, rtol=0, atol=0)
    s.close()


@pytest.mark.parametrize("B", [256, 333])
def test_gradient_matches_oracle(small_spheroid, B):
    s = _solver(small_spheroid)
    th = _params(11)
    s.mlp_set_params(th)
    rng = np.random.default_rng(100 + B)
    X = _bf16(rng.uniform(-1, 1, (B, 64)))
    T = rng.normal(size=(B, 2)).astype(np.float32)
    L, g = s.mlp_loss_grad(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    g = g.cpu().numpy()
    Lr, gr = oracle.mlp_loss_grad(th.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(L - Lr) <= 1e-2 * Lr
    for name, (off, shp) in oracle.mlp_param_slices().items():
        n = int(np.prod(shp))
        e = _rel(g[off:off + n], gr[off:off + n])
        assert e <= 4e-2, (name, e)
    s.close()


def test_adam_steps_match_oracle(small_spheroid):
    s = _solver(small_spheroid)
    th = _params(3)
    s.mlp_set_params(th)
    rng = np.random.default_rng(5)
    P = th.shape[0]
    t64, m, v = th.astype(np.float64), np.zeros(P), np.zeros(P)
    for t in (1, 2, 3):
        g = (rng.normal(size=P) * 10.0 ** rng.uniform(-4, 0, P)).astype(np.float32)
        s.mlp_adam_step(torch.tensor(g, device="cuda"), 1e-3)
        oracle.adam_step(t64, g.astype(np.float64), m, v, t, 1e-3)
    got = s.mlp_get_params().astype(np.float64)
    assert np.max(np.abs(got - t64)) <= 1e-6 * (1.0 + np.max(np.abs(t64)))
    s.close()


@pytest.fixture(scope="module")
def learned_case():
    """Hard prolate spheroid (642 nodes), 96 wavenumbers k_m = 0.02 m: anchors every 8th
    (spacing 0.16, as on the 1024-wavenumber spheroid workload)."""
    from paper_1706_07919_gb300 import binding as Bd
    mesh = W.ellipsoid_from_sphere(W.ico_sphere(4, 1.0, bc=0), (1.0, 1.0, 2.0))
    k = 0.02 * np.arange(1, 97)
    out = {}
    for x0 in (1, 0):
        s = _solver(mesh)
        s.set_option("learned.x0", x0)
        s.set_option("learned.epochs", 400)
        s.set_option("learned.batch", 1024)
        surf, rep = s.solve_frequencies(k, Bd.BIE_MODE_LEARNED)
        out[x0] = (surf.cpu().numpy(), rep, s.learned_info())
        s.close()
    return mesh, k, out


def test_learned_solves_match_oracle(learned_case):
    from paper_1706_07919_gb300 import binding as Bd
    mesh, k, out = learned_case
    surf, rep, info = out[1]
    assert info["anchors"] == 12 and info["krylov"] == 84
    paths = [r.path for r in rep]
    assert paths.count(Bd.BIE_MODE_LEARNED) + info["krylov_fallback"] == 84
    for i in (0, 4, 13, 22, 50, 94):  # non-anchor wavenumbers across the band (7, 15, ... are anchors)
        P, Pn = oracle.solve_frequency(mesh, k[i], [0.0, 0.0, 1.0])
        assert _rel(surf[i, 0], P) <= 1e-6, (i, k[i], rep[i].flags)
        assert _rel(surf[i, 1], Pn) <= 1e-6
    for i in (7, 95):  # anchors (direct path)
        P, _ = oracle.solve_frequency(mesh, k[i], [0.0, 0.0, 1.0])
        assert _rel(surf[i, 0], P) <= 1e-6
    for r in rep:
        assert r.backward_err <= 1e-10


def test_network_warm_start_gains(learned_case):
    mesh, k, out = learned_case
    _, _, net = out[1]
    _, _, zero = out[0]
    print("network:", net)
    print("zero start:", zero)
    assert zero["x0_rel_err"] == pytest.approx(1.0)
    assert net["last_loss"] < 0.05 * net["first_loss"]
    assert net["x0_rel_err"] < 0.1
    assert net["mean_iters"] < zero["mean_iters"]


def test_learned_soft_hard_ragged_and_single_anchor():
    """Mixed boundary conditions (a soft and a hard body, the unknown is dP/dnu on the soft one),
    a wavenumber count that is not a multiple of the stride, and a call with fewer wavenumbers
    than the stride (one anchor: the last wavenumber), started from the anchor's solution."""
    from paper_1706_07919_gb300 import binding as Bd
    s0 = W.ico_sphere(2)
    m = W.merge_meshes([W.scale_translate(s0, 0.8, (0, 0, -1.1), bc=1), W.scale_translate(s0, 1.0, (0.2, 0, 1.2), bc=0)])
    d = np.array([0.0, 0.0, 1.0])
    k = 0.1 * np.arange(1, 12)  # 11 wavenumbers, stride 4: anchors at indices 3 and 7
    s = _solver(m)
    s.set_option("learned.stride", 4)
    s.set_option("learned.epochs", 30)
    s.set_option("learned.batch", 256)
    surf, rep = s.solve_frequencies(k, Bd.BIE_MODE_LEARNED)
    info = s.learned_info()
    assert info["anchors"] == 2 and info["krylov"] == 9
    surf = surf.cpu().numpy()
    for i in (0, 5, 10):
        P, Pn = oracle.solve_frequency(m, k[i], d)
        assert _rel(surf[i, 0], P) <= 1e-6 and _rel(surf[i, 1], Pn) <= 1e-6
    s.set_option("learned.x0", 2)
    surf2, rep2 = s.solve_frequencies(k[:3], Bd.BIE_MODE_LEARNED)
    assert s.learned_info()["anchors"] == 1 and rep2[2].path == Bd.BIE_MODE_MIXED
    P, Pn = oracle.solve_frequency(m, k[0], d)
    assert _rel(surf2.cpu().numpy()[0, 1], Pn) <= 1e-6
    s.close()


def test_network_entry_points_report_errors(small_spheroid):
    from paper_1706_07919_gb300 import binding as Bd
    s = _solver(small_spheroid)
    with pytest.raises(Bd.BieError) as e:
        s.mlp_get_params()
    assert e.value.code == Bd.BIE_ERR_STATE
    with pytest.raises(Bd.BieError) as e:
        s.mlp_features([1.0])  # no wavenumber scale yet
    assert e.value.code == Bd.BIE_ERR_STATE
    with pytest.raises(ValueError):
        s.mlp_set_params(np.zeros(10, np.float32))
    th = _params(1)
    th[5] = np.nan
    with pytest.raises(Bd.BieError) as e:
        s.mlp_set_params(th)
    assert e.value.code == Bd.BIE_ERR_INVALID_ARG
    with pytest.raises(Bd.BieError):
        s.set_option("gmres.m", 100)
    with pytest.raises(Bd.BieError):
        s.set_option("learned.x0", 4)
    s.close()


def test_anchor_interpolant_start():
    """learned.x0 = 3: the bracketing anchors' demodulated solutions interpolated in k start GMRES;
    the solves match the oracle at the mixed bar, and the start is closer to the solution than the
    nearest anchor's (phase-uncorrected) solution."""
    from paper_1706_07919_gb300 import binding as Bd
    mesh = W.ellipsoid_from_sphere(W.ico_sphere(3, 1.0, bc=0), (1.0, 1.0, 2.0))
    k = 0.05 * np.arange(1, 33)
    info = {}
    for x0 in (3, 2):
        s = _solver(mesh)
        s.set_option("learned.x0", x0)
        s.set_option("learned.stride", 4)
        surf, rep = s.solve_frequencies(k, Bd.BIE_MODE_LEARNED)
        info[x0] = s.learned_info()
        sc = surf.cpu().numpy()
        s.close()
        if x0 == 3:
            for i in (0, 5, 14, 30):
                P, _ = oracle.solve_frequency(mesh, k[i], [0.0, 0.0, 1.0])
                assert np.linalg.norm(sc[i, 0] - P) / np.linalg.norm(P) <= 1e-6
    assert info[3]["x0_rel_err"] < info[2]["x0_rel_err"], (info[3]["x0_rel_err"], info[2]["x0_rel_err"])

