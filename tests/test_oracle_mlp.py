"""Pins of the oracle's learned-warm-start functions (feature map, network, loss gradient, Adam).

The learned warm start is not part of the paper's method, so nothing here comes from the paper:
the pins are closed forms of special networks, invariants of the feature map, central finite
differences of the loss (which pin the analytic backward pass to the forward pass) and the
closed form of Adam's bias-corrected steps.
"""
import numpy as np
import pytest

import oracle

P = oracle.mlp_param_count()
SL = oracle.mlp_param_slices()


def _zeros():
    return np.zeros(P)


def _view(theta, name):
    off, shp = SL[name]
    return theta[off:off + int(np.prod(shp))].reshape(shp)


def test_param_layout():
    assert P == 256 * 64 + 256 + 2 * (256 * 256 + 256) + 2 * 256 + 2 == 148738
    assert SL["b4"][0] + 2 == P


def _features(nodes, normals, kv, d=(0.0, 0.0, 1.0), centre=(0.0, 0.0, 0.0), scale=2.0, kmax=10.0):
    return oracle.mlp_features(np.asarray(nodes, float), np.asarray(normals, float), kv, np.asarray(d, float),
                               np.asarray(centre, float), scale, kmax)


def test_features_at_centre_and_invariants():
    rng = np.random.default_rng(11)
    x = rng.normal(size=(40, 3))
    nu = rng.normal(size=(40, 3))
    nu /= np.linalg.norm(nu, axis=1, keepdims=True)
    c = np.array([0.3, -0.2, 0.5])
    d = np.array([0.0, 0.6, 0.8])
    kv = np.array([0.7, 3.1])
    phi = _features(x, nu, kv, d, c, 2.5, 8.0)
    assert phi.shape == (2, 40, 64)
    # cos^2 + sin^2 = 1 for every phase
    cs = phi[..., 8:].reshape(2, 40, 28, 2)
    assert np.allclose(cs[..., 0] ** 2 + cs[..., 1] ** 2, 1.0, atol=1e-14)
    # normals and the wavenumber features pass through
    assert np.allclose(phi[:, :, 3:6], nu[None], atol=0)
    assert np.allclose(phi[0, :, 6], 0.7 / 8.0) and np.allclose(phi[1, :, 7], (3.1 / 8.0) ** 2)
    # translating the nodes and the centre together changes nothing
    phi2 = _features(x + 1.7, nu, kv, d, c + 1.7, 2.5, 8.0)
    assert np.allclose(phi, phi2, atol=1e-12)
    # a node at the centre: zero coordinates, all phases zero
    phic = _features(c[None], nu[:1], kv, d, c, 2.5, 8.0)
    assert np.allclose(phic[..., :3], 0.0)
    assert np.allclose(phic[..., 8::2], 1.0) and np.allclose(phic[..., 9::2], 0.0)
    # phases are linear in k: cos(2 th) = 2 cos^2(th) - 1, sin(2 th) = 2 sin cos
    pa = _features(x, nu, np.array([1.3]), d, c, 2.5, 8.0)[0, :, 8:].reshape(40, 28, 2)
    pb = _features(x, nu, np.array([2.6]), d, c, 2.5, 8.0)[0, :, 8:].reshape(40, 28, 2)
    assert np.allclose(pb[..., 0], 2 * pa[..., 0] ** 2 - 1, atol=1e-12)
    assert np.allclose(pb[..., 1], 2 * pa[..., 0] * pa[..., 1], atol=1e-12)


def test_features_phase_geometry():
    # a node displaced by t along e_x from the centre, incidence along e_z: the phases of the
    # directions orthogonal to e_x vanish; along e_x the scales 0.5, 1, 1.5, 2 give k t sc
    t, k = 0.9, 2.0
    phi = _features([[t, 0.0, 0.0]], [[1.0, 0.0, 0.0]], [k])[0, 0]
    ph = np.arctan2(phi[9::2], phi[8::2]).reshape(7, 4)
    assert np.allclose(ph[0], 0.0) and np.allclose(ph[2], 0.0) and np.allclose(ph[3], 0.0)  # d, e_y, e_z
    assert np.allclose(ph[5], 0.0)  # (e_y + e_z)/sqrt2
    scales = np.array([0.5, 1.0, 1.5, 2.0])
    wrap = lambda a: (a + np.pi) % (2 * np.pi) - np.pi
    assert np.allclose(ph[1], wrap(k * t * scales))
    assert np.allclose(ph[4], wrap(k * t * scales / np.sqrt(2.0)))
    assert np.allclose(ph[6], wrap(k * t * scales / np.sqrt(2.0)))


def test_forward_bias_only_and_single_path():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(7, 64))
    th = _zeros()
    _view(th, "b4")[:] = [0.25, -1.5]
    assert np.allclose(oracle.mlp_forward(th, X), [[0.25, -1.5]] * 7, atol=0)
    # W2 = W3 = 0: the output depends on the biases only, y = W4 tanh(b3) + b4
    th = rng.normal(size=P) * 0.3
    _view(th, "W2")[:] = 0.0
    _view(th, "W3")[:] = 0.0
    want = _view(th, "W4") @ np.tanh(_view(th, "b3")) + _view(th, "b4")
    assert np.allclose(oracle.mlp_forward(th, X), np.broadcast_to(want, (7, 2)), rtol=1e-14, atol=1e-14)
    # one path through asymmetric positions: phi[2] -> h1[5] -> h2[7] -> h3[9] -> y[1]
    th = _zeros()
    w1, w2, w3, w4 = 0.7, -1.3, 0.9, 2.2
    _view(th, "W1")[5, 2] = w1
    _view(th, "W2")[7, 5] = w2
    _view(th, "W3")[9, 7] = w3
    _view(th, "W4")[1, 9] = w4
    Y = oracle.mlp_forward(th, X)
    want1 = w4 * np.tanh(w3 * np.tanh(w2 * np.tanh(w1 * X[:, 2])))
    assert np.allclose(Y[:, 0], 0.0, atol=0) and np.allclose(Y[:, 1], want1, rtol=1e-14, atol=1e-15)


def test_loss_closed_form():
    rng = np.random.default_rng(9)
    X = rng.normal(size=(5, 64))
    T = rng.normal(size=(5, 2))
    th = _zeros()
    _view(th, "b4")[:] = [0.5, -0.25]
    want = np.mean(np.sum((np.array([0.5, -0.25]) - T) ** 2, axis=1))
    assert abs(oracle.mlp_loss(th, X, T) - want) < 1e-15
    L, g = oracle.mlp_loss_grad(th, X, T)
    assert abs(L - want) < 1e-15
    # with every weight zero only the output bias has a gradient: 2 mean(y - t)
    gb4 = g[SL["b4"][0]:]
    assert np.allclose(gb4, 2 * np.mean(np.array([0.5, -0.25]) - T, axis=0), atol=1e-15)
    # the hidden biases see zero gradient because W4 = 0
    assert np.all(g[:SL["W4"][0]] == 0.0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(21)
    B = 12
    X = rng.normal(size=(B, 64))
    T = rng.normal(size=(B, 2))
    th = np.zeros(P)
    for name, (off, shp) in SL.items():
        fan_in = shp[1] if len(shp) == 2 else 1
        th[off:off + int(np.prod(shp))] = rng.normal(size=int(np.prod(shp))) / np.sqrt(fan_in)
    L, g = oracle.mlp_loss_grad(th, X, T)
    assert abs(L - oracle.mlp_loss(th, X, T)) < 1e-13 * max(1.0, L)
    idx = []
    for name, (off, shp) in SL.items():
        n = int(np.prod(shp))
        idx += list(off + rng.choice(n, size=min(n, 6), replace=False))
    h = 1e-5
    for p in idx:
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.mlp_loss(tp, X, T) - oracle.mlp_loss(tm, X, T)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-7 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_adam_bias_corrected_steps():
    rng = np.random.default_rng(3)
    n = 50
    th0 = rng.normal(size=n)
    g = rng.normal(size=n)
    g[0] = 0.0
    th, m, v = th0.copy(), np.zeros(n), np.zeros(n)
    lr = 0.01
    oracle.adam_step(th, g, m, v, 1, lr)
    # the first step is lr * g / (|g| + eps): lr * sign(g) up to eps; zero gradient, no move
    assert np.allclose(th, th0 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert th[0] == th0[0]
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps the bias-corrected step at lr * sign(g)
    th1 = th.copy()
    oracle.adam_step(th, g, m, v, 2, lr)
    assert np.allclose(th, th1 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


def test_adam_training_reduces_loss():
    rng = np.random.default_rng(8)
    B = 48
    X = rng.normal(size=(B, 64)) * 0.5
    T = np.stack([np.sin(X[:, 0]), np.cos(X[:, 1])], axis=1)
    th = np.zeros(P)
    for name, (off, shp) in SL.items():
        if len(shp) == 2:
            a = np.sqrt(6.0 / (shp[0] + shp[1]))
            th[off:off + int(np.prod(shp))] = rng.uniform(-a, a, size=int(np.prod(shp)))
    m, v = np.zeros(P), np.zeros(P)
    L0 = oracle.mlp_loss(th, X, T)
    for t in range(1, 61):
        _, g = oracle.mlp_loss_grad(th, X, T)
        oracle.adam_step(th, g, m, v, t, 1e-3)
    assert oracle.mlp_loss(th, X, T) < 0.1 * L0
