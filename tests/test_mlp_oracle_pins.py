"""Pins of the FP64 initializer oracle against facts fixed outside it:
textbook values of GELU and the normal CDF, finite differences of its own
loss, closed forms of degenerate networks, hand-computed features of a
constant-speed platoon, and an independent float64 autograd restatement."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2412_16750_gb300 import synth


def test_gelu_textbook_values():
    # gelu(x) = x Phi(x): Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1)
    assert M.gelu(np.array(0.0)) == 0.0
    assert abs(M.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(np.array(-1.0)) + 1 - 0.8413447460685429) < 1e-15
    x = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-14)   # odd part is x / 2 twice
    assert abs(M.gelu_grad(np.array(0.0)) - 0.5) < 1e-16
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(x), (M.gelu(x + h) - M.gelu(x - h)) / (2 * h), rtol=1e-8, atol=1e-9)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    w = synth.mlp_init(0) * 3.0          # larger weights: non-trivial GELU curvature
    B = 7
    X = rng.normal(size=(B, 80))
    T = rng.uniform(size=(B, 5))
    L, g = M.loss_grad(w, X, T)
    assert abs(L - M.loss(w, X, T)) < 1e-15
    # a few coordinates of every tensor
    offs, o = [], 0
    for _, shape in M.SHAPES:
        n = int(np.prod(shape))
        offs += list(o + rng.choice(n, size=5, replace=False))
        o += n
    for i in offs:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (M.loss(wp, X, T) - M.loss(wm, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-6), (i, fd, g[i])


def test_zero_weight_network_closed_form():
    d = {name: np.zeros(shape) for name, shape in M.SHAPES}
    d["b4"] = np.array([0.0, 1.0, -2.0, 0.5, 3.0])
    d["b3"] = np.full(256, 0.3)
    w = M.pack(d)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(4, 80))
    T = rng.uniform(size=(4, 5))
    s = 1.0 / (1.0 + np.exp(-d["b4"]))
    a = M.forward(w, X)
    np.testing.assert_allclose(a["s"], np.tile(s, (4, 1)), rtol=1e-15)
    L, g = M.loss_grad(w, X, T)
    gd = M.unpack(g)
    dl = 2 * (s - T) * s * (1 - s) / 20.0                       # dL/do per row
    np.testing.assert_allclose(gd["b4"], dl.sum(0), rtol=1e-13)
    h3 = 0.3 * 0.5 * (1 + math.erf(0.3 / math.sqrt(2)))          # gelu(0.3), the constant last hidden layer
    np.testing.assert_allclose(gd["W4"], np.outer(dl.sum(0), np.full(256, h3)), rtol=1e-12)
    for name in ("W1", "W2", "W3", "b1", "b2", "b3"):
        assert np.all(gd[name] == 0.0), name                     # W4 = 0 blocks every lower gradient
    # sigmoid(0) maps to the middle of the box
    P = M.predict_params(w, X, synth.BOX_LO, synth.BOX_HI)
    assert abs(P[0, 0] - 0.5 * (synth.BOX_LO[0] + synth.BOX_HI[0])) < 1e-12


def test_features_of_a_constant_speed_platoon():
    # three vehicles of one lane and a lone vehicle, all at v = 20 m/s with
    # exact observations: central differences are exact on linear motion
    v, dt, s = 20.0, 0.1, 2
    lane_off = np.array([0, 3, 4])
    p0 = np.array([0.0, -30.0, -62.0, 5.0])
    K = 20 * s
    steps = np.arange(1, K // s + 1) * s
    Y = p0[None, :] + v * dt * steps[:, None]
    X = M.features(lane_off, p0, np.full(4, v), Y, s, dt)
    j = np.arange(20)
    x_self = v * dt * s * j / 100.0
    for i in range(4):
        np.testing.assert_allclose(X[i, :20], x_self, atol=1e-13)
        np.testing.assert_allclose(X[i, 20:40], v / 30.0, atol=1e-12)
        np.testing.assert_allclose(X[i, 60:80], v / 30.0, atol=1e-12)
    np.testing.assert_allclose(X[1, 40:60], (30.0 + v * dt * s * j) / 100.0, atol=1e-13)   # leader 30 m ahead
    np.testing.assert_allclose(X[2, 40:60], (32.0 + v * dt * s * j) / 100.0, atol=1e-13)
    for head in (0, 3):                                                    # virtual leader 200 m ahead
        np.testing.assert_allclose(X[head, 40:60], x_self + 2.0, atol=1e-13)
    # a permutation selects rows
    np.testing.assert_array_equal(M.features(lane_off, p0, np.full(4, v), Y, s, dt, perm=[3, 1]), X[[3, 1]])


def test_labels_map_the_box_to_unit_interval():
    lo, hi = np.array(synth.BOX_LO), np.array(synth.BOX_HI)
    th = np.vstack([np.stack([lo, hi, 0.5 * (lo + hi)], axis=1), np.full((1, 3), 4.0)])
    T = M.labels(th, lo, hi)
    np.testing.assert_allclose(T, [[0.0] * 5, [1.0] * 5, [0.5] * 5], atol=1e-15)


def test_matches_an_independent_autograd_restatement():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    w = synth.mlp_init(1)
    X = rng.normal(size=(16, 80))
    T = rng.uniform(size=(16, 5))
    L, g = M.loss_grad(w, X, T)
    p = {k: torch.tensor(a.copy(), dtype=torch.float64, requires_grad=True) for k, a in M.unpack(w).items()}
    h = torch.tensor(X)
    for l in (1, 2, 3):
        h = torch.nn.functional.gelu(torch.nn.functional.linear(h, p["W%d" % l], p["b%d" % l]))
    s = torch.sigmoid(torch.nn.functional.linear(h, p["W4"], p["b4"]))
    Lt = ((s - torch.tensor(T)) ** 2).sum() / (5 * 16)
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-14
    gt = M.pack({k: p[k].grad.numpy() for k, _ in M.SHAPES})
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-15)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    w0 = rng.normal(size=50)
    gs = [rng.normal(size=50) for _ in range(3)]
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    wt = torch.tensor(w0.copy(), requires_grad=True)
    opt = torch.optim.Adam([wt], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    for t, g in enumerate(gs, 1):
        w, m, v = M.adam_step(w, g, m, v, t, 0.01)
        wt.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(w, wt.detach().numpy(), rtol=1e-12, atol=1e-15)
