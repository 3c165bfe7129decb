"""Pins of the oracle's smoothing-length network (the learned form).

Each pin checks the oracle against something other than itself: central
finite differences of its own forward pass, closed forms of wired-up
networks, torch's bfloat16 conversion, textbook properties of Adam, and a
fit of a known smooth function.
"""
import math

import numpy as np
import pytest

from oracle import mlp
from paper_2603_19764_b300 import workloads as wl


def _rand_net(seed=1, scale=0.4):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, mlp.NPARAM)
    norm = np.concatenate([rng.normal(0, 0.1, 6), rng.uniform(0.5, 2.0, 6), [0.02, 0.3]])
    return theta, norm


def test_parameter_count_matches_the_layer_shapes():
    assert mlp.NPARAM == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4673
    assert wl.MLP_NPARAM == mlp.NPARAM
    assert wl.mlp_init().shape == (mlp.NPARAM,)


def test_gradient_matches_central_differences():
    theta, norm = _rand_net()
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (7, 6))
    y = rng.normal(0, 0.2, 7)
    L, g = mlp.loss_grad(theta, norm, X, y)
    h = 1e-6
    fd = np.empty_like(theta)
    for k in range(theta.shape[0]):
        tp = theta.copy()
        tp[k] += h
        tm = theta.copy()
        tm[k] -= h
        fd[k] = (mlp.loss_grad(tp, norm, X, y)[0] - mlp.loss_grad(tm, norm, X, y)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))
    # the loss itself: half the mean squared standardised error
    out = (mlp.forward(theta, norm, X) - norm[12]) / norm[13]
    yh = (y - norm[12]) / norm[13]
    assert math.isclose(L, 0.5 * np.mean((out - yh) ** 2), rel_tol=1e-12)


def test_forward_of_a_wired_network_matches_scalar_tanh():
    """One path through the layers: feature f -> hidden unit k -> unit j.
    A transposed weight matrix or a wrong slice routes it elsewhere."""
    W1 = np.zeros((64, 6))
    W2 = np.zeros((64, 64))
    W3 = np.zeros(64)
    f, k, j, al, be, w3, b3 = 4, 17, 41, 0.7, 1.3, -0.9, 0.25
    W1[k, f] = al
    W2[j, k] = be
    W3[j] = w3
    theta = mlp.pack(W1, np.zeros(64), W2, np.zeros(64), W3, b3)
    norm = np.concatenate([np.full(6, 0.5), np.full(6, 2.0), [0.1, 3.0]])
    X = np.linspace(-2, 2, 30)[:, None] * np.ones((1, 6))
    got = mlp.forward(theta, norm, X)
    xs = (X[:, f] - 0.5) / 2.0
    want = 0.1 + 3.0 * np.array([w3 * math.tanh(be * math.tanh(al * v)) + b3 for v in xs])
    assert np.allclose(got, want, rtol=0, atol=1e-14)
    # biases: every hidden unit saturated by its bias gives a constant output
    theta2 = mlp.pack(np.zeros((64, 6)), np.full(64, 50.0), np.zeros((64, 64)),
                      np.arange(64) * 0.01, np.ones(64), 0.0)
    c = sum(math.tanh(0.01 * q) for q in range(64))
    assert np.allclose(mlp.forward(theta2, norm, X), 0.1 + 3.0 * c, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-30, 50), rng.normal(0, 1e30, 50),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 3.14159265]])
    ours = mlp.bf16_round(x)
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert mlp.bf16_round([1.0 + 2.0 ** -8])[0] == 1.0            # tie to even
    assert mlp.bf16_round([1.0 + 3 * 2.0 ** -9])[0] == 1.0 + 2.0 ** -7


def test_bf16_emulation_is_close_to_exact():
    theta, norm = _rand_net(5, 0.3)
    X = np.random.default_rng(6).normal(0, 1, (64, 6))
    y = np.random.default_rng(7).normal(0, 0.3, 64)
    p0 = mlp.forward(theta, norm, X)
    p1 = mlp.forward(theta, norm, X, bf16=True)
    assert np.max(np.abs(p1 - p0)) < 3e-2 * np.max(np.abs(p0 - norm[12]))
    _, g0 = mlp.loss_grad(theta, norm, X, y)
    _, g1 = mlp.loss_grad(theta, norm, X, y, bf16=True)
    assert np.max(np.abs(g1 - g0)) < 3e-2 * np.max(np.abs(g0))


def test_adam_first_step_and_convergence():
    # at t = 1 the bias-corrected moments are g and g^2: the step is lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=0, atol=1e-15)
    # minimising 1/2 (theta - 3)^2
    th, m, v = np.array([0.0]), np.zeros(1), np.zeros(1)
    for t in range(1, 3001):
        th, m, v = mlp.adam(th, m, v, th - 3.0, t, 0.05)
    assert abs(th[0] - 3.0) < 1e-3


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(8)
    X = rng.normal(0, 1, (256, 6))
    y = 0.3 * np.sin(X[:, 0]) + 0.1 * X[:, 1] * X[:, 2] - 0.05 * X[:, 5]
    norm = mlp.fit_norm(X, y)
    theta = wl.mlp_init()
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    L0 = mlp.loss_grad(theta, norm, X, y)[0]
    for t in range(1, 401):
        L, g = mlp.loss_grad(theta, norm, X, y)
        theta, m, v = mlp.adam(theta, m, v, g, t, 3e-3)
    assert L < 0.05 * L0


def test_features_of_a_relaxed_lattice_particle_are_zero():
    n_ngb, rho0, m = 64, 2700.0, 2.0e6
    hbar = (3 * n_ngb * m / (4 * math.pi * rho0)) ** (1 / 3)
    F = mlp.features([hbar, 2 * hbar], [64, 80], [rho0, 1.5 * rho0], [1.0, 1.1],
                     [0.0, -0.02], [hbar, hbar], n_ngb, [m, m], rho0)
    assert np.allclose(F[0], 0.0, atol=1e-15)
    assert np.allclose(F[1], [math.log(2), 0.25, math.log(1.5), -0.02, math.log(2), 0.1],
                       atol=1e-14)


def test_fit_norm_standardises():
    rng = np.random.default_rng(9)
    X = rng.normal(3.0, 2.0, (5000, 6))
    y = rng.normal(-1.0, 0.5, 5000)
    nm = mlp.fit_norm(X, y)
    Z = (X - nm[:6]) / nm[6:12]
    assert np.allclose(Z.mean(0), 0, atol=1e-12) and np.allclose(Z.std(0), 1, atol=1e-12)
    assert math.isclose(nm[12], y.mean()) and math.isclose(nm[13], y.std())
