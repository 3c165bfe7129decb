"""The smoothing-length network's kernels against the oracle.

The oracle's bf16 emulation rounds where the kernels hold bf16 operands, so
the kernels must match it up to FP32-versus-FP64 accumulation (and the rare
bf16 rounding decision that the two precisions take differently); against
the exact FP64 network they agree to bf16 precision.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _case(seed=11, m=1003, scale=0.35):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, mlp.NPARAM).astype(np.float32).astype(np.float64)
    norm = np.concatenate([rng.normal(0, 0.1, 6), rng.uniform(0.5, 2.0, 6),
                           [0.02, 0.3]]).astype(np.float32).astype(np.float64)
    X = rng.normal(0, 1.2, (m, 6)).astype(np.float32)
    y = (0.3 * np.sin(X[:, 0]) + 0.1 * X[:, 1] * X[:, 2]).astype(np.float32)
    return theta, norm, X, y


def _net(theta, norm):
    net = sph.Mlp()
    net.set(theta, norm)
    return net


def test_forward_matches_bf16_emulation():
    theta, norm, X, _ = _case()
    net = _net(theta, norm)
    got = net.forward(X).cpu().numpy().astype(np.float64)
    want = mlp.forward(theta, norm, X.astype(np.float64), bf16=True)
    exact = mlp.forward(theta, norm, X.astype(np.float64))
    scale = np.max(np.abs(want - norm[12]))
    assert np.max(np.abs(got - want)) <= 2e-3 * scale
    assert np.median(np.abs(got - want)) <= 1e-5 * scale
    assert np.max(np.abs(got - exact)) <= 3e-2 * scale
    net.close()


def test_loss_and_gradient_match_bf16_emulation():
    theta, norm, X, y = _case(12, 2051)
    net = _net(theta, norm)
    L, g = net.loss_grad(X, y)
    g = g.cpu().numpy().astype(np.float64)
    Lw, gw = mlp.loss_grad(theta, norm, X.astype(np.float64), y.astype(np.float64), bf16=True)
    assert abs(L - Lw) <= 1e-4 * Lw
    assert np.max(np.abs(g - gw)) <= 2e-3 * np.max(np.abs(gw))
    # every block of the parameter vector, not just the largest entries
    for s, _ in mlp._SLICES.values():
        assert np.linalg.norm(g[s] - gw[s]) <= 5e-3 * np.linalg.norm(gw[s]) + 1e-9
    _, ge = mlp.loss_grad(theta, norm, X.astype(np.float64), y.astype(np.float64))
    assert np.max(np.abs(g - ge)) <= 5e-2 * np.max(np.abs(ge))
    # deterministic: a second evaluation gives the same bits
    L2, g2 = net.loss_grad(X, y)
    assert L2 == L and np.array_equal(g2.cpu().numpy(), g.astype(np.float32))
    net.close()


def test_masked_samples_carry_no_weight():
    theta, norm, X, y = _case(13, 700)
    bad = np.zeros(700, bool)
    bad[::7] = True
    Xn, yn = X.copy(), y.copy()
    yn[bad] = np.nan
    Xn[bad[::-1], 2] = np.inf          # some rows with a bad feature too
    keep = ~(bad | bad[::-1])
    net = _net(theta, norm)
    L0, g0 = net.loss_grad(X[keep], y[keep])
    L1, g1 = net.loss_grad(Xn, yn)
    assert np.isfinite(L1) and abs(L1 - L0) <= 1e-5 * L0
    assert np.max(np.abs(g1.cpu().numpy() - g0.cpu().numpy())) <= 1e-5 * float(g0.abs().max())
    # a gathered subset equals the same rows passed directly
    idx = np.nonzero(keep)[0][::-1].copy()
    L2, g2 = net.loss_grad(X, y, idx=idx)
    assert abs(L2 - L0) <= 1e-5 * L0
    assert np.max(np.abs(g2.cpu().numpy() - g0.cpu().numpy())) <= 1e-5 * float(g0.abs().max())
    net.close()


def test_adam_step_matches_oracle():
    theta, norm, X, y = _case(14, 512)
    net = _net(theta, norm)
    _, g = net.loss_grad(X, y)
    gh = g.cpu().numpy().astype(np.float64)
    th, mo, ve = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in (1, 2):
        net.adam_step(g, 1e-3)
        th, mo, ve = mlp.adam(th, mo, ve, gh, t, 1e-3)
    got, _ = net.get()
    assert np.max(np.abs(got - th)) <= 1e-6 + 1e-6 * np.max(np.abs(th))
    net.close()


def test_fit_norm_matches_oracle():
    rng = np.random.default_rng(15)
    X = (rng.normal(2.0, 3.0, (50000, 6)) * np.array([1, 0.1, 10, 1e-3, 0.5, 2])).astype(np.float32)
    y = rng.normal(0.01, 0.02, 50000).astype(np.float32)
    y[::11] = np.nan
    net = sph.Mlp()
    net.set(np.zeros(mlp.NPARAM), np.ones(14))
    net.fit_norm(X, y)
    _, nm = net.get()
    ok = np.isfinite(y)
    want = mlp.fit_norm(X[ok].astype(np.float64), y[ok].astype(np.float64))
    assert np.allclose(nm, want, rtol=1e-5, atol=1e-9)
    net.close()


def test_training_on_the_gpu_fits_a_smooth_function():
    """Minibatch Adam through the library's own kernels; the oracle then
    evaluates the trained parameters and agrees with the kernel's loss."""
    rng = np.random.default_rng(16)
    X = rng.normal(0, 1, (20000, 6)).astype(np.float32)
    y = (0.3 * np.sin(X[:, 0]) + 0.1 * X[:, 1] * X[:, 2] - 0.05 * X[:, 5]).astype(np.float32)
    net = sph.Mlp()
    net.set(wl.mlp_init(), np.ones(14))
    net.fit_norm(X, y)
    L0, _ = net.loss_grad(X, y)
    for ep in range(12):
        perm = np.random.default_rng(100 + ep).permutation(X.shape[0])
        net.train_epoch(X, y, perm, batch=512, lr=3e-3)
    L1, _ = net.loss_grad(X, y)
    assert L1 < 0.05 * L0
    th, nm = net.get()
    Lo, _ = mlp.loss_grad(th.astype(np.float64), nm.astype(np.float64), X.astype(np.float64),
                          y.astype(np.float64), bf16=True)
    assert abs(Lo - L1) <= 1e-3 * L1 + 1e-7
    net.close()


def test_hidden_tanh_against_numpy():
    """One path through the network isolates the second layer's tanh, which
    stays FP32: out = w3 tanh(beta bf16(tanh(alpha x))) + b3. The kernels'
    tanh (from the exponential identity) must stay within 1e-6 absolute of
    numpy's, apart from the rare first-layer value that the two round to
    different bf16 neighbours."""
    W1 = np.zeros((64, 6))
    W2 = np.zeros((64, 64))
    W3 = np.zeros(64)
    W1[9, 0], W2[30, 9], W3[30] = 1.0, 2.5, 1.0
    theta = mlp.pack(W1, np.zeros(64), W2, np.zeros(64), W3, 0.0)
    norm = np.concatenate([np.zeros(6), np.ones(6), [0.0, 1.0]])
    x = np.linspace(-6.0, 6.0, 40001).astype(np.float32)
    X = np.zeros((x.size, 6), np.float32)
    X[:, 0] = x
    net = _net(theta, norm)
    got = net.forward(X).cpu().numpy().astype(np.float64)
    net.close()
    xb = mlp.bf16_round(x.astype(np.float64))
    want = np.tanh(2.5 * mlp.bf16_round(np.tanh(xb)))
    err = np.abs(got - want)
    assert np.quantile(err, 0.999) <= 1e-6
    assert np.max(err) <= 2.5 * 2.0 ** -8      # one bf16 step of the first layer
    assert np.max(np.abs(got)) <= 1.0
