"""FP64 oracle of the learned smoothing-length proposal.

TEST INFRASTRUCTURE. Only the test suite and the benchmark's oracle legs
import this module; the product path never does, and the two share no code.

The paper has no learned component: its smoothing-length solve (§2.1,
Eq. 2-3) starts every Newton iteration from the previous support radius.
The learned form proposes the starting radius instead, with a 6-64-64-1
perceptron (tanh hidden units, linear output) that maps standardised
features of particle i at step n to the standardised log(H_{n+1} / H_n).
The exact Newton solve still decides H_{n+1}; the network only moves its
starting point.

Features of particle i at step n (H the support radius of §2.1, n_i the
neighbour count, rho_i and Omega_i from Eq. 1 and Eq. 3, tr G = div v the
trace of the corrected velocity gradient of Eq. 18-20, dt the step of
Eq. 38-39, H_bar the lattice radius (3 N_ngb m_i / (4 pi rho0))^(1/3)):

    f0 = log(H_n / H_bar)        f1 = n_n / N_ngb - 1
    f2 = log(rho_n / rho0)       f3 = dt_n * (div v)_n
    f4 = log(H_n / H_{n-1})      f5 = Omega_n - 1

Parameter vector (4673 values; the library uses the same order):
    W1[64][6] (row k = hidden unit k), b1[64], W2[64][64] (row = unit of
    the second layer, column = unit of the first), b2[64], W3[64], b3.
Normalisation (14 values): x_mu[6], x_sd[6], y_mu, y_sd.

Loss over m samples: L = 1/(2m) sum_s (out_s - (y_s - y_mu) / y_sd)^2.

``bf16=True`` rounds at the points where the library's tensor-core kernels
hold bfloat16 operands (standardised features, W1, W2, the first hidden
layer, and the back-propagated errors entering the two matrix products);
everything else, and every accumulation, stays FP64 here.
"""
from __future__ import annotations

import math

import numpy as np

NIN, NHID = 6, 64
NPARAM = NHID * NIN + NHID + NHID * NHID + NHID + NHID + 1   # 4673
NNORM = 2 * NIN + 2

_SLICES = {}
_o = 0
for _name, _shape in (("W1", (NHID, NIN)), ("b1", (NHID,)), ("W2", (NHID, NHID)),
                      ("b2", (NHID,)), ("W3", (NHID,)), ("b3", (1,))):
    _n = int(np.prod(_shape))
    _SLICES[_name] = (slice(_o, _o + _n), _shape)
    _o += _n
assert _o == NPARAM


def unpack(theta):
    """Views of the parameter vector: W1, b1, W2, b2, W3, b3 (b3 scalar)."""
    th = np.asarray(theta, np.float64)
    out = [th[s].reshape(shape) for s, shape in (_SLICES[k] for k in
                                                ("W1", "b1", "W2", "b2", "W3", "b3"))]
    out[5] = out[5][0]
    return out


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(W3), np.atleast_1d(b3)]).astype(np.float64)


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits
    of an IEEE binary32. The value is first rounded to binary32, then the low
    16 bits of that word are rounded away: add 0x7FFF plus the lowest kept
    bit and truncate."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    r = r.astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def features(h, nngb, rho, omega, dt_divv, h_prev, n_ngb, m, rho0):
    """The six features above, one row per particle."""
    h = np.asarray(h, np.float64)
    hbar = np.cbrt(3.0 * n_ngb * np.asarray(m, np.float64) / (4.0 * math.pi * rho0))
    return np.stack([np.log(h / hbar),
                     np.asarray(nngb, np.float64) / n_ngb - 1.0,
                     np.log(np.asarray(rho, np.float64) / rho0),
                     np.asarray(dt_divv, np.float64),
                     np.log(h / np.asarray(h_prev, np.float64)),
                     np.asarray(omega, np.float64) - 1.0], axis=1)


def _std(X, norm):
    norm = np.asarray(norm, np.float64)
    return (np.asarray(X, np.float64) - norm[:NIN]) / norm[NIN:2 * NIN]


def forward(theta, norm, X, bf16: bool = False, keep: bool = False):
    """Prediction of log(H_{n+1}/H_n) for every row of X (un-standardised).
    keep = True also returns the intermediate layers."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    x = r(_std(X, norm))
    z1 = x @ r(W1).T + b1
    a1 = np.tanh(z1)
    z2 = r(a1) @ r(W2).T + b2
    a2 = np.tanh(z2)
    out = a2 @ W3 + b3
    norm = np.asarray(norm, np.float64)
    pred = norm[2 * NIN] + norm[2 * NIN + 1] * out
    if keep:
        return pred, dict(x=x, a1=a1, a2=a2, out=out)
    return pred


def loss_grad(theta, norm, X, y, bf16: bool = False):
    """(L, dL/dtheta) by back-propagation through the layers above."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    norm = np.asarray(norm, np.float64)
    _, t = forward(theta, norm, X, bf16, keep=True)
    m = t["out"].shape[0]
    yh = (np.asarray(y, np.float64) - norm[2 * NIN]) / norm[2 * NIN + 1]
    e = t["out"] - yh
    L = 0.5 * float(np.dot(e, e)) / m
    d3 = e / m                                   # dL/d out
    gW3 = t["a2"].T @ d3
    gb3 = d3.sum()
    d2 = np.outer(d3, W3) * (1.0 - t["a2"] ** 2)  # dL/d z2
    gb2 = d2.sum(0)
    gW2 = r(d2).T @ r(t["a1"])
    d1 = (r(d2) @ r(W2)) * (1.0 - t["a1"] ** 2)   # dL/d z1
    gb1 = d1.sum(0)
    gW1 = r(d1).T @ t["x"]
    return L, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam(theta, mom, vel, grad, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) at step t >= 1."""
    mom = beta1 * np.asarray(mom, np.float64) + (1.0 - beta1) * grad
    vel = beta2 * np.asarray(vel, np.float64) + (1.0 - beta2) * grad * grad
    mh = mom / (1.0 - beta1 ** t)
    vh = vel / (1.0 - beta2 ** t)
    return np.asarray(theta, np.float64) - lr * mh / (np.sqrt(vh) + eps), mom, vel


def fit_norm(X, y, floor: float = 1e-6) -> np.ndarray:
    """Means and standard deviations of the features and the target."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    sd = np.maximum(X.std(0), floor)
    return np.concatenate([X.mean(0), sd, [y.mean(), max(float(y.std()), floor)]])
