"""The learned smoothing-length form inside the step.

The proposal only moves the starting point of the exact Newton solve
(§2.1, Eq. 2-3), so every guess mode must still meet the oracle's parity
bar; recording samples must not change a single bit of the physics; the
recorded features must be the oracle's features of the recorded state; and
a network trained on the GPU from recorded histories must save sweeps on an
impact it was not trained on.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = sph.F64_FIELDS + sph.I32_FIELDS
DERIVS = ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _by_id(g):
    order = np.argsort(g["id"], kind="stable")
    return {k: v[order] for k, v in g.items()}


def _p(w, precision=1):
    return dict(w.params, precision=precision, h_tol=1e-6 if precision else 1e-10)


def _train(w, p, steps=20, epochs=6, seed=0):
    """A network trained on the GPU from `steps` recorded steps of w."""
    import torch
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.set_learned_h(sph.GUESS_PREVIOUS, record=True)
    sim.prime()
    Xs, ys = [], []
    for _ in range(steps):
        sim.step(0.0)
        X, y = sim.learn_samples()
        Xs.append(X.clone())
        ys.append(y.clone())
    sim.close()
    X = torch.cat(Xs)
    y = torch.cat(ys)
    net = sph.Mlp()
    net.set(wl.mlp_init(), np.ones(sph.MLP_NNORM))
    net.fit_norm(X, y)
    for ep in range(epochs):
        perm = np.random.default_rng(seed + ep).permutation(X.shape[0])
        net.train_epoch(X, y, perm, batch=4096, lr=2e-3)
    return net


def test_recording_changes_no_bits():
    w = wl.impact(12000, 1500, precision=1, seed=41)
    p = _p(w)
    out = []
    for record in (False, True):
        sim = sph.Simulation(w.arrays, w.materials, p)
        if record:
            sim.set_learned_h(sph.GUESS_PREVIOUS, record=True)
        sim.prime()
        for _ in range(3):
            sim.step(0.0)
        out.append(_by_id(sim.to_numpy()))
        sim.close()
    for f in FIELDS:
        assert np.array_equal(out[0][f], out[1][f]), f


def test_recorded_samples_are_the_oracle_features():
    w = wl.impact(20000, 2500, precision=1, seed=42)
    p = _p(w)
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.set_learned_h(sph.GUESS_PREVIOUS, record=True)
    sim.prime()
    s0 = _by_id(sim.to_numpy())
    i1 = sim.step(0.0)
    s1 = _by_id(sim.to_numpy())
    sim.step(0.0)
    s2 = _by_id(sim.to_numpy())
    X, y = sim.learn_samples()
    sim.close()
    X = X.cpu().numpy().astype(np.float64)
    y = y.cpu().numpy().astype(np.float64)
    mat = w.materials[0]
    # the velocities the step-1 evaluation used: v + dt/2 a (Eq. 40)
    dt1 = i1["dt"]
    v = [s0[c] + 0.5 * dt1 * s0[a] for c, a in (("vx", "ax"), ("vy", "ay"), ("vz", "az"))]
    _, info = oracle.forces(p, w.materials, s1, v=v, want_tensors=True)
    trg = np.trace(info["G"], axis1=1, axis2=2)
    F = mlp.features(s1["h"], s1["nngb"], s1["rho"], s1["omega"], dt1 * trg, s0["h"],
                     p["n_ngb"], s1["m"], mat["rho0"])
    for k in (0, 1, 2, 4, 5):
        assert np.max(np.abs(X[:, k] - F[:, k])) <= 1e-6 * max(1.0, np.max(np.abs(F[:, k]))), k
    # dt tr G from the FP32 pair sums with the correction tensor
    assert np.max(np.abs(X[:, 3] - F[:, 3])) <= 1e-3 * np.max(np.abs(F[:, 3]))
    assert np.max(np.abs(y - np.log(s2["h"] / s1["h"]))) <= 1e-6


@pytest.mark.parametrize("guess", [sph.GUESS_CONTINUITY, sph.GUESS_NETWORK])
def test_every_guess_keeps_oracle_parity(guess):
    """Starting points differ, the exact solve judges: counts exact,
    density 1e-5, derivatives 1e-4 of the max norm."""
    w = wl.impact(30000, 3500, precision=1, seed=43)
    p = _p(w)
    net = None
    if guess == sph.GUESS_NETWORK:
        net = sph.Mlp()
        # an untrained network: large, arbitrary proposals within the limits
        norm = np.concatenate([np.zeros(6), np.full(6, 0.01), [0.0, 0.2]])
        net.set(wl.mlp_init(5), norm)
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.set_learned_h(guess, net=net)
    sim.prime()
    for _ in range(3):
        sim.step(0.0)
    sim.forces_strength()
    g = sim.to_numpy()
    sim.close()
    rho, om, cnt = oracle.density_given_h(p, g)
    assert np.array_equal(cnt, g["nngb"])
    assert np.max(np.abs(g["rho"] / rho - 1)) < 1e-5
    st, S = oracle.eos_yield(p, w.materials, g)
    out, _ = oracle.forces(p, w.materials, st, S=S)
    for f in DERIVS:
        scale = np.max(np.abs(g[f]))
        assert np.max(np.abs(g[f] - out[f])) <= 1e-4 * scale, f
    # the converged radius meets the solve's tolerance whatever the guess
    dens = oracle.density_given_h(p, g)[0]
    hbar3 = 3 * p["n_ngb"] * g["m"] / (4 * np.pi)
    gq = g["h"] ** 3 * dens / hbar3 - 1
    assert np.quantile(np.abs(gq), 0.99) < 2e-5


def test_trained_network_saves_sweeps_on_an_unseen_impact():
    wa = wl.impact(90000, 10000, precision=1, seed=44)
    net = _train(wa, _p(wa))
    wb = wl.impact(90000, 10000, precision=1, seed=45, angle_deg=30.0, v_imp=8.0e3)
    p = _p(wb)
    mean_sweeps = {}
    for guess in (sph.GUESS_PREVIOUS, sph.GUESS_NETWORK):
        sim = sph.Simulation(wb.arrays, wb.materials, p)
        sim.set_learned_h(guess, net=net if guess == sph.GUESS_NETWORK else None)
        sim.prime()
        sw = [sim.step(0.0)["sweeps_total"] / wb.n for _ in range(10)]
        mean_sweeps[guess] = float(np.mean(sw[2:]))
        sim.close()
    assert mean_sweeps[sph.GUESS_NETWORK] < mean_sweeps[sph.GUESS_PREVIOUS] - 0.05, mean_sweeps


def test_learned_mode_needs_ids_in_range_and_a_network():
    w = wl.impact(3000, 400, precision=0, seed=46)
    a = {k: v.copy() for k, v in w.arrays.items()}
    a["id"][5] = 10 ** 9
    sim = sph.Simulation(a, w.materials, _p(w, 0))
    with pytest.raises(sph.SphError):
        sim.set_learned_h(sph.GUESS_CONTINUITY)
    sim.close()
    sim = sph.Simulation(w.arrays, w.materials, _p(w, 0))
    with pytest.raises(sph.SphError):
        sim.set_learned_h(sph.GUESS_NETWORK, net=None)
    with pytest.raises(sph.SphError):
        sim.learn_samples()
    sim.close()


def _proposal_run(guess, theta=None, norm=None, seed=43):
    """Proposal of step 1 (by id), the features it was made from (recorded
    by step 2, by id) and the radii of step 1."""
    w = wl.impact(20000, 2500, precision=1, seed=seed)
    p = _p(w)
    sim = sph.Simulation(w.arrays, w.materials, p)
    net = None
    if guess == sph.GUESS_NETWORK:
        net = sph.Mlp()
        net.set(theta, norm)
    sim.set_learned_h(guess, record=True, net=net)
    sim.prime()
    sim.step(0.0)
    s1 = sim.to_numpy(["h", "id"])
    prop = sim.learn_proposal().cpu().numpy()
    sim.step(0.0)
    X, _ = sim.learn_samples()
    sim.close()
    if net is not None:
        net.close()
    order = np.argsort(s1["id"], kind="stable")
    return prop[order], s1["h"][order], X.cpu().numpy().astype(np.float64)


LOG_LIM = np.log(1.25)   # proposals limited to [0.8, 1.25] H


def test_in_step_network_proposal_matches_the_oracle():
    """The in-step guess (k_learn: tanh.approx on bf16 pairs) element by
    element against oracle/mlp.py's forward pass on the same features.
    Error bound per particle, from the in-step path's extra roundings: the
    standardised features (FP32, then bf16: one bf16 ulp apart at most)
    through |W1|; the first layer's pre-activation rounded to bf16 (2^-9
    relative) and its tanh approximate (within 3 2^-9 absolute of the
    oracle's bf16 value), carried through |W2|; the second layer likewise;
    then |W3| and y_sd."""
    theta = wl.mlp_init()
    x_sd = [0.05, 0.2, 0.05, 2e-3, 0.01, 0.1]
    norm = np.array([0.0] * 6 + x_sd + [0.0, 0.05])
    prop, H, X = _proposal_run(sph.GUESS_NETWORK, theta, norm)
    pred, t = mlp.forward(theta, norm, X, bf16=True, keep=True)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    xb = mlp.bf16_round(t["x"])
    W1b = mlp.bf16_round(W1)
    z1 = xb @ W1b.T + b1
    # the FP32 standardisation may round a feature to the neighbouring bf16
    # value (one bf16 ulp, 2^-8 relative)
    ez1 = 2.0 ** -9 * np.abs(z1) + (2.0 ** -8 * np.abs(xb)) @ np.abs(W1b).T
    e1 = ez1 / np.cosh(z1) ** 2 + 3 * 2.0 ** -9
    z2 = mlp.bf16_round(t["a1"]) @ mlp.bf16_round(W2).T + b2
    e2 = e1 @ np.abs(mlp.bf16_round(W2)).T + 2.0 ** -9 * np.abs(z2) + 3 * 2.0 ** -9
    bound = norm[13] * (e2 @ np.abs(W3)) + 1e-6
    want = np.clip(pred, -LOG_LIM, LOG_LIM)
    got = np.log(prop / H)
    err = np.abs(got - want)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), (err.max(), bound[np.argmax(err - bound)])
    # typical error far inside the bound, far below the spread of the proposals
    rms = float(np.sqrt(np.mean(err ** 2)))
    print("proposal error: rms %.3e, max %.3e, median bound %.3e, spread %.3e"
          % (rms, err.max(), np.median(bound), np.std(want)))
    assert rms < 0.05 * np.std(want)


def test_in_step_continuity_proposal_is_exact():
    """The continuity guess H exp(-dt tr G / 3) from the recorded f3 = dt
    tr G, to FP32 rounding."""
    prop, H, X = _proposal_run(sph.GUESS_CONTINUITY)
    want = np.clip(-X[:, 3] / 3.0, -LOG_LIM, LOG_LIM)
    assert np.max(np.abs(np.log(prop / H) - want)) < 1e-6
