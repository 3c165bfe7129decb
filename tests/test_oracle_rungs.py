"""Pins of the oracle's hierarchical individual time steps (ref_step_rungs;
the scheme is a reading, see oracle/sphref.c):

* with R = 0 it is the global step (bit for bit);
* with every particle on the finest rung R it is 2^R global steps of
  dt / 2^R (bit for bit); with every particle on rung 0 it is one global
  step of dt up to the rounding of the substep drifts;
* isolated particles under uniform g, each on its own rung, follow the
  leapfrog's exact solution for constant acceleration with their own step;
* particles that do not interact evolve as they would alone: two distant
  clumps stepped together equal each clump stepped by itself;
* every big step ends with all particles at the same time, and the number
  of particle updates is the sum over particles of 2^rung.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import cloud

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "sxx", "sxy", "ax", "dudt", "dsxx",
          "eps_ii")


def _crit(p, st):
    a = np.sqrt(st["ax"] ** 2 + st["ay"] ** 2 + st["az"] ** 2)
    ta = np.where(a > 0, p["eta_a"] * np.sqrt(st["h"] / np.where(a > 0, a, 1.0)), np.inf)
    tc = p["eta_c"] * st["h"] / st["vsig"]
    return np.minimum(ta, tc)


def _clump(n, seed, c0=100.0, dx=0.0):
    gm = dict(wl.granular_material(), c0=c0, A=1600.0 * c0 ** 2)
    a = cloud(n, seed=seed, jitter=0.2, spacing=0.05, mat=gm, vsig=0.01, ssig=100.0)
    a["x"] += dx
    return a, gm


def _primed(a, mats, p):
    st, _ = oracle.derivatives(p, mats, a)
    return st


def test_max_rung_zero_is_the_global_step():
    a, gm = _clump(400, 1)
    p = wl.default_params(0)
    st = _primed(a, [gm], p)
    dt = 0.5 * _crit(p, st).min()
    g, gi = oracle.step(p, [gm], st, dt)
    r, ri, rung, upd = oracle.step_rungs(p, [gm], st, dt, 0)
    for f in FIELDS:
        assert np.array_equal(g[f], r[f]), f
    assert gi[-1]["e_kin"] == ri[-1]["e_kin"] and gi[-1]["dt_next"] == ri[-1]["dt_next"]
    assert np.all(rung == 0) and upd == [400]


def test_all_on_the_finest_rung_are_global_substeps():
    a, gm = _clump(400, 2)
    p = wl.default_params(0)
    st = _primed(a, [gm], p)
    R = 2
    dt = 1.1 * (2 ** R) * _crit(p, st).max()   # every particle asks for more than rung R
    g, _ = oracle.step(p, [gm], st, dt / 2 ** R, nsteps=2 ** R)
    r, _, rung, upd = oracle.step_rungs(p, [gm], st, dt, R)
    assert np.all(rung == R) and upd == [400 * 2 ** R]
    for f in FIELDS:
        assert np.array_equal(g[f], r[f]), f


def test_all_on_rung_zero_is_one_global_step():
    a, gm = _clump(400, 3)
    p = wl.default_params(0)
    st = _primed(a, [gm], p)
    dt = 0.9 * _crit(p, st).min()
    g, gi = oracle.step(p, [gm], st, dt)
    r, ri, rung, upd = oracle.step_rungs(p, [gm], st, dt, 3)
    assert np.all(rung == 0) and upd == [400]
    for f in ("x", "y", "z"):           # four substep drifts of dt / 4 against one of dt
        assert np.allclose(g[f], r[f], rtol=0, atol=1e-14 * np.abs(g[f]).max()), f
    for f in FIELDS[3:]:
        scale = np.abs(g[f]).max() or 1.0
        assert np.max(np.abs(g[f] - r[f])) <= 1e-9 * scale, f


def test_isolated_particles_integrate_constant_g_exactly_on_their_rungs():
    mat = wl.granular_material()
    n = 12
    a = wl._empty_arrays(n)
    a["x"][:] = np.arange(n) * 1e4
    a["m"][:] = np.logspace(-3, 5, n)           # support radii over a factor ~460
    a["h"][:] = wl.lattice_h(mat, a["m"])
    a["vx"][:] = np.linspace(-1, 1, n)
    a["vz"][:] = 0.5
    g = np.array([0.0, 0.0, -9.81])
    p = wl.default_params(0)
    p.update(gravity=1, g_uniform=tuple(g), max_sweeps=64)
    st = _primed(a, [mat], p)
    c = _crit(p, st)
    R = 4
    dt = 2.0 * c.max()
    out, _, rung, upd = oracle.step_rungs(p, [mat], st, dt, R)
    assert len(set(rung.tolist())) >= 3, rung
    N = 2.0 ** rung                                 # steps of dt / N each
    h = dt / N
    assert np.allclose(out["x"], a["x"] + N * h * a["vx"], rtol=1e-13, atol=1e-12)
    assert np.allclose(out["z"], N * h * 0.5 + N * (N - 1) / 2 * h * h * g[2], rtol=1e-12,
                       atol=1e-12)
    assert np.allclose(out["vz"], 0.5 + N * h * g[2], rtol=1e-12)    # v at the half step
    assert upd == [int(N.sum())]


def test_distant_clumps_evolve_as_alone():
    a1, gm1 = _clump(300, 4, c0=100.0)
    a2, gm2 = _clump(300, 5, c0=400.0, dx=50.0)
    a2["mat"][:] = 1
    both = {f: np.concatenate([a1[f], a2[f]]) for f in a1}
    both["id"] = np.arange(600)
    mats = [gm1, gm2]
    p = wl.default_params(0)
    st = _primed(both, mats, p)
    R = 3
    dt = 1.5 * _crit(p, st)[:300].min()
    out, infos, rung, upd = oracle.step_rungs(p, mats, st, dt, R, nsteps=2)
    assert len(set(rung.tolist())) >= 3, np.bincount(rung)
    s1 = {f: v[:300].copy() for f, v in st.items()}
    s2 = {f: v[300:].copy() for f, v in st.items()}
    o1, _, r1, u1 = oracle.step_rungs(p, mats, s1, dt, R, nsteps=2)
    o2, _, r2, u2 = oracle.step_rungs(p, mats, s2, dt, R, nsteps=2)
    assert np.array_equal(rung, np.concatenate([r1, r2]))
    assert upd == [x + y for x, y in zip(u1, u2)]
    for f in FIELDS:
        assert np.array_equal(out[f], np.concatenate([o1[f], o2[f]])), f
