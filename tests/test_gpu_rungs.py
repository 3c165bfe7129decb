"""Hierarchical individual steps on the GPU (sph_params.max_rung) against
the oracle's ref_step_rungs, through the C ABI: two distant clumps with
different sound speeds (so different rungs) and a small impact, in both
forms; the rung histogram and the number of particle updates; a captured
graph replays the substeps bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import cloud

pytestmark = pytest.mark.gpu

DERIVS = ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz")
STATE = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "sxx", "syy", "sxy", "sxz", "syz",
         "eps_ii")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _crit(p, st):
    a = np.sqrt(st["ax"] ** 2 + st["ay"] ** 2 + st["az"] ** 2)
    ta = np.where(a > 0, p["eta_a"] * np.sqrt(st["h"] / np.where(a > 0, a, 1.0)), np.inf)
    tc = p["eta_c"] * st["h"] / st["vsig"]
    return np.minimum(ta, tc)


def _clumps():
    mats = []
    parts = []
    for k, (c0, seed) in enumerate(((100.0, 4), (400.0, 5))):
        gm = dict(wl.granular_material(), c0=c0, A=1600.0 * c0 ** 2)
        a = cloud(300, seed=seed, jitter=0.2, spacing=0.05, mat=gm, vsig=0.01, ssig=100.0)
        a["x"] += 50.0 * k
        a["mat"][:] = k
        mats.append(gm)
        parts.append(a)
    arr = {f: np.concatenate([a[f] for a in parts]) for f in parts[0]}
    arr["id"] = np.arange(arr["x"].shape[0], dtype=np.int64)
    return arr, mats


def _maxnorm_err(a, b):
    scale = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)


def _run(arrays, mats, p, dt, R, nbig, graph=False):
    q = dict(p, max_rung=R)
    sim = sph.Simulation(arrays, mats, q)
    sim.prime()
    if graph:
        sim.set_graph(True)
    infos = [sim.step(dt) for _ in range(nbig)]
    g = sim.by_id()
    sim.close()
    return g, infos


@pytest.mark.parametrize("precision", [0, 1])
def test_clumps_follow_the_oracle(precision):
    arr, mats = _clumps()
    p = dict(wl.default_params(precision), h_tol=1e-10 if precision == 0 else 1e-6)
    st, _ = oracle.derivatives(p, mats, arr)
    R = 3
    dt = 1.5 * _crit(p, st)[:300].min()
    ref, rinfos, rung, upd = oracle.step_rungs(p, mats, st, dt, R, nsteps=2)
    g, infos = _run(arr, mats, p, dt, R, 2)
    hist = np.bincount(rung[arr["flags"] == 0], minlength=16)
    assert tuple(hist) == infos[-1]["rung_counts"]
    assert infos[-1]["particle_updates"] == upd[-1]
    assert len(set(rung.tolist())) >= 3
    tol = 1e-9 if precision == 0 else 1e-4
    for f in STATE + DERIVS:
        e = _maxnorm_err(g[f], ref[f])
        assert e < tol, (f, e)
    assert infos[-1]["e_kin"] == pytest.approx(rinfos[-1]["e_kin"], rel=1e-9 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_small_impact_follows_the_oracle(precision):
    w = wl.impact(9000, 1000, seed=21)
    p = dict(w.params, precision=precision, h_tol=1e-10 if precision == 0 else 1e-6)
    st, info = oracle.derivatives(p, w.materials, w.arrays)
    R = 2
    dt = 3.0 * info["dt_next"]
    ref, rinfos, rung, upd = oracle.step_rungs(p, w.materials, st, dt, R)
    g, infos = _run(w.arrays, w.materials, p, dt, R, 1)
    assert upd[0] < w.n * 2 ** R                      # fewer updates than global substeps
    hist = np.bincount(rung, minlength=16)
    got = np.array(infos[0]["rung_counts"])
    assert np.abs(got - hist).sum() <= (0 if precision == 0 else max(2, w.n // 2000))
    if precision == 0:
        assert infos[0]["particle_updates"] == upd[0]
        for f in STATE + DERIVS:
            e = _maxnorm_err(g[f], ref[f])
            assert e < 1e-9, (f, e)
    else:
        for f in STATE + DERIVS:
            e = _maxnorm_err(g[f], ref[f])
            assert e < 1e-4, (f, e)


def test_graph_replays_substeps_bit_for_bit():
    arr, mats = _clumps()
    p = dict(wl.default_params(1), h_tol=1e-6)
    st, _ = oracle.derivatives(p, mats, arr)
    dt = 1.5 * _crit(p, st)[:300].min()
    a, ia = _run(arr, mats, p, dt, 3, 3)
    b, ib = _run(arr, mats, p, dt, 3, 3, graph=True)
    for f in STATE + DERIVS:
        assert np.array_equal(a[f], b[f]), f
    assert ia[-1]["rung_counts"] == ib[-1]["rung_counts"]


def test_rejects_bad_rung_limit():
    w = wl.granular_column()
    for bad in (-1, 16):
        with pytest.raises(sph.SphError):
            sph.Simulation(w.arrays, w.materials, dict(w.params, max_rung=bad))
