"""The batched form: many independent impacts in one context.

A batch is a set of systems that never interact. Each system has its own
bounding box, cell grid, 32-particle buckets, time step and sums, so the
batched step must give every system exactly the bits that the same system
gives when stepped alone (64 sequential plain launches are the comparison
the batched form is measured against). A CUDA-graph replay of the step must
give the same bits as direct launches. Steps are adaptive: every system
takes its own dt_next (Eq. 38-39).
"""
import numpy as np
import pytest

import oracle

from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = sph.F64_FIELDS + sph.I32_FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _batch(precision, n_systems=6, scale=0.05):
    return wl.impact_batch(n_systems, precision=precision, scale=scale)


def _by_id(g):
    order = np.argsort(g["id"], kind="stable")
    return {k: v[order] for k, v in g.items()}


def _run(w, p, steps, systems=None, graph=False):
    sim = sph.Simulation(w.arrays, w.materials, p, systems=systems)
    if graph:
        sim.set_graph(True)
    infos = [sim.prime()]
    for _ in range(steps):
        infos.append(sim.step_batch(np.zeros(sim.nsys)) if systems is not None else sim.step(0.0))
    per = sim.batch_info() if systems is not None else None
    g = _by_id(sim.to_numpy())
    sim.close()
    return g, infos, per


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_bits_equal_sequential(precision):
    w = _batch(precision)
    p = dict(w.params, precision=precision, h_tol=1e-10 if precision == 0 else 1e-6)
    steps = 3
    gb, _, per = _run(w, p, steps, systems=w.systems)
    assert len(per) == len(w.systems)
    for k, (off, cnt) in enumerate(w.systems):
        ws = w.system(k)
        gs, infos, _ = _run(ws, p, steps)
        for f in FIELDS:
            a, b = gb[f][off:off + cnt], gs[f]
            assert np.array_equal(a, b), (k, f, np.max(np.abs(a - b)))
        assert np.array_equal(gb["id"][off:off + cnt] - off, gs["id"])
        last = infos[-1]
        for key in ("e_kin", "e_int", "e_pot", "dt", "dt_next"):
            assert per[k][key] == last[key], (k, key, per[k][key], last[key])
        assert per[k]["p"] == last["p"] and per[k]["L"] == last["L"]


def test_batch_graph_replay_bits_equal():
    w = _batch(1, n_systems=5)
    p = dict(w.params, precision=1, h_tol=1e-6)
    g0, i0, _ = _run(w, p, 4, systems=w.systems)
    g1, i1, _ = _run(w, p, 4, systems=w.systems, graph=True)
    for f in FIELDS:
        assert np.array_equal(g0[f], g1[f]), f
    assert [i["e_kin"] for i in i0] == [i["e_kin"] for i in i1]


def test_single_system_graph_with_changing_dt():
    """The graph reads dt from a staging buffer at replay, so a new dt per
    call needs no re-capture."""
    w = wl.impact(6000, 800, seed=33)
    p = dict(w.params, precision=0)
    sims = []
    for graph in (False, True):
        sim = sph.Simulation(w.arrays, w.materials, p)
        sim.set_graph(graph)
        d0 = sim.prime()["dt_next"]
        for k in range(3):
            info = sim.step(d0 * (0.5 + 0.1 * k))
            # drift, box, grid, keys, 4 x 5 radix kernels, permutation (2),
            # cells (2), predict, density, EOS pack, forces, kick, sums
            assert info["kernel_launches"] == 34
        sim.step(0.0)   # dt_next of the last step
        sims.append(_by_id(sim.to_numpy()))
        sim.close()
    for f in FIELDS:
        assert np.array_equal(sims[0][f], sims[1][f]), f


def test_batch_rejects_bad_bounds():
    w = _batch(0, n_systems=3)
    p = dict(w.params, precision=0)
    bad = [w.systems[0], (w.systems[1][0] + 1, w.systems[1][1] - 1), w.systems[2]]
    with pytest.raises(ValueError):
        sph.Simulation(w.arrays, w.materials, p, systems=bad)
    # ids outside 0..n-1 are refused by the device validation
    a = {k: v.copy() for k, v in w.arrays.items()}
    a["id"][7] = w.n + 3
    with pytest.raises(sph.SphError):
        sph.Simulation(a, w.materials, p, systems=w.systems)
    # radial-table gravity is a single-system feature
    with pytest.raises(sph.SphError):
        sph.Simulation(w.arrays, w.materials,
                       dict(p, gravity=2, g_table=np.ones(8), phi_table=np.ones(8),
                            g_rmin=1.0, g_rmax=1e5, g_gm=1.0), systems=w.systems)


def _tuned_run(w, p, steps, rounds, graph):
    sim = sph.Simulation(w.arrays, w.materials, p, systems=w.systems)
    sim.set_graph(graph)
    sim.prime()
    if rounds:
        sim.autotune(rounds)
    for _ in range(steps):
        sim.step_batch(np.zeros(sim.nsys))
    rep = sim.tune_info()
    g = _by_id(sim.to_numpy())
    sim.close()
    return g, rep


def test_autotune_leaves_fp64_bits_unchanged():
    """Every candidate group span visits each particle's neighbours in the
    same order, so tuning steps in the FP64 form give the untuned bits."""
    w = _batch(0, n_systems=4)
    p = dict(w.params, precision=0, h_tol=1e-10)
    g0, rep0 = _tuned_run(w, p, 8, 0, False)
    g1, rep1 = _tuned_run(w, p, 8, 2, True)
    assert rep0["span_density"] == 2 and rep0["span_forces"] == 2
    assert rep1["steps_left"] == 0 and rep1["timed"] == [2, 2, 2]
    assert rep1["span_density"] in rep1["cand"] and rep1["span_forces"] in rep1["cand"]
    assert all(t > 0 for t in rep1["ms_density"] + rep1["ms_forces"])
    for f in FIELDS:
        assert np.array_equal(g0[f], g1[f]), f


@pytest.mark.parametrize("span", [1, 2, 3])
def test_every_span_fp32_parity_after_tuning(span):
    """After a tuned run, the FP32 form with each group span against the
    oracle, system by system, on the state it reached: counts exact,
    density 1e-5 relative, derivatives 1e-4 of the max norm."""
    w = _batch(1, n_systems=4)
    p = dict(w.params, precision=1, h_tol=1e-6)
    sim = sph.Simulation(w.arrays, w.materials, p, systems=w.systems)
    sim.prime()
    sim.autotune(1)
    for _ in range(5):   # three span steps, then two staging-depth steps
        sim.step_batch(np.zeros(sim.nsys))
    rep = sim.tune_info()
    assert rep["steps_left"] == 0 and rep["depth_timed"] == [1, 1]
    assert rep["depth_density"] in (3, 4) and rep["depth_forces"] in (3, 4)
    sim.set_spans(span, span)
    sim.density()
    sim.forces_strength()
    ga = sim.to_numpy()
    sim.close()
    for off, cnt_k in w.systems:
        g = {k: v[off:off + cnt_k].copy() for k, v in ga.items()}
        rho, om, cnt = oracle.density_given_h(p, g)
        assert np.array_equal(cnt, g["nngb"])
        assert np.max(np.abs(g["rho"] / rho - 1)) < 1e-5
        st, S = oracle.eos_yield(p, w.materials, g)
        out, _ = oracle.forces(p, w.materials, st, S=S)
        for f in ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz"):
            scale = np.max(np.abs(g[f]))
            assert np.max(np.abs(g[f] - out[f])) <= 1e-4 * scale, (off, f)


def test_set_spans_rejects_out_of_range():
    w = _batch(0, n_systems=2)
    sim = sph.Simulation(w.arrays, w.materials, dict(w.params, precision=0), systems=w.systems)
    for bad in ((0, 2), (2, 4), (-1, -1)):
        with pytest.raises(sph.SphError):
            sim.set_spans(*bad)
    sim.close()


@pytest.mark.parametrize("graph", [False, True])
def test_staging_depth_changes_no_bit(graph):
    """The FP32 form's staging depth (chunks of 32 candidate positions
    located and loaded before the first is tested) only overlaps loads: the
    chunks are consumed in order, so every depth builds the same candidate
    lists and steps to the same bits."""
    w = _batch(1, n_systems=4)
    p = dict(w.params, precision=1, h_tol=1e-6)
    out = []
    for depths in ((3, 3), (4, 4), (3, 4)):
        sim = sph.Simulation(w.arrays, w.materials, p, systems=w.systems)
        sim.set_graph(graph)
        sim.set_stage_depths(*depths)
        sim.prime()
        for _ in range(3):
            sim.step_batch(np.zeros(sim.nsys))
        rep = sim.tune_info()
        assert (rep["depth_density"], rep["depth_forces"]) == depths
        out.append(_by_id(sim.to_numpy()))
        sim.close()
    for g in out[1:]:
        for f in FIELDS:
            assert np.array_equal(g[f], out[0][f]), f


def test_set_stage_depths_rejects_uncompiled_depths():
    w = _batch(1, n_systems=2)
    sim = sph.Simulation(w.arrays, w.materials, dict(w.params, precision=1), systems=w.systems)
    for bad in ((2, 3), (3, 5), (0, 0)):
        with pytest.raises(sph.SphError):
            sim.set_stage_depths(*bad)
    sim.close()

