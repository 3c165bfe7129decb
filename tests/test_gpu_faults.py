"""Failure detection through the C ABI, with every failure made on the host.

* A NaN internal energy in the caller's state (device arrays, and host
  arrays through sph_step_host) gives non-finite pressures and derivatives;
  the step reports SPH_E_NONFINITE. Only u is poisoned: positions, masses
  and H stay finite, so the cell list and the pair walks see a valid
  particle set and every loop keeps its data-bounded trip count.
* max_sweeps = 1 on an unrelaxed lattice with a poor first radius gives
  SPH_E_NOCONV, with the particle count the oracle reports after one sweep.
* A CUDA failure faked on the host (sph_inject_cuda_failure turns a
  successful runtime call into an error, as the runtime would report it)
  gives SPH_E_CUDA; every later call on that context returns SPH_E_STATE
  until it is destroyed, and a new context on the same device works.
* Checkpoint / restore: the state arrays are the whole state, so k steps,
  a copy to the host, a new context from that copy and N - k more steps
  equal N steps in one context bit for bit.
Nothing here faults, traps or hangs the GPU."""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import cloud

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _impact(precision):
    w = wl.impact(6000, 700, seed=71)
    return w, dict(w.params, precision=precision, h_tol=1e-10 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_energy_in_device_state_reports_nonfinite(precision):
    w, p = _impact(precision)
    sim = sph.Simulation(w.arrays, w.materials, p)
    info = sim.prime()
    sim.t["u"][w.n // 3] = float("nan")
    r = sim.step(0.5 * info["dt_next"], allow=(sph.SPH_E_NONFINITE,))
    assert r["status"] == sph.SPH_E_NONFINITE
    assert "non-finite" in sph.lib().sph_last_error(sim.ctx).decode()
    sim.close()


def test_nan_energy_in_host_state_reports_nonfinite():
    w, p = _impact(1)
    sim = sph.Simulation(w.arrays, w.materials, p)
    info = sim.prime()
    a = sim.to_numpy()
    u17 = a["u"][17]
    a["u"][17] = float("nan")
    host = sph.HostState(a)
    with pytest.raises(sph.SphError) as e:
        sim.step_host(host, 0.5 * info["dt_next"])
    assert e.value.status == sph.SPH_E_NONFINITE
    sim.close()
    # the same host state without the NaN steps cleanly
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.prime()
    a["u"][17] = u17
    r = sim.step_host(sph.HostState(a), 0.5 * info["dt_next"])
    assert np.isfinite(r["e_kin"])
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_sweep_reports_noconv(precision):
    mat = wl.basalt_material()
    a = cloud(3000, seed=72, jitter=0.2, spacing=100.0, vsig=5.0, ssig=1e6)
    a["h"] *= 1.3                       # a poor first radius
    p = dict(wl.default_params(precision), max_sweeps=1,
             h_tol=1e-10 if precision == 0 else 1e-6)
    ref, rinfo = oracle.density_solve(p, [mat], a)
    assert rinfo["n_unconverged"] > a["x"].size // 2
    sim = sph.Simulation(a, [mat], p)
    with pytest.raises(sph.SphError) as e:
        sim.prime()
    assert e.value.status == sph.SPH_E_NOCONV
    sim.close()
    sim = sph.Simulation(a, [mat], p)
    sim.neighbours()
    sw = sim.density(allow_noconv=True)
    assert sw == 1
    g = sim.by_id()
    # the last evaluation is kept: the density at the radius reached
    rho, _, cnt = oracle.density_given_h(p, dict(a, h=g["h"]))
    assert np.max(np.abs(g["rho"] / rho - 1)) < (1e-12 if precision == 0 else 1e-5)
    assert np.array_equal(cnt, g["nngb"])
    if precision == 0:
        assert np.allclose(g["h"], ref["h"], rtol=1e-12, atol=0)
    sim.close()


def test_injected_cuda_failure_leaves_the_context_unusable():
    w, p = _impact(1)
    lib = sph.lib()
    sim = sph.Simulation(w.arrays, w.materials, p)
    info = sim.prime()
    dt = 0.5 * info["dt_next"]
    sim.inject_cuda_failure(1)
    r = lib.sph_step(sim.ctx, dt, None)
    assert r == sph.SPH_E_CUDA
    assert "unknown error" in lib.sph_last_error(sim.ctx).decode()
    for rc in (lib.sph_step(sim.ctx, dt, None), lib.sph_neighbours(sim.ctx),
               lib.sph_forces_strength(sim.ctx), lib.sph_set_graph(sim.ctx, 1)):
        assert rc == sph.SPH_E_STATE
    sim.close()
    # a failure in the middle of enqueueing a step, and one in a host step
    for after, host in ((6, False), (3, True)):
        sim = sph.Simulation(w.arrays, w.materials, p)
        sim.prime()
        sim.inject_cuda_failure(after)
        if host:
            with pytest.raises(sph.SphError) as e:
                sim.step_host(sph.HostState(w.arrays), dt)
            assert e.value.status == sph.SPH_E_CUDA
        else:
            assert lib.sph_step(sim.ctx, dt, None) == sph.SPH_E_CUDA
        assert lib.sph_step(sim.ctx, dt, None) == sph.SPH_E_STATE
        sim.close()
    # cancelling a pending injection; a fresh context on the same device
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.prime()
    sim.inject_cuda_failure(2)
    sim.inject_cuda_failure(0)
    assert sim.step(dt)["status"] == sph.SPH_OK
    assert lib.sph_inject_cuda_failure(sim.ctx, -1) == sph.SPH_E_ARG
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_restore_is_bit_identical(precision):
    w, p = _impact(precision)
    _, rinfo = oracle.derivatives(p, w.materials, w.arrays)
    dt = 0.5 * rinfo["dt_next"]
    N, k = 6, 2
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.prime()
    for _ in range(N):
        sim.step(dt)
    whole = sim.by_id()
    sim.close()
    sim = sph.Simulation(w.arrays, w.materials, p)
    sim.prime()
    for _ in range(k):
        sim.step(dt)
    snap = sim.to_numpy()          # the checkpoint: every caller array
    sim.close()
    sim = sph.Simulation(snap, w.materials, p)
    for _ in range(N - k):
        sim.step(dt)
    resumed = sim.by_id()
    sim.close()
    for f in wl.FIELDS_F64 + ("nngb",):
        assert np.array_equal(whole[f], resumed[f]), f
