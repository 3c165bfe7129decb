"""The no-allocation diagnostics entry point against the existing one.

sph_diagnostics_noalloc serves callers that may not allocate device memory
(a host program whose own allocator already owns the device heap, or a
monitoring hook that must leave the allocation state untouched between
steps); its scratch is an array compiled into the library. The test calls it
through the C ABI twice in a row on one state and checks both results
against the sums that the context's own reduction reports (sph_prime, whose
scratch sph_init allocated), at the FP64 tolerance the parity tests use for
global sums.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_context_sums():
    import torch

    build.build()
    w = wl.impact(9000, 1000, seed=21)
    w.arrays["u"][:] = np.linspace(0.0, 1.0e6, w.n)
    sim = sph.Simulation(w.arrays, w.materials, dict(w.params, precision=0))
    info = sim.prime()
    ref = np.array([info["e_kin"], info["e_int"], *info["p"], *info["L"]])
    a = sim.to_numpy()
    m = a["m"]
    v = np.stack([a["vx"], a["vy"], a["vz"]], 1)
    r = np.stack([a["x"], a["y"], a["z"]], 1)
    speed = np.sqrt((v * v).sum(1))
    scale = np.array([(0.5 * m * speed ** 2).sum(), (m * np.abs(a["u"])).sum()] +
                     [(m * speed).sum()] * 3 +
                     [(m * speed * np.sqrt((r * r).sum(1))).sum()] * 3)
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=sim.device)
    stream = torch.cuda.current_stream(sim.device).cuda_stream
    results = []
    for _ in range(2):
        rc = sph.lib().sph_diagnostics_noalloc(C.byref(sim.state), sim.n,
                                               C.c_void_p(out.data_ptr()), C.c_void_p(stream))
        assert rc == sph.SPH_OK
        torch.cuda.synchronize(sim.device)
        got = out.cpu().numpy().copy()
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
        results.append(got)
        out.fill_(float("nan"))
    assert np.array_equal(results[0], results[1])
    # bad sizes are refused before anything is enqueued
    assert sph.lib().sph_diagnostics_noalloc(C.byref(sim.state), 0, C.c_void_p(out.data_ptr()),
                                             C.c_void_p(stream)) == sph.SPH_E_ARG
    assert sph.lib().sph_diagnostics_noalloc(C.byref(sim.state), (1 << 31) + 1,
                                             C.c_void_p(out.data_ptr()),
                                             C.c_void_p(stream)) == sph.SPH_E_ARG
    sim.close()
