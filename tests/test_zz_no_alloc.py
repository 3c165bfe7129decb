"""The allocation-free diagnostics entry point.

sph_diagnostics_noalloc serves callers that may not allocate device memory
(a host program whose own allocator already owns the device heap, or a
monitoring hook that must leave the allocation state untouched between
steps); its scratch is an array compiled into the library. Through the C
ABI the test calls it twice in a row on one state, right after sph_prime and
again after two sph_step calls (when v and u are stored at the half step),
and checks each result
* against the FP64 oracle's sums of the same stored arrays
  (oracle.diagnostics, which shares no code with the library), at the FP64
  tolerance of the parity tests for global sums;
* against the existing entry point's sums (sph_prime's report, whose
  scratch sph_init allocated) where both describe the same state;
and that the device's free memory is the same before and after each pair of
calls (the first call may load the library's module; it is made before any
measurement)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _scale(a):
    m = a["m"]
    v = np.stack([a["vx"], a["vy"], a["vz"]], 1)
    r = np.stack([a["x"], a["y"], a["z"]], 1)
    speed = np.sqrt((v * v).sum(1))
    return np.array([(0.5 * m * speed ** 2).sum(), (m * np.abs(a["u"])).sum()] +
                    [(m * speed).sum()] * 3 +
                    [(m * speed * np.sqrt((r * r).sum(1))).sum()] * 3)


def _oracle_sums(p, a):
    d = oracle.diagnostics(p, a)
    return np.array([d["e_kin"], d["e_int"], *d["p"], *d["L"]])


def test_noalloc_sums_match_oracle_and_context_sums():
    import torch

    build.build()
    w = wl.impact(9000, 1000, seed=21)
    w.arrays["u"][:] = np.linspace(0.0, 1.0e6, w.n)
    p = dict(w.params, precision=0)
    sim = sph.Simulation(w.arrays, w.materials, p)
    info = sim.prime()
    ctx_sums = np.array([info["e_kin"], info["e_int"], *info["p"], *info["L"]])
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=sim.device)
    stream = torch.cuda.current_stream(sim.device).cuda_stream
    lib = sph.lib()

    def call():
        rc = lib.sph_diagnostics_noalloc(C.byref(sim.state), sim.n, C.c_void_p(out.data_ptr()),
                                         C.c_void_p(stream))
        assert rc == sph.SPH_OK
        torch.cuda.synchronize(sim.device)
        got = out.cpu().numpy().copy()
        out.fill_(float("nan"))
        torch.cuda.synchronize(sim.device)
        return got

    call()   # first call on the device: symbol lookup (and module load, if lazy)
    for stage in ("primed", "stepped"):
        if stage == "stepped":
            for _ in range(2):
                sim.step(0.0)
        a = sim.to_numpy()
        ref = _oracle_sums(p, a)
        scale = _scale(a)
        free0 = torch.cuda.mem_get_info(sim.device)[0]
        results = [call(), call()]
        assert torch.cuda.mem_get_info(sim.device)[0] == free0
        for got in results:
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - ref) <= 1e-12 * scale), (stage, got, ref)
        assert np.array_equal(results[0], results[1])
        if stage == "primed":
            # after sph_prime the stored v and u are those of time 0, the
            # state sph_step_info describes
            assert np.all(np.abs(results[0] - ctx_sums) <= 1e-12 * scale)
    # bad sizes are refused before anything is enqueued
    assert lib.sph_diagnostics_noalloc(C.byref(sim.state), 0, C.c_void_p(out.data_ptr()),
                                       C.c_void_p(stream)) == sph.SPH_E_ARG
    assert lib.sph_diagnostics_noalloc(C.byref(sim.state), (1 << 31) + 1,
                                       C.c_void_p(out.data_ptr()),
                                       C.c_void_p(stream)) == sph.SPH_E_ARG
    sim.close()
