"""The C ABI without a GPU: the library loads, exports every function that
include/sph.h declares, and the binding's struct layouts match the C
compiler's. No compute call is made here."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2603_19764_b300 import build, sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def libsph():
    build.build()
    return C.CDLL(sph.LIB_PATH)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sph_init", "sph_neighbours", "sph_density", "sph_forces_strength",
                     "sph_stress_update", "sph_step", "sph_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(libsph):
    out = subprocess.check_output(["nm", "-D", "--defined-only", sph.LIB_PATH], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(libsph, name)
    assert set(sph.EXPORTS) <= set(declared_functions())


def _c_layout():
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "sph.h"
#define S(T) printf(#T " %zu\n", sizeof(T));
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  S(sph_state) S(sph_material) S(sph_params) S(sph_step_info) S(sph_tune_report) S(sph_peak_report)
  O(sph_state, id) O(sph_state, nngb) O(sph_material, strength) O(sph_material, xi)
  O(sph_params, g_table) O(sph_params, g_n) O(sph_params, box_hi) O(sph_params, precision)
  O(sph_params, gradient_form)
  O(sph_step_info, pairs_density) O(sph_step_info, device_flags) O(sph_step_info, sweeps)
  O(sph_step_info, kernel_launches) O(sph_step_info, n_expanded)
  O(sph_step_info, particle_updates) O(sph_step_info, rung_counts) O(sph_params, max_rung)
  O(sph_tune_report, timed) O(sph_tune_report, ms_density) O(sph_tune_report, ms_forces)
  O(sph_tune_report, depth_density) O(sph_tune_report, n_depth)
  O(sph_tune_report, depth_timed) O(sph_tune_report, ms_depth_density)
  O(sph_tune_report, ms_depth_forces)
  O(sph_peak_report, sm_mhz) O(sph_peak_report, n_sm)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), "-o", exe, c])
        out = subprocess.check_output([exe], text=True)
    return dict(ln.rsplit(" ", 1) for ln in out.strip().splitlines())


def test_struct_layouts_match_binding():
    lay = _c_layout()
    py = {"sph_state": sph.SphState, "sph_material": sph.SphMaterial,
          "sph_params": sph.SphParams, "sph_step_info": sph.SphStepInfo,
          "sph_tune_report": sph.SphTuneReport, "sph_peak_report": sph.SphPeakReport}
    for name, cls in py.items():
        assert int(lay[name]) == C.sizeof(cls), name
    for key, val in lay.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(py[t], f).offset == int(val), key


def test_status_strings(libsph):
    libsph.sph_status_string.restype = C.c_char_p
    for k, name in enumerate(sph.STATUS_NAMES):
        s = libsph.sph_status_string(k)
        assert s and len(s) > 1


def test_fma_peak_rejects_bad_arguments_without_touching_the_gpu(libsph):
    libsph.sph_measure_fma_peak.restype = C.c_int
    r = sph.SphPeakReport()
    assert libsph.sph_measure_fma_peak(2, 10, C.byref(r), None) == sph.SPH_E_ARG
    assert libsph.sph_measure_fma_peak(1, 0, C.byref(r), None) == sph.SPH_E_ARG
    assert libsph.sph_measure_fma_peak(1, 10, None, None) == sph.SPH_E_ARG


def test_init_rejects_bad_arguments_without_touching_the_gpu(libsph):
    """Argument checks run before any CUDA call."""
    libsph.sph_init.restype = C.c_int
    ctx = C.c_void_p()
    assert libsph.sph_init(C.byref(ctx), None, None, 1, None, 10, None) == sph.SPH_E_ARG
    assert libsph.sph_init(None, None, None, 1, None, 10, None) == sph.SPH_E_ARG
    assert ctx.value is None
    libsph.sph_destroy.restype = C.c_int
    assert libsph.sph_destroy(None) == sph.SPH_OK


def test_tuning_setters_reject_a_missing_context_without_touching_the_gpu(libsph):
    for name, args in (("sph_autotune", (2,)), ("sph_set_spans", (1, 2)),
                       ("sph_set_stage_depths", (3, 4)), ("sph_set_copy_chunks", (8,))):
        f = getattr(libsph, name)
        f.restype = C.c_int
        assert f(None, *[C.c_int32(a) for a in args]) == sph.SPH_E_ARG, name
    libsph.sph_tune_info.restype = C.c_int
    r = sph.SphTuneReport()
    assert libsph.sph_tune_info(None, C.byref(r)) == sph.SPH_E_ARG


def test_batch_init_rejects_bad_system_bounds_without_touching_the_gpu(libsph):
    """System bounds are checked on the host before any CUDA call."""
    from paper_2603_19764_b300 import workloads as wl
    w = wl.impact(500, 60, seed=3)
    keep = []
    p = sph.make_params(dict(w.params, precision=0), keep)
    mats = (sph.SphMaterial * 1)(sph.make_material(w.materials[0]))
    st = sph.state_from_ptrs({f: 4096 for f in sph.F64_FIELDS + sph.I32_FIELDS + ("id",)})
    f = libsph.sph_init_batch
    f.restype = C.c_int
    f.argtypes = [C.POINTER(C.c_void_p), C.POINTER(sph.SphParams), C.POINTER(sph.SphMaterial),
                  C.c_int32, C.POINTER(sph.SphState), C.c_int64, C.c_int32,
                  C.POINTER(C.c_int64), C.c_void_p]
    n = 100
    ctx = C.c_void_p()

    def call(bounds, nsys=None):
        b = (C.c_int64 * len(bounds))(*bounds)
        k = len(bounds) - 1 if nsys is None else nsys
        return f(C.byref(ctx), C.byref(p), mats, 1, C.byref(st), n, k, b, None)

    assert call([1, 50, 100]) == sph.SPH_E_ARG          # does not start at 0
    assert call([0, 50, 99]) == sph.SPH_E_ARG           # does not end at n
    assert call([0, 50, 50, 100]) == sph.SPH_E_ARG      # empty system
    assert call([0, 60, 40, 100]) == sph.SPH_E_ARG      # decreasing
    assert call([0, 100], nsys=0) == sph.SPH_E_ARG      # no system
    assert call([0] * 1026, nsys=sph.SPH_MAX_SYSTEMS + 1) == sph.SPH_E_ARG
    assert f(C.byref(ctx), C.byref(p), mats, 1, C.byref(st), n, 2, None, None) == sph.SPH_E_ARG
    assert ctx.value is None
    # an unknown gradient form or rung limit is refused before any CUDA call
    for bad in (dict(gradient_form=2), dict(gradient_form=-1), dict(max_rung=16),
                dict(max_rung=-1)):
        q = sph.make_params(dict(w.params, precision=0, **bad), keep)
        b = (C.c_int64 * 2)(0, n)
        assert f(C.byref(ctx), C.byref(q), mats, 1, C.byref(st), n, 1, b, None) == sph.SPH_E_ARG
    assert ctx.value is None
