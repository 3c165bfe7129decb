"""Python binding of libsph (include/sph.h): argument marshalling only.

Every step of the SPH path runs in the CUDA library; this module loads it
with ctypes, mirrors its structs, and hands it the device pointers of torch
tensors. There is no fallback: if libsph.so is missing or CUDA is not
available the calls raise.

Function names follow the C ABI: sph_init, sph_neighbours, sph_density,
sph_forces_strength, sph_stress_update, sph_step, sph_step_host, sph_prime,
sph_destroy. ``Simulation`` bundles a workload's arrays as device tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_CHECKED=1 in the environment selects the checked build (index tests on
# every data-derived index; paper_2603_19764_b300.build(checked=True))
LIB_PATH = os.path.join(_HERE, "libsph_check.so" if os.environ.get("SPH_CHECKED") == "1"
                        else "libsph.so")
_lib = None

SPH_OK, SPH_E_ARG, SPH_E_CUDA, SPH_E_NOCONV, SPH_E_CAPACITY, SPH_E_NONFINITE, \
    SPH_E_TIMEOUT, SPH_E_STATE, SPH_E_INTERNAL = range(9)
STATUS_NAMES = ["SPH_OK", "SPH_E_ARG", "SPH_E_CUDA", "SPH_E_NOCONV", "SPH_E_CAPACITY",
                "SPH_E_NONFINITE", "SPH_E_TIMEOUT", "SPH_E_STATE", "SPH_E_INTERNAL"]
MAX_MATERIALS = 8
SPH_MAX_SYSTEMS = 1024


class SphError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s returned %s%s" % (where, name, (": " + detail) if detail else ""))


_P = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int32)
_PL = C.POINTER(C.c_int64)

F64_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h", "sxx", "syy", "sxy", "sxz", "syz",
              "rho", "omega", "pres", "cs", "ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy",
              "dsxz", "dsyz", "eps_ii")
I32_FIELDS = ("nngb", "mat", "flags")


class SphState(C.Structure):
    _fields_ = ([(f, _P) for f in F64_FIELDS] + [(f, _PI) for f in I32_FIELDS] + [("id", _PL)])


class SphMaterial(C.Structure):
    _fields_ = [("eos", C.c_int32), ("rho0", C.c_double), ("c0", C.c_double),
                ("A", C.c_double), ("B", C.c_double), ("E0", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("Eiv", C.c_double), ("Ecv", C.c_double), ("shear_G", C.c_double),
                ("Y0", C.c_double), ("mu_i", C.c_double), ("Ym", C.c_double),
                ("mu_d", C.c_double), ("thermal_softening", C.c_int32), ("xi", C.c_double),
                ("Tm", C.c_double), ("T0", C.c_double), ("cv", C.c_double),
                ("strength", C.c_int32), ("p_min", C.c_double)]


class SphParams(C.Structure):
    _fields_ = [("n_ngb", C.c_int32), ("av_alpha", C.c_double), ("av_beta", C.c_double),
                ("av_eps", C.c_double), ("eta_c", C.c_double), ("eta_a", C.c_double),
                ("h_tol", C.c_double), ("max_sweeps", C.c_int32), ("h_cap_factor", C.c_double),
                ("precision", C.c_int32), ("jaumann", C.c_int32), ("yield_norm", C.c_int32),
                ("correction_tensor", C.c_int32), ("gravity", C.c_int32),
                ("g_uniform", C.c_double * 3), ("g_table", _P), ("phi_table", _P),
                ("g_n", C.c_int32), ("g_rmin", C.c_double), ("g_rmax", C.c_double),
                ("g_center", C.c_double * 3), ("g_gm", C.c_double), ("periodic", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("gradient_form", C.c_int32), ("max_rung", C.c_int32)]


class SphStepInfo(C.Structure):
    _fields_ = [("dt", C.c_double), ("dt_next", C.c_double), ("e_kin", C.c_double),
                ("e_int", C.c_double), ("e_pot", C.c_double), ("p", C.c_double * 3),
                ("L", C.c_double * 3), ("sweeps", C.c_int32), ("n_unconverged", C.c_int32),
                ("n_capped", C.c_int32), ("n_cfallback", C.c_int32),
                ("pairs_density", C.c_int64), ("pairs_force", C.c_int64),
                ("device_flags", C.c_uint32), ("cand_density", C.c_int64),
                ("cand_force", C.c_int64), ("groups_density", C.c_int64),
                ("groups_force", C.c_int64), ("kernel_launches", C.c_int32),
                ("sweeps_total", C.c_int64), ("n_expanded", C.c_int32),
                ("particle_updates", C.c_int64), ("rung_counts", C.c_int32 * 16)]

    def as_dict(self) -> dict:
        return dict(dt=self.dt, dt_next=self.dt_next, e_kin=self.e_kin, e_int=self.e_int,
                    e_pot=self.e_pot, p=tuple(self.p), L=tuple(self.L), sweeps=self.sweeps,
                    n_unconverged=self.n_unconverged, n_capped=self.n_capped,
                    n_cfallback=self.n_cfallback, pairs_density=self.pairs_density,
                    pairs_force=self.pairs_force, device_flags=self.device_flags,
                    cand_density=self.cand_density, cand_force=self.cand_force,
                    groups_density=self.groups_density, groups_force=self.groups_force,
                    kernel_launches=self.kernel_launches, sweeps_total=self.sweeps_total,
                    n_expanded=self.n_expanded, particle_updates=self.particle_updates,
                    rung_counts=tuple(self.rung_counts))


class SphTuneReport(C.Structure):
    _fields_ = [("span_density", C.c_int32), ("span_forces", C.c_int32),
                ("steps_left", C.c_int32), ("n_cand", C.c_int32), ("cand", C.c_int32 * 4),
                ("timed", C.c_int32 * 4), ("ms_density", C.c_double * 4),
                ("ms_forces", C.c_double * 4), ("depth_density", C.c_int32),
                ("depth_forces", C.c_int32), ("n_depth", C.c_int32),
                ("depth_cand", C.c_int32 * 2), ("depth_timed", C.c_int32 * 2),
                ("reserved_", C.c_int32), ("ms_depth_density", C.c_double * 2),
                ("ms_depth_forces", C.c_double * 2)]


class SphPeakReport(C.Structure):
    _fields_ = [("tflops", C.c_double), ("ms", C.c_double), ("sm_mhz", C.c_double),
                ("flops", C.c_double), ("n_sm", C.c_int32), ("pad_", C.c_int32)]


EXPORTS = ("sph_init", "sph_neighbours", "sph_density", "sph_forces_strength",
           "sph_stress_update", "sph_step", "sph_step_host", "sph_prime", "sph_destroy",
           "sph_status_string", "sph_last_error", "sph_set_timing", "sph_phase_times",
           "sph_diagnostics_noalloc", "sph_init_batch", "sph_step_batch", "sph_batch_info",
           "sph_set_graph", "sph_autotune", "sph_tune_info",
           "sph_set_spans", "sph_mlp_create", "sph_mlp_destroy", "sph_mlp_last_error",
           "sph_mlp_set", "sph_mlp_get", "sph_mlp_fit_norm", "sph_mlp_forward",
           "sph_mlp_loss_grad", "sph_mlp_adam_step", "sph_mlp_train_epoch",
           "sph_set_learned_h", "sph_learn_samples", "sph_check_conversions",
           "sph_measure_fma_peak", "sph_inject_cuda_failure", "sph_learn_proposal",
           "sph_set_copy_chunks", "sph_set_stage_depths")
MLP_NPARAM, MLP_NNORM = 4673, 14
GUESS_PREVIOUS, GUESS_CONTINUITY, GUESS_NETWORK = 0, 1, 2
PHASES = ("neighbours", "pack", "density", "predict_eos", "forces", "kick")


def lib():
    """Load libsph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libsph.so not built: run `python -m paper_2603_19764_b300.build`")
        L = C.CDLL(LIB_PATH)
        st = C.c_int
        VP = C.c_void_p
        L.sph_init.restype = st
        L.sph_init.argtypes = [C.POINTER(VP), C.POINTER(SphParams), C.POINTER(SphMaterial),
                               C.c_int32, C.POINTER(SphState), C.c_int64, VP]
        for name in ("sph_neighbours", "sph_destroy"):
            getattr(L, name).restype = st
            getattr(L, name).argtypes = [VP]
        L.sph_density.restype = st
        L.sph_density.argtypes = [VP, _PI]
        L.sph_forces_strength.restype = st
        L.sph_forces_strength.argtypes = [VP]
        L.sph_stress_update.restype = st
        L.sph_stress_update.argtypes = [VP, C.c_double]
        L.sph_step.restype = st
        L.sph_step.argtypes = [VP, C.c_double, C.POINTER(SphStepInfo)]
        L.sph_step_host.restype = st
        L.sph_step_host.argtypes = [VP, C.POINTER(SphState), C.c_double, C.POINTER(SphStepInfo),
                                    _PL, _PL]
        L.sph_prime.restype = st
        L.sph_prime.argtypes = [VP, C.POINTER(SphStepInfo)]
        L.sph_set_timing.restype = st
        L.sph_set_timing.argtypes = [VP, C.c_int32]
        L.sph_phase_times.restype = st
        L.sph_phase_times.argtypes = [VP, _P, C.c_int32, _PI]
        L.sph_init_batch.restype = st
        L.sph_init_batch.argtypes = [C.POINTER(VP), C.POINTER(SphParams), C.POINTER(SphMaterial),
                                     C.c_int32, C.POINTER(SphState), C.c_int64, C.c_int32, _PL,
                                     VP]
        L.sph_step_batch.restype = st
        L.sph_step_batch.argtypes = [VP, _P, C.POINTER(SphStepInfo)]
        L.sph_batch_info.restype = st
        L.sph_batch_info.argtypes = [VP, C.POINTER(SphStepInfo), C.c_int32]
        _PF = C.POINTER(C.c_float)
        L.sph_mlp_create.restype = st
        L.sph_mlp_create.argtypes = [C.POINTER(VP), VP]
        L.sph_mlp_destroy.restype = st
        L.sph_mlp_destroy.argtypes = [VP]
        L.sph_mlp_last_error.restype = C.c_char_p
        L.sph_mlp_last_error.argtypes = [VP]
        L.sph_mlp_set.restype = st
        L.sph_mlp_set.argtypes = [VP, _PF, _PF]
        L.sph_mlp_get.restype = st
        L.sph_mlp_get.argtypes = [VP, _PF, _PF]
        L.sph_mlp_fit_norm.restype = st
        L.sph_mlp_fit_norm.argtypes = [VP, VP, VP, C.c_int64]
        L.sph_mlp_forward.restype = st
        L.sph_mlp_forward.argtypes = [VP, VP, C.c_int64, VP]
        L.sph_mlp_loss_grad.restype = st
        L.sph_mlp_loss_grad.argtypes = [VP, VP, VP, VP, C.c_int64, _PF, VP]
        L.sph_mlp_adam_step.restype = st
        L.sph_mlp_adam_step.argtypes = [VP, VP, C.c_float, C.c_float, C.c_float, C.c_float]
        L.sph_mlp_train_epoch.restype = st
        L.sph_mlp_train_epoch.argtypes = [VP, VP, VP, VP, C.c_int64, C.c_int32, C.c_float, _PF]
        L.sph_set_learned_h.restype = st
        L.sph_set_learned_h.argtypes = [VP, C.c_int32, C.c_int32, VP]
        L.sph_learn_samples.restype = st
        L.sph_learn_samples.argtypes = [VP, VP, VP]
        L.sph_check_conversions.restype = st
        L.sph_check_conversions.argtypes = [VP, C.c_int64, _PL, VP]
        L.sph_measure_fma_peak.restype = st
        L.sph_measure_fma_peak.argtypes = [C.c_int32, C.c_int32, C.POINTER(SphPeakReport), VP]
        L.sph_autotune.restype = st
        L.sph_autotune.argtypes = [VP, C.c_int32]
        L.sph_set_spans.restype = st
        L.sph_set_spans.argtypes = [VP, C.c_int32, C.c_int32]
        L.sph_tune_info.restype = st
        L.sph_tune_info.argtypes = [VP, C.POINTER(SphTuneReport)]
        L.sph_set_graph.restype = st
        L.sph_set_graph.argtypes = [VP, C.c_int32]
        L.sph_set_copy_chunks.restype = st
        L.sph_set_copy_chunks.argtypes = [VP, C.c_int32]
        L.sph_set_stage_depths.restype = st
        L.sph_set_stage_depths.argtypes = [VP, C.c_int32, C.c_int32]
        L.sph_diagnostics_noalloc.restype = st
        L.sph_diagnostics_noalloc.argtypes = [C.POINTER(SphState), C.c_int64, VP, VP]
        L.sph_learn_proposal.restype = st
        L.sph_learn_proposal.argtypes = [VP, VP]
        L.sph_inject_cuda_failure.restype = st
        L.sph_inject_cuda_failure.argtypes = [VP, C.c_int32]
        L.sph_status_string.restype = C.c_char_p
        L.sph_status_string.argtypes = [st]
        L.sph_last_error.restype = C.c_char_p
        L.sph_last_error.argtypes = [VP]
        _lib = L
    return _lib


# ------------------------------------------------------------- marshalling
def measure_fma_peak(precision: int, launches: int = 20) -> dict:
    """FMA throughput of the current device in FP32 (precision 1) or FP64 (0)."""
    r = SphPeakReport()
    rc = lib().sph_measure_fma_peak(int(precision), int(launches), C.byref(r), None)
    if rc != SPH_OK:
        raise SphError("sph_measure_fma_peak: %s" % lib().sph_status_string(rc).decode())
    return dict(tflops=r.tflops, ms=r.ms, sm_mhz=r.sm_mhz, flops=r.flops, n_sm=r.n_sm)


def make_material(d: dict) -> SphMaterial:
    m = SphMaterial()
    for name, _ in SphMaterial._fields_:
        setattr(m, name, d[name])
    return m


def make_params(d: dict, keep: list) -> SphParams:
    p = SphParams()
    for name, _ in SphParams._fields_:
        if name in ("g_table", "phi_table", "g_n"):
            continue
        if name in ("g_uniform", "g_center", "box_lo", "box_hi"):
            getattr(p, name)[:] = tuple(float(v) for v in d[name])
        elif name in ("gradient_form", "max_rung"):
            setattr(p, name, int(d.get(name, 0)))
        else:
            setattr(p, name, d[name])
    if d.get("g_table") is not None:
        g = np.ascontiguousarray(d["g_table"], np.float64)
        ph = np.ascontiguousarray(d["phi_table"], np.float64)
        keep += [g, ph]
        p.g_table = g.ctypes.data_as(_P)
        p.phi_table = ph.ctypes.data_as(_P)
        p.g_n = g.shape[0]
    return p


def state_from_ptrs(ptrs: dict) -> SphState:
    s = SphState()
    for f in F64_FIELDS:
        setattr(s, f, C.cast(C.c_void_p(ptrs[f]), _P))
    for f in I32_FIELDS:
        setattr(s, f, C.cast(C.c_void_p(ptrs[f]), _PI))
    s.id = C.cast(C.c_void_p(ptrs["id"]), _PL)
    return s


class Simulation:
    """Device-resident particle set driven through the C ABI.

    arrays: dict of numpy arrays (workloads.FIELDS_*); params / materials:
    dicts as built by workloads. The state lives in torch CUDA tensors.
    """

    def __init__(self, arrays: dict, materials: list, params: dict, device: str = "cuda:0",
                 stream=None, systems=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required: the SPH path has no CPU fallback")
        self.torch = torch
        self.device = torch.device(device)
        self.n = int(arrays["x"].shape[0])
        self.t = {}
        for f in F64_FIELDS:
            self.t[f] = torch.as_tensor(np.ascontiguousarray(arrays[f], np.float64)).to(self.device)
        for f in I32_FIELDS:
            self.t[f] = torch.as_tensor(np.ascontiguousarray(arrays[f], np.int32)).to(self.device)
        self.t["id"] = torch.as_tensor(np.ascontiguousarray(arrays["id"], np.int64)).to(self.device)
        self._keep = []
        self.params = make_params(params, self._keep)
        mats = (SphMaterial * len(materials))()
        for k, d in enumerate(materials):
            mats[k] = make_material(d)
        self._mats = mats
        self.state = state_from_ptrs({k: v.data_ptr() for k, v in self.t.items()})
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        torch.cuda.synchronize(self.device)
        self.ctx = C.c_void_p()
        if systems is None:
            self.nsys = 1
            rc = lib().sph_init(C.byref(self.ctx), C.byref(self.params), mats, len(materials),
                                C.byref(self.state), self.n, C.c_void_p(self.stream.cuda_stream))
        else:
            first = np.array([0] + [o + c for o, c in systems], dtype=np.int64)
            if any(int(first[k]) != int(o) for k, (o, _) in enumerate(systems)):
                raise ValueError("systems must be contiguous (offset, count) ranges from 0")
            self.nsys = len(systems)
            rc = lib().sph_init_batch(C.byref(self.ctx), C.byref(self.params), mats,
                                      len(materials), C.byref(self.state), self.n, self.nsys,
                                      first.ctypes.data_as(_PL),
                                      C.c_void_p(self.stream.cuda_stream))
        if rc != SPH_OK:
            raise SphError(rc, "sph_init")

    # -- calls ---------------------------------------------------------------
    def _check(self, rc, where, allow=()):
        if rc != SPH_OK and rc not in allow:
            detail = lib().sph_last_error(self.ctx).decode()
            raise SphError(rc, where, detail)
        return rc

    def neighbours(self):
        return self._check(lib().sph_neighbours(self.ctx), "sph_neighbours")

    def density(self, allow_noconv: bool = False) -> int:
        sw = C.c_int32()
        self._check(lib().sph_density(self.ctx, C.byref(sw)), "sph_density",
                    (SPH_E_NOCONV,) if allow_noconv else ())
        return sw.value

    def forces_strength(self):
        return self._check(lib().sph_forces_strength(self.ctx), "sph_forces_strength")

    def stress_update(self, dt: float):
        return self._check(lib().sph_stress_update(self.ctx, float(dt)), "sph_stress_update")

    def prime(self) -> dict:
        info = SphStepInfo()
        self._check(lib().sph_prime(self.ctx, C.byref(info)), "sph_prime")
        return info.as_dict()

    def step(self, dt: float = 0.0, allow=()) -> dict:
        info = SphStepInfo()
        rc = self._check(lib().sph_step(self.ctx, float(dt), C.byref(info)), "sph_step", allow)
        d = info.as_dict()
        d["status"] = rc
        return d

    def step_batch(self, dts) -> dict:
        d = np.ascontiguousarray(dts, np.float64)
        if d.shape != (self.nsys,):
            raise ValueError("step_batch needs one dt per system (%d)" % self.nsys)
        info = SphStepInfo()
        self._check(lib().sph_step_batch(self.ctx, d.ctypes.data_as(_P), C.byref(info)),
                    "sph_step_batch")
        return info.as_dict()

    def batch_info(self) -> list:
        arr = (SphStepInfo * self.nsys)()
        self._check(lib().sph_batch_info(self.ctx, arr, self.nsys), "sph_batch_info")
        return [a.as_dict() for a in arr]

    def autotune(self, rounds: int = 2):
        return self._check(lib().sph_autotune(self.ctx, int(rounds)), "sph_autotune")

    def set_learned_h(self, guess: int, record: bool = False, net: "Mlp | None" = None):
        self._net = net
        return self._check(lib().sph_set_learned_h(self.ctx, int(guess), 1 if record else 0,
                                                   net.ptr if net is not None else None),
                           "sph_set_learned_h")

    def learn_samples(self):
        """(X, y) of the last step as torch tensors indexed by particle id."""
        torch = self.torch
        X = torch.empty((self.n, 6), dtype=torch.float32, device=self.device)
        y = torch.empty(self.n, dtype=torch.float32, device=self.device)
        self._check(lib().sph_learn_samples(self.ctx, C.c_void_p(X.data_ptr()),
                                            C.c_void_p(y.data_ptr())), "sph_learn_samples")
        self.stream.synchronize()
        return X, y

    def learn_proposal(self):
        """Starting radii proposed for the next solve, in the current
        (sorted) particle order, as a torch tensor."""
        h = self.torch.zeros(self.n, dtype=self.torch.float64, device=self.device)
        self._check(lib().sph_learn_proposal(self.ctx, C.c_void_p(h.data_ptr())),
                    "sph_learn_proposal")
        self.stream.synchronize()
        return h

    def set_spans(self, span_density: int, span_forces: int):
        return self._check(lib().sph_set_spans(self.ctx, int(span_density), int(span_forces)),
                           "sph_set_spans")

    def tune_info(self) -> dict:
        r = SphTuneReport()
        self._check(lib().sph_tune_info(self.ctx, C.byref(r)), "sph_tune_info")
        k, q = r.n_cand, r.n_depth
        return {"span_density": r.span_density, "span_forces": r.span_forces,
                "steps_left": r.steps_left, "cand": list(r.cand[:k]), "timed": list(r.timed[:k]),
                "ms_density": list(r.ms_density[:k]), "ms_forces": list(r.ms_forces[:k]),
                "depth_density": r.depth_density, "depth_forces": r.depth_forces,
                "depth_cand": list(r.depth_cand[:q]), "depth_timed": list(r.depth_timed[:q]),
                "ms_depth_density": list(r.ms_depth_density[:q]),
                "ms_depth_forces": list(r.ms_depth_forces[:q])}

    def set_stage_depths(self, depth_density: int, depth_forces: int):
        return self._check(lib().sph_set_stage_depths(self.ctx, int(depth_density),
                                                      int(depth_forces)), "sph_set_stage_depths")

    def set_graph(self, on: bool = True):
        return self._check(lib().sph_set_graph(self.ctx, 1 if on else 0), "sph_set_graph")

    def set_copy_chunks(self, chunks: int):
        return self._check(lib().sph_set_copy_chunks(self.ctx, int(chunks)), "sph_set_copy_chunks")

    def step_host(self, host: "HostState", dt: float) -> dict:
        info = SphStepInfo()
        bi, bo = C.c_int64(), C.c_int64()
        self._check(lib().sph_step_host(self.ctx, C.byref(host.state), float(dt), C.byref(info),
                                        C.byref(bi), C.byref(bo)), "sph_step_host")
        d = info.as_dict()
        d.update(bytes_in=bi.value, bytes_out=bo.value)
        return d

    def inject_cuda_failure(self, after: int = 1):
        """Report the after-th checked CUDA call of this context as failed
        (host-side fault injection for tests of the error paths)."""
        return self._check(lib().sph_inject_cuda_failure(self.ctx, int(after)),
                           "sph_inject_cuda_failure")

    def set_timing(self, on: bool = True):
        return self._check(lib().sph_set_timing(self.ctx, 1 if on else 0), "sph_set_timing")

    def phase_times(self) -> dict:
        """Accumulated CUDA-event milliseconds per phase and the step count."""
        ms = (C.c_double * len(PHASES))()
        steps = C.c_int32()
        self._check(lib().sph_phase_times(self.ctx, ms, len(PHASES), C.byref(steps)),
                    "sph_phase_times")
        d = {name: ms[k] for k, name in enumerate(PHASES)}
        d["steps"] = steps.value
        return d

    # -- data ----------------------------------------------------------------
    def to_numpy(self, fields=None) -> dict:
        self.torch.cuda.synchronize(self.device)
        fields = fields or list(self.t)
        return {f: self.t[f].cpu().numpy() for f in fields}

    def by_id(self, fields=None) -> dict:
        """Arrays reordered by the caller's particle id (undoes the sort)."""
        a = self.to_numpy(list(fields or self.t) + ["id"])
        order = np.argsort(a["id"], kind="stable")
        return {k: v[order] for k, v in a.items()}

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lib().sph_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostState:
    """Pinned host copy of a particle set for sph_step_host."""

    def __init__(self, arrays: dict):
        import torch
        self.t = {}
        for f in F64_FIELDS:
            self.t[f] = torch.as_tensor(np.ascontiguousarray(arrays[f], np.float64)).pin_memory()
        for f in I32_FIELDS:
            self.t[f] = torch.as_tensor(np.ascontiguousarray(arrays[f], np.int32)).pin_memory()
        self.t["id"] = torch.as_tensor(np.ascontiguousarray(arrays["id"], np.int64)).pin_memory()
        self.state = state_from_ptrs({k: v.data_ptr() for k, v in self.t.items()})


class Mlp:
    """The smoothing-length network on one device (torch tensors in and out)."""

    def __init__(self, device: str = "cuda:0", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required: the network has no CPU fallback")
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ptr = C.c_void_p()
        rc = lib().sph_mlp_create(C.byref(self.ptr), C.c_void_p(self.stream.cuda_stream))
        if rc != SPH_OK:
            raise SphError(rc, "sph_mlp_create")

    def _check(self, rc, where):
        if rc != SPH_OK:
            raise SphError(rc, where, lib().sph_mlp_last_error(self.ptr).decode())
        return rc

    def _dev(self, a, dtype):
        t = self.torch
        x = a if isinstance(a, t.Tensor) else t.as_tensor(np.asarray(a))
        return x.to(device=self.device, dtype=dtype).contiguous()

    def set(self, theta, norm):
        th = np.ascontiguousarray(theta, np.float32)
        nm = np.ascontiguousarray(norm, np.float32)
        if th.shape != (MLP_NPARAM,) or nm.shape != (MLP_NNORM,):
            raise ValueError("theta needs %d values and norm %d" % (MLP_NPARAM, MLP_NNORM))
        _PF = C.POINTER(C.c_float)
        return self._check(lib().sph_mlp_set(self.ptr, th.ctypes.data_as(_PF),
                                             nm.ctypes.data_as(_PF)), "sph_mlp_set")

    def get(self):
        th = np.empty(MLP_NPARAM, np.float32)
        nm = np.empty(MLP_NNORM, np.float32)
        _PF = C.POINTER(C.c_float)
        self._check(lib().sph_mlp_get(self.ptr, th.ctypes.data_as(_PF), nm.ctypes.data_as(_PF)),
                    "sph_mlp_get")
        return th, nm

    def fit_norm(self, X, y):
        X = self._dev(X, self.torch.float32)
        y = self._dev(y, self.torch.float32)
        return self._check(lib().sph_mlp_fit_norm(self.ptr, C.c_void_p(X.data_ptr()),
                                                  C.c_void_p(y.data_ptr()), X.shape[0]),
                           "sph_mlp_fit_norm")

    def forward(self, X):
        X = self._dev(X, self.torch.float32)
        out = self.torch.empty(X.shape[0], dtype=self.torch.float32, device=self.device)
        self._check(lib().sph_mlp_forward(self.ptr, C.c_void_p(X.data_ptr()), X.shape[0],
                                          C.c_void_p(out.data_ptr())), "sph_mlp_forward")
        self.stream.synchronize()
        return out

    def loss_grad(self, X, y, idx=None):
        X = self._dev(X, self.torch.float32)
        y = self._dev(y, self.torch.float32)
        m = X.shape[0] if idx is None else len(idx)
        ix = None if idx is None else self._dev(idx, self.torch.int64)
        g = self.torch.empty(MLP_NPARAM, dtype=self.torch.float32, device=self.device)
        loss = C.c_float()
        self._check(lib().sph_mlp_loss_grad(self.ptr, C.c_void_p(X.data_ptr()),
                                            C.c_void_p(y.data_ptr()),
                                            C.c_void_p(ix.data_ptr()) if ix is not None else None,
                                            m, C.byref(loss), C.c_void_p(g.data_ptr())),
                    "sph_mlp_loss_grad")
        return loss.value, g

    def adam_step(self, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        g = self._dev(grad, self.torch.float32)
        return self._check(lib().sph_mlp_adam_step(self.ptr, C.c_void_p(g.data_ptr()), lr, beta1,
                                                   beta2, eps), "sph_mlp_adam_step")

    def train_epoch(self, X, y, perm, batch=4096, lr=1e-3) -> float:
        X = self._dev(X, self.torch.float32)
        y = self._dev(y, self.torch.float32)
        p = self._dev(perm, self.torch.int64)
        loss = C.c_float()
        self._check(lib().sph_mlp_train_epoch(self.ptr, C.c_void_p(X.data_ptr()),
                                              C.c_void_p(y.data_ptr()), C.c_void_p(p.data_ptr()),
                                              p.shape[0], int(batch), float(lr), C.byref(loss)),
                    "sph_mlp_train_epoch")
        return loss.value

    def close(self):
        if self.ptr:
            lib().sph_mlp_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
