"""FP64 CPU oracle of the SPH particle step with material strength.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package. The product path (the
CUDA library and its binding) never imports it; the two share no code.

The C source ``sphref.c`` follows the paper's equations (§2.1-§2.4) per
particle in FP64; this module compiles it with gcc (``build()``) and wraps it
with ctypes. Arrays are numpy float64 / int32 in structure-of-arrays layout,
ordered by original particle id.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sphref.c")
_HDR = os.path.join(_HERE, "sphref.h")
_LIB = os.path.join(_HERE, "libsphref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -ffp-contract=off -fopenmp)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared",
                               "-fPIC", "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class RefMaterial(C.Structure):
    _fields_ = [("eos", C.c_int32), ("rho0", C.c_double), ("c0", C.c_double),
                ("A", C.c_double), ("B", C.c_double), ("E0", C.c_double), ("a", C.c_double),
                ("b", C.c_double), ("alpha", C.c_double), ("beta", C.c_double),
                ("Eiv", C.c_double), ("Ecv", C.c_double), ("shear_G", C.c_double),
                ("Y0", C.c_double), ("mu_i", C.c_double), ("Ym", C.c_double),
                ("mu_d", C.c_double), ("thermal_softening", C.c_int32), ("xi", C.c_double),
                ("Tm", C.c_double), ("T0", C.c_double), ("cv", C.c_double),
                ("strength", C.c_int32), ("p_min", C.c_double)]


_P = C.POINTER(C.c_double)
_PI = C.POINTER(C.c_int32)
_PL = C.POINTER(C.c_int64)


class RefParams(C.Structure):
    _fields_ = [("n_ngb", C.c_int32), ("av_alpha", C.c_double), ("av_beta", C.c_double),
                ("av_eps", C.c_double), ("eta_c", C.c_double), ("eta_a", C.c_double),
                ("h_tol", C.c_double), ("max_sweeps", C.c_int32), ("h_cap_factor", C.c_double),
                ("jaumann", C.c_int32), ("yield_norm", C.c_int32),
                ("correction_tensor", C.c_int32), ("gravity", C.c_int32),
                ("g_uniform", C.c_double * 3), ("g_table", _P), ("phi_table", _P),
                ("g_n", C.c_int32), ("g_rmin", C.c_double), ("g_rmax", C.c_double),
                ("g_center", C.c_double * 3), ("g_gm", C.c_double), ("periodic", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("brute_force", C.c_int32), ("gradient_form", C.c_int32)]


_STATE_F = ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h", "sxx", "syy", "sxy", "sxz", "syz",
            "rho", "omega", "pres", "cs", "yld", "ax", "ay", "az", "dudt", "dsxx", "dsyy",
            "dsxy", "dsxz", "dsyz", "eps_ii", "vsig")
_STATE_I = ("nngb", "mat", "flags")


class RefState(C.Structure):
    _fields_ = [(f, _P) for f in _STATE_F] + [(f, _PI) for f in _STATE_I]


class RefInfo(C.Structure):
    _fields_ = [("dt_next", C.c_double), ("e_kin", C.c_double), ("e_int", C.c_double),
                ("e_pot", C.c_double), ("p", C.c_double * 3), ("L", C.c_double * 3),
                ("max_sweeps", C.c_int32), ("n_unconverged", C.c_int32),
                ("n_capped", C.c_int32), ("n_cfallback", C.c_int32)]

    def as_dict(self) -> dict:
        return dict(dt_next=self.dt_next, e_kin=self.e_kin, e_int=self.e_int, e_pot=self.e_pot,
                    p=tuple(self.p), L=tuple(self.L), max_sweeps=self.max_sweeps,
                    n_unconverged=self.n_unconverged, n_capped=self.n_capped,
                    n_cfallback=self.n_cfallback)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d = C.c_double
        L.ref_W.restype = L.ref_dWdr.restype = L.ref_dWdH.restype = d
        L.ref_W.argtypes = L.ref_dWdr.argtypes = L.ref_dWdH.argtypes = [d, d]
        L.ref_eos.argtypes = [C.POINTER(RefMaterial), d, d, _P, _P]
        L.ref_yield.restype = d
        L.ref_yield.argtypes = [C.POINTER(RefMaterial), d, d]
        L.ref_radial_return.restype = d
        L.ref_radial_return.argtypes = [_P, d, C.c_int32]
        L.ref_stress_rate.argtypes = [_P, _P, d, C.c_int32, _P]
        L.ref_inv3.restype = d
        L.ref_inv3.argtypes = [_P, _P]
        L.ref_gravity.argtypes = [C.POINTER(RefParams), d, d, d, _P]
        L.ref_potential.restype = d
        L.ref_potential.argtypes = [C.POINTER(RefParams), d, d, d]
        L.ref_neighbours.restype = C.c_int64
        L.ref_neighbours.argtypes = [C.POINTER(RefParams), C.c_int64, _P, _P, _P, _P,
                                     C.c_int64, C.c_int32, _PL, C.c_int64]
        L.ref_count_neighbours.argtypes = [C.POINTER(RefParams), C.c_int64,
                                           C.POINTER(RefState), C.c_int64, _PL, _PI]
        L.ref_density_given_h.argtypes = [C.POINTER(RefParams), C.c_int64,
                                          C.POINTER(RefState), C.c_int64, _PL, _P, _P, _PI]
        L.ref_density_solve.restype = C.c_int32
        L.ref_density_solve.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial),
                                        C.c_int64, C.POINTER(RefState), _PI, _PI]
        L.ref_eos_yield.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial), C.c_int64,
                                    C.POINTER(RefState), _P, _P, _P, _P, _P, _P]
        L.ref_forces.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial), C.c_int64,
                                 C.POINTER(RefState), _P, _P, _P, _P, _P, _P, _P, _P,
                                 C.c_int64, _PL, _P, _P, _PI]
        L.ref_step_rungs.restype = C.c_int32
        L.ref_step_rungs.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial), C.c_int64,
                                     C.POINTER(RefState), C.c_double, C.c_int32, _PI, _PL,
                                     C.POINTER(RefInfo)]
        L.ref_step.restype = C.c_int32
        L.ref_step.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial), C.c_int64,
                               C.POINTER(RefState), d, C.POINTER(RefInfo)]
        L.ref_derivatives.restype = C.c_int32
        L.ref_derivatives.argtypes = [C.POINTER(RefParams), C.POINTER(RefMaterial), C.c_int64,
                                      C.POINTER(RefState), C.POINTER(RefInfo)]
        L.ref_diagnostics.argtypes = [C.POINTER(RefParams), C.c_int64, C.POINTER(RefState),
                                      C.POINTER(RefInfo)]
        L.ref_threads.restype = C.c_int32
        L.ref_set_threads.restype = C.c_int32
        L.ref_set_threads.argtypes = [C.c_int32]
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# Marshalling
# --------------------------------------------------------------------------
def _dp(a):
    return a.ctypes.data_as(_P) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_PI) if a is not None else None


def _lp(a):
    return a.ctypes.data_as(_PL) if a is not None else None


def material(d: dict) -> RefMaterial:
    m = RefMaterial()
    for name, _ in RefMaterial._fields_:
        setattr(m, name, d[name])
    return m


def materials(lst) -> C.Array:
    arr = (RefMaterial * len(lst))()
    for k, d in enumerate(lst):
        arr[k] = material(d)
    return arr


class Params:
    """RefParams plus the numpy buffers its pointers refer to."""

    def __init__(self, d: dict, brute_force: bool = False):
        self.p = RefParams()
        self._keep = []
        for name, _ in RefParams._fields_:
            if name in ("g_table", "phi_table"):
                continue
            if name == "brute_force":
                self.p.brute_force = 1 if brute_force else 0
            elif name == "gradient_form":
                self.p.gradient_form = int(d.get(name, 0))
            elif name == "g_n":
                continue
            elif name in ("g_uniform", "g_center", "box_lo", "box_hi"):
                getattr(self.p, name)[:] = tuple(float(v) for v in d[name])
            else:
                setattr(self.p, name, d[name])
        g = d.get("g_table")
        if g is not None:
            g = np.ascontiguousarray(g, np.float64)
            ph = np.ascontiguousarray(d["phi_table"], np.float64)
            self._keep += [g, ph]
            self.p.g_table, self.p.phi_table, self.p.g_n = _dp(g), _dp(ph), g.shape[0]

    @property
    def ref(self):
        return C.byref(self.p)


class State:
    """Owns contiguous copies of a particle set and the RefState view."""

    def __init__(self, arrays: dict):
        n = arrays["x"].shape[0]
        self.n = n
        self.a = {}
        for f in _STATE_F:
            src = arrays.get(f)
            self.a[f] = (np.ascontiguousarray(src, np.float64).copy() if src is not None
                         else np.zeros(n, np.float64))
        for f in _STATE_I:
            self.a[f] = np.ascontiguousarray(arrays[f], np.int32).copy()
        self.s = RefState()
        for f in _STATE_F:
            setattr(self.s, f, _dp(self.a[f]))
        for f in _STATE_I:
            setattr(self.s, f, _ip(self.a[f]))

    def __getitem__(self, k):
        return self.a[k]

    @property
    def ref(self):
        return C.byref(self.s)


# --------------------------------------------------------------------------
# Point functions (vectorised over numpy inputs by plain loops)
# --------------------------------------------------------------------------
def W(r, H):
    return np.vectorize(lambda a, b: lib().ref_W(float(a), float(b)))(r, H)


def dWdr(r, H):
    return np.vectorize(lambda a, b: lib().ref_dWdr(float(a), float(b)))(r, H)


def dWdH(r, H):
    return np.vectorize(lambda a, b: lib().ref_dWdH(float(a), float(b)))(r, H)


def eos(mat: dict, rho, u):
    m = material(mat)
    P, c = C.c_double(), C.c_double()

    def one(r, e):
        lib().ref_eos(C.byref(m), float(r), float(e), C.byref(P), C.byref(c))
        return P.value, c.value

    out = np.vectorize(one, otypes=[np.float64, np.float64])(rho, u)
    return out[0], out[1]


def yield_strength(mat: dict, P, u):
    m = material(mat)
    return np.vectorize(lambda a, b: lib().ref_yield(C.byref(m), float(a), float(b)))(P, u)


def radial_return(S, Y, yield_norm: int = 0):
    s = np.ascontiguousarray(S, np.float64).copy()
    f = lib().ref_radial_return(_dp(s), float(Y), int(yield_norm))
    return s, f


def stress_rate(S, G, shear_G: float, jaumann: int = 0):
    s = np.ascontiguousarray(S, np.float64)
    g = np.ascontiguousarray(np.asarray(G, np.float64).reshape(9))
    out = np.zeros(5)
    lib().ref_stress_rate(_dp(s), _dp(g), float(shear_G), int(jaumann), _dp(out))
    return out


def inv3(A):
    a = np.ascontiguousarray(np.asarray(A, np.float64).reshape(9))
    out = np.zeros(9)
    det = lib().ref_inv3(_dp(a), _dp(out))
    return out.reshape(3, 3), det


def gravity(params: dict, x, y, z):
    P = Params(params)
    g = np.zeros(3)
    lib().ref_gravity(P.ref, float(x), float(y), float(z), _dp(g))
    return g


def potential(params: dict, x, y, z):
    P = Params(params)
    return lib().ref_potential(P.ref, float(x), float(y), float(z))


def threads() -> int:
    return int(lib().ref_threads())


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's parallel loops (results do not depend
    on it); returns the count in effect."""
    return int(lib().ref_set_threads(int(n)))


# --------------------------------------------------------------------------
# Particle-set functions
# --------------------------------------------------------------------------
def neighbours(params: dict, arrays: dict, i: int, mode: int = 0, brute_force: bool = False):
    P = Params(params, brute_force)
    x, y, z, h = (np.ascontiguousarray(arrays[k], np.float64) for k in ("x", "y", "z", "h"))
    n = x.shape[0]
    out = np.zeros(n, np.int64)
    cnt = lib().ref_neighbours(P.ref, n, _dp(x), _dp(y), _dp(z), _dp(h), int(i), int(mode),
                               _lp(out), n)
    return out[:cnt].copy()


def count_neighbours(params: dict, arrays: dict, idx=None, brute_force: bool = False):
    P = Params(params, brute_force)
    st = State(arrays)
    sel = None if idx is None else np.ascontiguousarray(idx, np.int64)
    nl = st.n if sel is None else sel.shape[0]
    out = np.zeros(nl, np.int32)
    lib().ref_count_neighbours(P.ref, st.n, st.ref, nl, _lp(sel), _ip(out))
    return out


def density_given_h(params: dict, arrays: dict, idx=None, brute_force: bool = False):
    P = Params(params, brute_force)
    st = State(arrays)
    sel = None if idx is None else np.ascontiguousarray(idx, np.int64)
    nl = st.n if sel is None else sel.shape[0]
    rho, om, cnt = np.zeros(nl), np.zeros(nl), np.zeros(nl, np.int32)
    lib().ref_density_given_h(P.ref, st.n, st.ref, nl, _lp(sel), _dp(rho), _dp(om), _ip(cnt))
    return rho, om, cnt


def density_solve(params: dict, mats: list, arrays: dict, brute_force: bool = False):
    """Returns (state dict with h, rho, omega, nngb updated, info dict)."""
    P = Params(params, brute_force)
    M = materials(mats)
    st = State(arrays)
    unc, cap = C.c_int32(), C.c_int32()
    sw = lib().ref_density_solve(P.ref, M, st.n, st.ref, C.byref(unc), C.byref(cap))
    return st.a, dict(max_sweeps=sw, n_unconverged=unc.value, n_capped=cap.value)


def eos_yield(params: dict, mats: list, arrays: dict, u=None, S=None):
    """EOS + yield + radial return; returns (state dict, S tuple after return)."""
    P = Params(params)
    M = materials(mats)
    st = State(arrays)
    ue = np.ascontiguousarray(st["u"] if u is None else u, np.float64)
    Ss = [np.ascontiguousarray(st[k] if S is None else S[q], np.float64).copy()
          for q, k in enumerate(("sxx", "syy", "sxy", "sxz", "syz"))]
    lib().ref_eos_yield(P.ref, M, st.n, st.ref, _dp(ue), *[_dp(s) for s in Ss])
    return st.a, tuple(Ss)


def forces(params: dict, mats: list, arrays: dict, v=None, S=None, idx=None,
           want_tensors: bool = False, brute_force: bool = False):
    """Pair sums + finalize with the given evaluation velocities and stress.

    arrays must carry rho, omega, pres, cs, nngb (from density_solve and
    eos_yield). Returns (state dict with ax..dsyz, vsig; info dict). With
    want_tensors, info holds 'G' and 'C' (n_sel x 3 x 3).
    """
    P = Params(params, brute_force)
    M = materials(mats)
    st = State(arrays)
    vv = [np.ascontiguousarray(st[k] if v is None else v[q], np.float64)
          for q, k in enumerate(("vx", "vy", "vz"))]
    Ss = [np.ascontiguousarray(st[k] if S is None else S[q], np.float64)
          for q, k in enumerate(("sxx", "syy", "sxy", "sxz", "syz"))]
    sel = None if idx is None else np.ascontiguousarray(idx, np.int64)
    nl = st.n if sel is None else sel.shape[0]
    G = np.zeros((nl, 3, 3)) if want_tensors else None
    Cm = np.zeros((nl, 3, 3)) if want_tensors else None
    fb = C.c_int32()
    lib().ref_forces(P.ref, M, st.n, st.ref, *[_dp(a) for a in vv], *[_dp(s) for s in Ss],
                     nl, _lp(sel), _dp(G), _dp(Cm), C.byref(fb))
    info = dict(n_cfallback=fb.value)
    if want_tensors:
        info.update(G=G, C=Cm)
    return st.a, info


def derivatives(params: dict, mats: list, arrays: dict, brute_force: bool = False):
    P = Params(params, brute_force)
    M = materials(mats)
    st = State(arrays)
    info = RefInfo()
    rc = lib().ref_derivatives(P.ref, M, st.n, st.ref, C.byref(info))
    d = info.as_dict()
    d["status"] = rc
    return st.a, d


def step(params: dict, mats: list, arrays: dict, dt: float, nsteps: int = 1,
         brute_force: bool = False, callback=None):
    """Advance nsteps steps of length dt; returns (state dict, list of infos)."""
    P = Params(params, brute_force)
    M = materials(mats)
    st = State(arrays)
    infos = []
    for k in range(nsteps):
        info = RefInfo()
        rc = lib().ref_step(P.ref, M, st.n, st.ref, float(dt), C.byref(info))
        d = info.as_dict()
        d["status"] = rc
        infos.append(d)
        if callback is not None:
            callback(k, st.a, d)
    return st.a, infos


def step_rungs(params: dict, mats: list, arrays: dict, dt: float, max_rung: int,
               nsteps: int = 1):
    """Advance nsteps big steps of length dt with hierarchical individual
    steps on 2^max_rung substeps (ref_step_rungs). Returns (state dict,
    list of infos, rungs at the end, particle updates per big step)."""
    P = Params(params)
    M = materials(mats)
    st = State(arrays)
    rung = np.zeros(st.n, np.int32)
    infos, updates = [], []
    for _ in range(nsteps):
        info = RefInfo()
        na = C.c_int64(0)
        rc = lib().ref_step_rungs(P.ref, M, st.n, st.ref, float(dt), int(max_rung), _ip(rung),
                                  C.byref(na), C.byref(info))
        if rc == 4:
            raise ValueError("ref_step_rungs: max_rung outside 0..15 or no vsig in the state")
        d = info.as_dict()
        d["status"] = rc
        infos.append(d)
        updates.append(int(na.value))
    return st.a, infos, rung, updates


def diagnostics(params: dict, arrays: dict) -> dict:
    P = Params(params)
    st = State(arrays)
    info = RefInfo()
    lib().ref_diagnostics(P.ref, st.n, st.ref, C.byref(info))
    return info.as_dict()
