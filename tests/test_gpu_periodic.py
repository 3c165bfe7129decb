"""Periodic boxes on the CUDA path against the FP64 oracle, through the C ABI.

In a periodic box [box_lo, box_hi) drifted positions wrap back into the box
and every pair takes the minimum image (the oracle's definition: x_i - x_j
shifted by one box length where it exceeds half the box). Checked here:
* a perfect 64 x 8 x 8 lattice carrying a standing wave, and a jittered box
  whose particles cross the faces within the first steps: counts bit-exact
  given the GPU's H, density and derivatives at the parity tolerances, over
  several full steps;
* the elastic-wave check of the method: a longitudinal standing wave in the
  64 x 8 x 8 box stepped by sph_step travels at sqrt((K + 4/3 Gamma) / rho)
  within 1 %, with a constant shear modulus and with that of Eq. 30;
* a box not wider than twice the search radius is reported
  (SPH_E_CAPACITY), and sph_init refuses what the periodic form does not
  support."""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import check_density_solve, cloud

pytestmark = pytest.mark.gpu

RHO_TOL = {0: 1e-6, 1: 1e-5}
DERIV_TOL = {0: 1e-9, 1: 1e-4}
DERIVS = ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _p(params, precision):
    return dict(params, precision=precision, h_tol=1e-10 if precision == 0 else 1e-6)


def _maxnorm_err(a, b):
    scale = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)


def _wrapped_diff(a, b, box):
    d = a - b
    return np.abs(d - box * np.round(d / box))


def _jittered_box(n_side=16, seed=81):
    """A jittered lattice filling a periodic box, with random velocities and
    stresses and a bulk drift that carries particles through the faces."""
    mat = wl.elastic_material()
    a = cloud(n_side ** 3, seed=seed, jitter=0.3, spacing=1.0, mat=mat, vsig=2.0, ssig=2e4,
              shape="cube")
    L = float(n_side)
    for f in ("x", "y", "z"):
        a[f] = np.mod(a[f] + 0.5, L)          # inside [0, L)
    a["vx"] += 120.0
    a["vy"] -= 60.0
    a["u"][:] = 0.0
    p = dict(wl.default_params(0), periodic=1, box_lo=(0.0, 0.0, 0.0), box_hi=(L, L, L))
    return a, [mat], p


@pytest.mark.parametrize("precision", [0, 1])
def test_wave_lattice_prime(precision):
    """Perfect lattice with the standing wave's velocity: the wave's
    compression gives du/dt and the diagonal stress rates; pressure is
    uniform and there is no viscosity or shear, so the accelerations and the
    off-diagonal rates vanish up to round-off of the pressure-force scale."""
    w = wl.periodic_wave_box(64, 8, 8, amp=1e-3)
    mats = [dict(w.materials[0], rho0=990.0)]
    p = _p(w.params, precision)
    sim = sph.Simulation(w.arrays, mats, p)
    info = sim.prime()
    g = sim.by_id()
    sim.close()
    ref, rinfo = oracle.derivatives(p, mats, w.arrays)
    check_density_solve(g, ref, p, mats, w.arrays, RHO_TOL[precision])
    for f in ("dudt", "dsxx", "dsyy"):
        e = _maxnorm_err(g[f], ref[f])
        assert e < DERIV_TOL[precision], (f, e)
    a_scale = float(np.mean(ref["pres"]) / (np.mean(ref["rho"]) * np.mean(ref["h"])))
    s_scale = float(np.max(np.abs(ref["dsxx"])))
    zero_tol = 1e-12 if precision == 0 else 1e-4
    for f, sc in (("ax", a_scale), ("ay", a_scale), ("az", a_scale), ("dsxy", s_scale),
                  ("dsxz", s_scale), ("dsyz", s_scale)):
        assert np.max(np.abs(g[f])) < zero_tol * sc, (f, np.max(np.abs(g[f])), sc)
        assert np.max(np.abs(ref[f])) < 1e-12 * sc, f
    assert info["dt_next"] == pytest.approx(rinfo["dt_next"], rel=1e-6 if precision == 0 else 1e-4)
    # every particle of a perfect periodic lattice is alike
    assert np.ptp(g["nngb"]) == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_jittered_box_steps_through_the_faces(precision):
    a, mats, p0 = _jittered_box()
    p = _p(p0, precision)
    L = p["box_hi"][0]
    ref, rinfo = oracle.derivatives(p, mats, a)
    dt = 0.8 * rinfo["dt_next"]
    sim = sph.Simulation(a, mats, p)
    sim.prime()
    g0 = sim.by_id()
    for f in DERIVS:
        assert _maxnorm_err(g0[f], ref[f]) < DERIV_TOL[precision], f
    x0, y0 = a["x"].copy(), a["y"].copy()
    for k in range(6):
        ref, _ = oracle.step(p, mats, ref, dt)
        info = sim.step(dt)
        assert info["status"] == sph.SPH_OK
    g = sim.by_id()
    sim.close()
    # particles did cross the faces, and both sides wrapped them alike
    crossed = np.sum((np.abs(g["x"] - x0) > 0.5 * L) | (np.abs(g["y"] - y0) > 0.5 * L))
    assert crossed > 50
    for f in ("x", "y", "z"):
        assert np.all((g[f] >= 0.0) & (g[f] < L))
        d = _wrapped_diff(g[f], ref[f], L)
        assert d.max() < (1e-10 if precision == 0 else 1e-4), (f, d.max())
    # counts given the GPU's own radius, then the usual parity
    rho, _, cnt = oracle.density_given_h(p, dict(ref, x=g["x"], y=g["y"], z=g["z"], h=g["h"]))
    assert np.array_equal(cnt, g["nngb"])
    assert np.max(np.abs(g["rho"] / ref["rho"] - 1)) < RHO_TOL[precision]
    for f in DERIVS:
        e = _maxnorm_err(g[f], ref[f])
        assert e < DERIV_TOL[precision], (f, e)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("modulus", ["constant", "eq30"])
def test_elastic_wave_speed_on_the_gpu(precision, modulus):
    w = wl.periodic_wave_box(64, 8, 8, amp=1e-3)
    mat = dict(w.materials[0], rho0=990.0)
    if modulus == "eq30":
        mat["shear_G"] = -1.0
    p = _p(w.params, precision)
    sim = sph.Simulation(w.arrays, [mat], p)
    info = sim.prime()
    rho = float(np.mean(sim.to_numpy(["rho"])["rho"]))
    gam = 0.6 * rho * mat["c0"] ** 2 if modulus == "eq30" else mat["shear_G"]
    c_l = math.sqrt(mat["c0"] ** 2 + 4.0 / 3.0 * gam / rho)
    lx = p["box_hi"][0]
    k = 2 * math.pi / lx
    s = np.sin(k * w.arrays["x"])
    dt = 0.2 * float(w.arrays["h"][0]) / c_l
    nsteps = int(1.3 * lx / c_l / dt)
    amps = []
    for _ in range(nsteps):
        r = sim.step(dt)
        assert r["status"] == sph.SPH_OK
        vx = sim.by_id(["vx"])["vx"]
        amps.append((vx * s).sum() / (s * s).sum())
    sim.close()
    t = (np.arange(nsteps) + 0.5) * dt
    amps = np.array(amps)
    f = lambda tt, A, om, ph: A * np.cos(om * tt + ph)
    (A, om, ph), _ = optimize.curve_fit(f, t, amps, p0=[amps[0], c_l * k, 0.0])
    assert abs(om / k / c_l - 1) < 0.01, (om / k, c_l)


def test_narrow_box_reports_capacity():
    w = wl.periodic_wave_box(4, 4, 4, amp=1e-3)      # H ~ 2.5 in a box of 4
    sim = sph.Simulation(w.arrays, w.materials, w.params)
    with pytest.raises(sph.SphError) as e:
        sim.prime()
    assert e.value.status == sph.SPH_E_CAPACITY
    sim.close()


def test_periodic_init_refusals():
    w = wl.periodic_wave_box(16, 8, 8, amp=1e-3)
    bad = [dict(w.params, max_rung=2),
           dict(w.params, box_hi=(16.0, 8.0, 0.0)),
           dict(w.params, gravity=2)]
    for p in bad:
        with pytest.raises(sph.SphError) as e:
            sph.Simulation(w.arrays, w.materials, p)
        assert e.value.status == sph.SPH_E_ARG
    out = {k: v.copy() for k, v in w.arrays.items()}
    out["x"][5] = 16.0                                # on box_hi: outside [lo, hi)
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(out, w.materials, w.params)
    assert e.value.status == sph.SPH_E_ARG
    with pytest.raises(sph.SphError) as e:
        sph.Simulation(w.arrays, w.materials, w.params, systems=[(0, 512), (512, 512)])
    assert e.value.status == sph.SPH_E_ARG
