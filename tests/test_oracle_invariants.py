"""Pins of two oracle quantities that no other pin fixes by value.

* The strain-rate invariant integrated at the closing kick (§2.4, Eq. 43):
  eps_ii accumulates dt * 1/2 edot:edot with edot = sym(G) (Eq. 24). A
  body with no forces at all (no pressure, no viscosity, no strength, no
  gravity) keeps every particle's velocity, so a velocity field v = A x0 + b
  stays linear in the drifted positions x_k = x0 + k dt v: v = G_k x + const
  with G_k = A (I + k dt A)^-1. The correction tensor makes the SPH gradient
  of a linear field exact (Eq. 20-22), so after n steps every particle holds
  sum_k dt 1/2 |sym(G_k)|^2 to round-off. A dropped 1/2, G in place of
  sym(G), or a gradient taken at the undrifted positions each fail it.
* The shear modulus of Eq. 30 (Poisson ratio 0.25): Gamma = 3 (1 - 2 nu) /
  (2 (1 + nu)) K with K = rho c^2. Under a pure-shear linear field with
  S = 0 the stress rate is 2 Gamma dev(edot) exactly (Eq. 13 with no
  rotation term acting on S = 0), so every particle's dS/dt over 2 edot is
  its Gamma; and a longitudinal wave in a periodic box then travels at
  sqrt((K + 4/3 Gamma) / rho) = c0 sqrt(1 + 4/3 * 0.6).
* The global sums of the step report (kinetic, internal and potential
  energy, momentum, angular momentum L = sum m r x v of Eq. 46) against
  rigid-body mechanics (inertia tensor about the centre of mass).
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import cloud

NU = 0.25
EQ30 = 3.0 * (1.0 - 2.0 * NU) / (2.0 * (1.0 + NU))


def _forceless_material():
    """Linear EOS with c0 = 0 (P = 0 at any density), no strength."""
    m = wl.elastic_material()
    m.update(c0=0.0, A=0.0, strength=0)
    return m


@pytest.mark.parametrize("nsteps", [1, 4])
def test_strain_invariant_accumulates_half_edot_squared(nsteps):
    mat = _forceless_material()
    a = cloud(1500, seed=31, jitter=0.25, spacing=1.0, mat=mat)
    a["u"][:] = 0.0
    A = np.array([[0.30, -0.45, 0.20], [0.15, -0.10, 0.35], [-0.25, 0.40, 0.05]])
    b = np.array([0.7, -0.2, 0.4])
    x0 = np.stack([a["x"], a["y"], a["z"]], 1)
    v = x0 @ A.T + b
    a["vx"], a["vy"], a["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    a["eps_ii"][:] = 0.0
    p = dict(wl.default_params(0), av_alpha=0.0, av_beta=0.0)
    st, info = oracle.derivatives(p, [mat], a)
    assert info["n_cfallback"] == 0
    for f in ("ax", "ay", "az", "dudt"):
        assert np.all(st[f] == 0.0)          # no force of any kind
    dt = 0.05
    st, infos = oracle.step(p, [mat], st, dt, nsteps=nsteps)
    assert all(i["n_cfallback"] == 0 for i in infos)
    # velocities unchanged, positions drifted linearly
    assert np.array_equal(st["vx"], v[:, 0])
    want = 0.0
    for k in range(1, nsteps + 1):
        G = A @ np.linalg.inv(np.eye(3) + k * dt * A)
        e = 0.5 * (G + G.T)
        want += dt * 0.5 * float((e * e).sum())
    assert want > 0
    assert np.max(np.abs(st["eps_ii"] / want - 1.0)) < 1e-9, np.max(np.abs(st["eps_ii"] / want - 1))
    # the plausible mistakes are far outside that tolerance
    Gs = [A @ np.linalg.inv(np.eye(3) + k * dt * A) for k in range(1, nsteps + 1)]
    e0 = 0.5 * (A + A.T)
    wrong = {"no 1/2": 2.0 * want,
             "G for sym(G)": sum(dt * 0.5 * float((G * G).sum()) for G in Gs),
             "undrifted positions": nsteps * dt * 0.5 * float((e0 * e0).sum())}
    for name, val in wrong.items():
        assert abs(val / want - 1.0) > 1e-3, name


@pytest.mark.parametrize("eos", ["linear", "tillotson"])
def test_eq30_shear_modulus_from_bulk_modulus(eos):
    if eos == "linear":
        mat = wl.elastic_material()
        mat.update(shear_G=-1.0)
    else:
        mat = dict(wl.basalt_material(), shear_G=-1.0, Y0=1e30, mu_i=0.0, Ym=math.inf,
                   mu_d=1e30, thermal_softening=0)
    a = cloud(1200, seed=33, jitter=0.25, spacing=1.0 if eos == "linear" else 100.0, mat=mat)
    if eos == "linear":
        a["u"][:] = 0.0
    for f in ("sxx", "syy", "sxy", "sxz", "syz"):
        a[f][:] = 0.0
    p = dict(wl.default_params(0), av_alpha=0.0, av_beta=0.0)
    st, _ = oracle.density_solve(p, [mat], a)
    st, S = oracle.eos_yield(p, [mat], st)
    # pure shear: symmetric and traceless, no rotation
    E = np.array([[0.2, 0.5, -0.3], [0.5, -0.6, 0.1], [-0.3, 0.1, 0.4]])
    x = np.stack([st["x"], st["y"], st["z"]], 1)
    v = x @ E.T
    out, info = oracle.forces(p, [mat], st, v=(v[:, 0], v[:, 1], v[:, 2]), S=S,
                              want_tensors=True)
    assert info["n_cfallback"] == 0
    assert np.allclose(info["G"], E[None], rtol=0, atol=1e-9)
    gamma = EQ30 * st["rho"] * st["cs"] ** 2
    assert EQ30 == pytest.approx(0.6, rel=1e-15)
    for f, (r, c) in (("dsxx", (0, 0)), ("dsyy", (1, 1)), ("dsxy", (0, 1)),
                      ("dsxz", (0, 2)), ("dsyz", (1, 2))):
        got = out[f] / (2.0 * E[r, c])
        assert np.max(np.abs(got / gamma - 1.0)) < 1e-8, (f, np.max(np.abs(got / gamma - 1.0)))
    if eos == "linear":
        # c = c0 for the linear EOS: Gamma = 0.6 rho c0^2 per particle
        assert np.allclose(gamma, 0.6 * st["rho"] * mat["c0"] ** 2, rtol=1e-14, atol=0)
    # a constant modulus is taken as given
    mat_c = dict(mat, shear_G=7.5e6)
    out_c, _ = oracle.forces(p, [mat_c], st, v=(v[:, 0], v[:, 1], v[:, 2]), S=S)
    assert np.allclose(out_c["dsxy"] / (2.0 * E[0, 1]), 7.5e6, rtol=1e-8, atol=0)


def test_elastic_wave_speed_with_eq30_modulus():
    """Periodic 64 x 8 x 8 lattice, Gamma from Eq. 30: c_L = c0 sqrt(1.8)."""
    w = wl.periodic_wave_box(64, 8, 8, amp=1e-3)
    mat = dict(w.materials[0], rho0=990.0, shear_G=-1.0)
    a = w.arrays
    st, _ = oracle.derivatives(w.params, [mat], a)
    c_l = mat["c0"] * math.sqrt(1.0 + 4.0 / 3.0 * EQ30)
    lx = w.params["box_hi"][0]
    k = 2 * math.pi / lx
    s = np.sin(k * a["x"])
    dt = 0.2 * float(a["h"][0]) / c_l
    nsteps = int(1.3 * lx / c_l / dt)
    amps = []

    def cb(i, arr, inf):
        amps.append((arr["vx"] * s).sum() / (s * s).sum())

    oracle.step(w.params, [mat], st, dt, nsteps=nsteps, callback=cb)
    t = (np.arange(nsteps) + 0.5) * dt
    amps = np.array(amps)
    f = lambda tt, A, om, ph: A * np.cos(om * tt + ph)
    (A, om, ph), _ = optimize.curve_fit(f, t, amps, p0=[amps[0], c_l * k, 0.0])
    assert abs(om / k / c_l - 1) < 0.01, om / k / c_l
    # the constant modulus of the same box would give a clearly different speed
    c_const = math.sqrt(mat["c0"] ** 2 + 4.0 / 3.0 * 3.0e6 / 1000.0)
    assert abs(c_const / c_l - 1) > 0.05


def test_global_sums_of_a_rigid_motion():
    """The diagnostics of the step (energies, momentum and angular momentum
    of Eq. 46) against rigid-body mechanics: for v = v0 + w x (r - c) with c
    the centre of mass, p = M v0, L = M c x v0 + I_c w (I_c the inertia
    tensor about c), E_kin = 1/2 M |v0|^2 + 1/2 w.I_c w, E_int = sum m u and,
    in a uniform field g, E_pot = -M g.c."""
    rng = np.random.default_rng(91)
    n = 500
    a = wl._empty_arrays(n)
    m = rng.uniform(0.5, 2.0, n)
    r = rng.normal(size=(n, 3)) * np.array([3.0, 1.0, 2.0])
    c = np.array([10.0, -4.0, 7.0])
    r = r - (m[:, None] * r).sum(0) / m.sum() + c          # centre of mass at c
    v0 = np.array([1.5, -0.5, 2.0])
    w = np.array([0.3, -0.2, 0.7])
    v = v0 + np.cross(w, r - c)
    a["m"][:] = m
    a["x"], a["y"], a["z"] = r[:, 0].copy(), r[:, 1].copy(), r[:, 2].copy()
    a["vx"], a["vy"], a["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    a["u"][:] = rng.uniform(0.0, 5.0, n)
    g = np.array([0.0, -1.0, -9.81])
    p = dict(wl.default_params(0), gravity=1, g_uniform=tuple(g))
    d = oracle.diagnostics(p, a)
    M = m.sum()
    q = r - c
    I = (m[:, None, None] * ((q * q).sum(1)[:, None, None] * np.eye(3)
                             - q[:, :, None] * q[:, None, :])).sum(0)
    L = M * np.cross(c, v0) + I @ w
    scale = M * (np.linalg.norm(c) + 5.0) * (np.linalg.norm(v0) + 5.0)
    assert np.allclose(d["p"], M * v0, rtol=0, atol=1e-12 * M * 5.0)
    assert np.allclose(d["L"], L, rtol=0, atol=1e-12 * scale)
    assert d["e_kin"] == pytest.approx(0.5 * M * v0 @ v0 + 0.5 * w @ I @ w, rel=1e-12)
    assert d["e_int"] == pytest.approx((m * a["u"]).sum(), rel=1e-14)
    assert d["e_pot"] == pytest.approx(-M * g @ c, rel=1e-12)
