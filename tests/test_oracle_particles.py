"""Pins of the oracle's particle-set functions.

* neighbour sets: O(N^2) brute force = uniform grid = scipy's KD-tree;
* density (Eq. 1): a perfect lattice reproduces the lattice sum and rho0;
* grad-h term (Eq. 3): Omega against a finite difference of rho(H);
* smoothing-length solve: the constant-kernel-mass condition (Eq. 2);
* momentum and energy: the pair terms of Eq. 4, 7, 8, 18, 19 conserve
  sum m a and sum m (v.a + du/dt) exactly;
* gradient: a linear velocity field gives G = A exactly with the
  correction tensor (Eq. 20-22);
* integrator (§2.4): constant acceleration is integrated exactly;
* elastic wave: a standing longitudinal wave travels at
  sqrt((K + 4/3 G) / rho).
"""
import math

import numpy as np
import pytest
from scipy import optimize
from scipy.spatial import cKDTree

import oracle
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import cloud


def _params(**kw):
    p = wl.default_params(0)
    p.update(kw)
    return p


# ------------------------------------------------------------ neighbours ---
@pytest.mark.parametrize("periodic", [0, 1])
def test_neighbour_sets_three_ways(periodic):
    rng = np.random.default_rng(1)
    n = 1500
    L = 12.0
    pos = rng.uniform(0, L, size=(n, 3))
    h = rng.uniform(0.8, 2.2, size=n)
    a = dict(x=pos[:, 0], y=pos[:, 1], z=pos[:, 2], h=h)
    p = _params(periodic=periodic, box_lo=(0, 0, 0), box_hi=(L, L, L))
    tree = cKDTree(pos, boxsize=L if periodic else None)
    for i in rng.choice(n, 60, replace=False):
        g0 = oracle.neighbours(p, a, i, 0)
        b0 = oracle.neighbours(p, a, i, 0, brute_force=True)
        assert np.array_equal(g0, b0)
        assert np.all(np.diff(g0) > 0)
        kd = np.sort(tree.query_ball_point(pos[i], h[i]))
        assert np.array_equal(g0, kd)
        g1 = oracle.neighbours(p, a, i, 1)
        b1 = oracle.neighbours(p, a, i, 1, brute_force=True)
        assert np.array_equal(g1, b1)
        d = pos - pos[i]
        if periodic:
            d -= L * np.round(d / L)
        r = np.sqrt((d ** 2).sum(1))
        union = np.nonzero((r < np.maximum(h, h[i])) & (np.arange(n) != i))[0]
        assert np.array_equal(g1, union)


def test_counts_given_h_match_kdtree():
    a = cloud(3000, seed=9, jitter=0.3)
    tree = cKDTree(np.stack([a["x"], a["y"], a["z"]], 1))
    c = oracle.count_neighbours(_params(), a)
    ref = np.array([len(tree.query_ball_point([a["x"][i], a["y"][i], a["z"][i]], a["h"][i])) - 1
                    for i in range(3000)])
    assert np.array_equal(c, ref)


# --------------------------------------------------------------- density ---
def test_lattice_density_is_lattice_sum():
    """Interior particle of a perfect cubic lattice: rho = m sum_n W(|n| D, H)."""
    k = 14
    D = 1.0
    g = np.stack(np.meshgrid(*(np.arange(k),) * 3, indexing="ij"), -1).reshape(-1, 3) * D
    n = g.shape[0]
    a = wl._empty_arrays(n)
    a["x"], a["y"], a["z"] = g[:, 0].copy(), g[:, 1].copy(), g[:, 2].copy()
    a["m"][:] = 1000.0 * D ** 3
    H = 2.6 * D                           # between the sqrt(6) and sqrt(8) shells
    a["h"][:] = H
    centre = int(np.argmin(((g - (k - 1) / 2 * D) ** 2).sum(1)))
    rho, om, cnt = oracle.density_given_h(_params(), a, idx=[centre])
    m = np.arange(-4, 5)
    v = np.stack(np.meshgrid(m, m, m, indexing="ij"), -1).reshape(-1, 3) * D
    r = np.sqrt((v ** 2).sum(1))
    lattice = 1000.0 * oracle.W(r, H).sum()
    assert rho[0] == pytest.approx(lattice, rel=1e-13)
    assert cnt[0] == int((r < H).sum()) - 1
    # rho0 within the kernel's discretisation error, which shrinks as H grows
    assert abs(rho[0] / 1000.0 - 1.0) < 1.2e-2
    errs = [abs(1000.0 * oracle.W(r, f * D).sum() / 1000.0 - 1.0) for f in (2.6, 2.9, 3.4)]
    assert errs[0] > errs[1] > errs[2]


def test_omega_matches_finite_difference():
    a = cloud(2500, seed=4, jitter=0.3)
    p = _params()
    idx = np.array([0, 10, 700, 2400])
    rho, om, _ = oracle.density_given_h(p, a, idx=idx)
    e = 1e-6
    for q, i in enumerate(idx):
        hp = dict(a, h=a["h"].copy())
        hm = dict(a, h=a["h"].copy())
        hp["h"][i] *= 1 + e
        hm["h"][i] *= 1 - e
        rp = oracle.density_given_h(p, hp, idx=[i])[0][0]
        rm = oracle.density_given_h(p, hm, idx=[i])[0][0]
        drho_dh = (rp - rm) / (2 * e * a["h"][i])
        assert om[q] == pytest.approx(1 + a["h"][i] / (3 * rho[q]) * drho_dh, rel=1e-6)


def test_density_solve_constant_kernel_mass():
    w = wl.granular_column()
    st, info = oracle.density_solve(w.params, w.materials, w.arrays)
    assert info["n_unconverged"] == 0
    lhs = 4 * math.pi / 3 * st["h"] ** 3 * st["rho"]
    rhs = w.params["n_ngb"] * st["m"]
    assert np.max(np.abs(lhs / rhs - 1)) <= w.params["h_tol"] * (1 + 1e-9)
    # the outputs belong to the final H
    rho, om, cnt = oracle.density_given_h(w.params, st)
    assert np.allclose(rho, st["rho"], rtol=1e-14, atol=0)
    assert np.allclose(om, st["omega"], rtol=1e-13, atol=0)
    assert np.array_equal(cnt, st["nngb"])
    # from a guess off by 20 % the solve lands on the same H
    off = dict(w.arrays, h=w.arrays["h"] * 1.2)
    st2, _ = oracle.density_solve(w.params, w.materials, off)
    assert np.allclose(st2["h"], st["h"], rtol=1e-9)


def test_lattice_interior_omega_near_one():
    w = wl.basalt_sphere(8000)
    st, _ = oracle.density_solve(w.params, w.materials, w.arrays)
    r = np.sqrt(st["x"] ** 2 + st["y"] ** 2 + st["z"] ** 2)
    inner = r < 0.5 * r.max()
    assert np.all(np.abs(st["omega"][inner] - 1) < 0.1)
    # Wendland C2 at 64 neighbours over-estimates a lattice density by ~1.4 %;
    # the 1 % position jitter spreads it to about 2.6 %
    assert np.all(np.abs(st["rho"][inner] / 2700 - 1) < 0.03)


# ---------------------------------------------------------------- forces ---
def _forces_state(n=1200, seed=5, **kw):
    mats = [wl.basalt_material(), dict(wl.basalt_material(), strength=0)]
    a = cloud(n, seed=seed, jitter=0.3, spacing=100.0, vsig=30.0, ssig=5e6, **kw)
    a["mat"][n // 2:] = 1
    p = _params()
    st, _ = oracle.density_solve(p, mats, a)
    st, S = oracle.eos_yield(p, mats, st)
    return p, mats, st, S


def test_momentum_and_energy_conserved():
    p, mats, st, S = _forces_state()
    out, _ = oracle.forces(p, mats, st, S=S)
    m = out["m"]
    a = np.stack([out["ax"], out["ay"], out["az"]], 1)
    scale = np.abs(m[:, None] * a).sum(0)
    assert np.all(np.abs((m[:, None] * a).sum(0)) < 1e-13 * scale)
    v = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    pw = m * ((v * a).sum(1) + out["dudt"])
    assert abs(pw.sum()) < 1e-12 * np.abs(m * (v * a).sum(1)).sum()


def test_strength_terms_alone_conserve():
    """Pressure and viscosity switched off: the S terms of Eq. 18-19 alone."""
    p, mats, st, S = _forces_state(seed=6)
    st = dict(st, pres=np.zeros_like(st["pres"]))
    p = dict(p, av_alpha=0.0, av_beta=0.0)
    out, _ = oracle.forces(p, mats, st, S=S)
    m = out["m"]
    a = np.stack([out["ax"], out["ay"], out["az"]], 1)
    assert np.abs(a).max() > 0
    assert np.all(np.abs((m[:, None] * a).sum(0)) < 1e-13 * np.abs(m[:, None] * a).sum(0))
    v = np.stack([out["vx"], out["vy"], out["vz"]], 1)
    assert abs((m * ((v * a).sum(1) + out["dudt"])).sum()) < 1e-12 * np.abs(
        m * (v * a).sum(1)).sum()


def test_linear_velocity_field_gives_exact_gradient():
    p, mats, st, S = _forces_state(seed=8)
    A = np.array([[0.3, -1.1, 0.4], [0.7, 0.2, -0.5], [-0.2, 0.9, -0.6]])
    x = np.stack([st["x"], st["y"], st["z"]], 1)
    v = x @ A.T + np.array([3.0, -2.0, 1.0])
    _, info = oracle.forces(p, mats, st, v=(v[:, 0], v[:, 1], v[:, 2]), S=S, want_tensors=True)
    assert info["n_cfallback"] == 0
    assert np.allclose(info["G"], A[None], rtol=0, atol=1e-9)
    # without the correction tensor only the interior is close to A
    _, info0 = oracle.forces(dict(p, correction_tensor=0), mats, st,
                             v=(v[:, 0], v[:, 1], v[:, 2]), S=S, want_tensors=True)
    err = np.abs(info0["G"] - A[None]).max(axis=(1, 2))
    assert err.max() > 1e-2
    r = np.sqrt((x ** 2).sum(1))
    assert np.median(err[r < 0.4 * r.max()]) < 0.25   # 30 % jitter, 20 % mass spread


def test_fixed_particles_get_no_derivatives():
    w = wl.granular_column()
    st, info = oracle.derivatives(w.params, w.materials, w.arrays)
    fixed = st["flags"] == 1
    for f in ("ax", "ay", "az", "dudt", "dsxx", "dsyz"):
        assert np.all(st[f][fixed] == 0.0)
    assert np.abs(st["az"][~fixed]).max() > 0


# ------------------------------------------------------------ integrator ---
def test_constant_acceleration_is_exact():
    """Two isolated particles under uniform g: x_n = x0 + n dt v + n(n-1)/2 dt^2 g."""
    mat = wl.granular_material()
    a = wl._empty_arrays(2)
    a["x"][:] = [0.0, 1e3]
    a["m"][:] = 1.0
    a["h"][:] = 0.1
    a["vx"][:] = [1.0, -2.0]
    a["vz"][:] = [0.5, 0.0]
    a["rho"][:] = 1600.0
    a["flags"][1] = 1                      # the second particle is fixed
    g = np.array([0.0, 0.0, -9.81])
    p = _params(gravity=1, g_uniform=tuple(g), max_sweeps=64)
    st, _ = oracle.derivatives(p, [mat], a)
    dt, n = 0.01, 25
    out, infos = oracle.step(p, [mat], st, dt, nsteps=n)
    assert out["x"][0] == pytest.approx(n * dt * 1.0, rel=1e-12)
    assert out["z"][0] == pytest.approx(n * dt * 0.5 + n * (n - 1) / 2 * dt * dt * g[2], rel=1e-12)
    assert out["vz"][0] == pytest.approx(0.5 + n * dt * g[2], rel=1e-12)   # v at n + 1/2
    assert out["x"][1] == 1e3 and out["vx"][1] == -2.0


# ---------------------------------------------------------- elastic wave ---
def test_elastic_wave_speed():
    """Standing longitudinal wave in a periodic 64 x 8 x 8 lattice. The
    material is pre-compressed so that P > 0 and Y never binds."""
    w = wl.periodic_wave_box(64, 8, 8, amp=1e-3)
    mat = dict(w.materials[0], rho0=990.0)
    a = w.arrays
    st, info = oracle.derivatives(w.params, [mat], a)
    rho = float(np.mean(st["rho"]))
    c_l = math.sqrt(mat["c0"] ** 2 + 4.0 / 3.0 * mat["shear_G"] / rho)
    lx = w.params["box_hi"][0]
    k = 2 * math.pi / lx
    x0 = a["x"].copy()
    s = np.sin(k * x0)
    period = lx / c_l
    dt = w.dt
    nsteps = int(1.3 * period / dt)
    amps = []

    def cb(i, arr, inf):
        amps.append((arr["vx"] * s).sum() / (s * s).sum())

    oracle.step(w.params, [mat], st, dt, nsteps=nsteps, callback=cb)
    t = (np.arange(nsteps) + 0.5) * dt
    amps = np.array(amps)
    f = lambda tt, A, om, ph: A * np.cos(om * tt + ph)
    (A, om, ph), _ = optimize.curve_fit(f, t, amps, p0=[amps[0], c_l * k, 0.0])
    assert abs(om / k / c_l - 1) < 0.01


# ------------------------------------------------- gradient forms (§2.2) ---
@pytest.mark.parametrize("form", [0, 1])
def test_linear_field_exact_in_both_gradient_forms(form):
    """With the correction tensor built in the same form as F, G = F C = A
    for any linear field, whatever the kernel weights (they cancel)."""
    p, mats, st, S = _forces_state(seed=9)
    A = np.array([[0.3, -1.1, 0.4], [0.7, 0.2, -0.5], [-0.2, 0.9, -0.6]])
    x = np.stack([st["x"], st["y"], st["z"]], 1)
    v = x @ A.T - np.array([1.0, 2.0, 0.5])
    _, info = oracle.forces(dict(p, gradient_form=form), mats, st,
                            v=(v[:, 0], v[:, 1], v[:, 2]), S=S, want_tensors=True)
    assert info["n_cfallback"] == 0
    assert np.allclose(info["G"], A[None], rtol=0, atol=1e-9)


def test_symmetric_gradient_is_better_at_a_material_interface():
    """§2.2: the symmetric form of Eq. 20-21 does better at material
    interfaces than the non-symmetric one. A 24^3 block with a density jump
    of 3 across z = 0 (same spacing, masses in proportion), a linear
    velocity field, no correction tensor: the worst gradient error on the
    interface layer is smaller with the symmetric form; away from the
    interface the two forms are alike."""
    mats = [wl.basalt_material(), dict(wl.basalt_material(), rho0=900.0, strength=0)]
    a = cloud(13824, seed=3, jitter=0.05, spacing=100.0, shape="box")
    z = a["z"]
    zc = np.median(z)
    top = z > zc
    a["mat"][top] = 1
    a["m"][top] *= 900.0 / 2700.0
    p = _params(correction_tensor=0)
    st, _ = oracle.density_solve(p, mats, a)
    st, S = oracle.eos_yield(p, mats, st)
    A = np.array([[0.3, -1.1, 0.4], [0.7, 0.2, -0.5], [-0.2, 0.9, -0.6]])
    x = np.stack([st["x"], st["y"], st["z"]], 1)
    v = x @ A.T
    lo, hi = x.min(0), x.max(0)
    inner = np.all((x[:, :2] > lo[:2] + 600) & (x[:, :2] < hi[:2] - 600), axis=1)
    iface = inner & (np.abs(z - zc) < 150)
    bulk = inner & (np.abs(z - zc) > 450) & (z > lo[2] + 600) & (z < hi[2] - 600)
    err = {}
    for form in (0, 1):
        _, info = oracle.forces(dict(p, gradient_form=form), mats, st,
                                v=(v[:, 0], v[:, 1], v[:, 2]), S=S, want_tensors=True)
        err[form] = np.abs(info["G"] - A[None]).max(axis=(1, 2))
    assert iface.sum() > 300 and bulk.sum() > 300
    assert err[0][iface].max() < 0.9 * err[1][iface].max(), (err[0][iface].max(), err[1][iface].max())
    assert np.median(err[0][iface]) < np.median(err[1][iface])
    ratio = np.median(err[0][bulk]) / np.median(err[1][bulk])
    assert 0.5 < ratio < 2.0, ratio


def test_lone_particle_grad_h_term_and_cap():
    """A particle alone: rho = m W(0, H) = 21 m / (2 pi H^3), and Eq. 3
    gives Omega = 1 + (H / 3 rho)(-3 rho / H) = 0 exactly. The solve caps
    its H and, by the cap reading, gives it Omega = 1, so that the terms
    over Omega rho stay finite (no neighbours: du/dt = 0, dS/dt = 0)."""
    a = cloud(1, seed=3, spacing=100.0, vsig=5.0, ssig=1e6)
    p = _params()
    H = float(a["h"][0])
    rho, om, cnt = oracle.density_given_h(p, a)
    assert rho[0] == pytest.approx(21.0 * a["m"][0] / (2.0 * math.pi * H ** 3), rel=1e-14)
    assert abs(om[0]) < 1e-14 and cnt[0] == 0
    st, info = oracle.derivatives(p, [wl.basalt_material()], a)
    assert info["n_capped"] == 1 and st["omega"][0] == 1.0
    for f in ("ax", "ay", "az", "dudt", "dsxx", "dsyz"):
        assert st[f][0] == 0.0, f
