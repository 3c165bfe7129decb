"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI:

* tiny and ragged inputs: one particle (no neighbour, H capped, C = I),
  fewer particles than a 32-particle bucket, a bucket plus one;
* coincident particles (pairs at r = 0, which every pair term multiplies
  by x_ij = 0, and which the count includes unless j = i);
* a body whose particles are all fixed (no derivative, no motion);
* mixed materials in one body (Tillotson with strength, linear EOS with
  a pressure-only yield, Tillotson without strength);
* the parameter variants: the stress rate as printed (Eq. 25-29), the
  sqrt(3 J2) yield normalisation, no thermal softening, the shear modulus
  of Eq. 30 (Gamma = 0.6 rho c^2);
* a batch of many tiny systems (1 to 40 particles each, far apart);
* a long thin rod whose cell grid is about 800 cells long, so that the
  Morton sort keys need more than 24 bits and all four 8-bit radix passes
  run (the other workloads need one to three; a pass whose digit and every
  higher one are zero in all keys is left out, and the sorted order is then
  read from the buffers of the last pass that ran).

Tolerances as in the parity suite: counts bit-exact given the GPU's H;
density 1e-6 (FP64) / 1e-5 (FP32) relative at the GPU's H, and against the
oracle's own solve within the window its stopping rule leaves; derivatives
1e-9 / 1e-4 of the field's max norm."""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import build, sph
from paper_2603_19764_b300 import workloads as wl
from tests.conftest import check_density_solve, cloud

pytestmark = pytest.mark.gpu

DERIVS = ("ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz")
RHO_TOL = {0: 1e-6, 1: 1e-5}
DERIV_TOL = {0: 1e-9, 1: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _p(params, precision):
    return dict(params, precision=precision, h_tol=1e-10 if precision == 0 else 1e-6)


def _maxnorm_err(a, b):
    scale = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)


def _compare(g, ref, p, mats, arrays, precision):
    check_density_solve(g, ref, p, mats, arrays, RHO_TOL[precision])
    for f in DERIVS:
        e = _maxnorm_err(g[f], ref[f])
        assert e < DERIV_TOL[precision], (f, e)


def _prime_check(arrays, mats, params, precision):
    p = _p(params, precision)
    sim = sph.Simulation(arrays, mats, p)
    info = sim.prime()
    g = sim.by_id()
    sim.close()
    ref, rinfo = oracle.derivatives(p, mats, arrays)
    assert info["n_capped"] == rinfo["n_capped"]
    assert info["n_cfallback"] == rinfo["n_cfallback"]
    _compare(g, ref, p, mats, arrays, precision)
    assert info["dt_next"] == pytest.approx(rinfo["dt_next"], rel=1e-6 if precision == 0 else 1e-4)
    return g, info


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 97])
def test_tiny_and_ragged_inputs(n, precision):
    a = cloud(n, seed=50 + n, jitter=0.2, spacing=100.0, vsig=10.0, ssig=1e6)
    g, info = _prime_check(a, [wl.basalt_material()], wl.default_params(), precision)
    if n == 1:
        assert info["n_capped"] == 1 and g["nngb"][0] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_coincident_particles(precision):
    a = cloud(400, seed=61, jitter=0.2, spacing=100.0, vsig=10.0, ssig=1e6)
    for k in ("x", "y", "z"):
        a[k][1] = a[k][0]
        a[k][6] = a[k][7] = a[k][5]
    g, _ = _prime_check(a, [wl.basalt_material()], wl.default_params(), precision)
    assert np.all(np.isfinite(g["ax"]))


def test_all_particles_fixed():
    w = wl.granular_column()
    a = dict(w.arrays, flags=np.ones(w.n, np.int32))
    p = _p(w.params, 0)
    sim = sph.Simulation(a, w.materials, p)
    sim.prime()
    for _ in range(3):
        sim.step(w.dt)
    g = sim.by_id()
    sim.close()
    for f in ("x", "y", "z", "vx", "vy", "vz", "sxx", "syz"):
        assert np.array_equal(g[f], a[f]), f
    for f in DERIVS:
        assert np.all(g[f] == 0.0), f


def _mixed_body(n=3000, seed=62):
    gran = wl.granular_material()
    mats = [wl.basalt_material(), gran, dict(wl.basalt_material(), strength=0)]
    a = cloud(n, seed=seed, jitter=0.25, spacing=100.0, vsig=10.0, ssig=2e6)
    x = a["x"]
    t1, t2 = np.quantile(x, [1 / 3, 2 / 3])
    a["mat"][(x > t1) & (x <= t2)] = 1
    a["mat"][x > t2] = 2
    m1 = a["mat"] == 1
    a["m"][m1] *= gran["rho0"] / wl.basalt_material()["rho0"]
    a["u"][m1] = 0.0
    return a, mats


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_materials(precision):
    a, mats = _mixed_body()
    _prime_check(a, mats, wl.default_params(), precision)
    # and a few full steps
    p = _p(wl.default_params(), precision)
    ref, rinfo = oracle.derivatives(p, mats, a)
    dt = 0.5 * rinfo["dt_next"]
    sim = sph.Simulation(a, mats, p)
    sim.prime()
    for _ in range(5):
        ref, _ = oracle.step(p, mats, ref, dt)
        sim.step(dt)
    g = sim.by_id()
    sim.close()
    assert np.max(np.abs(g["rho"] / ref["rho"] - 1)) < RHO_TOL[precision]
    for f in DERIVS:
        e = _maxnorm_err(g[f], ref[f])
        assert e < DERIV_TOL[precision], (f, e)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", ["jaumann_printed", "yield_sqrt3", "no_softening",
                                     "shear_eq30"])
def test_parameter_variants(variant, precision):
    w = wl.impact(6000, 700, seed=63)
    params, mats = dict(w.params), list(w.materials)
    if variant == "jaumann_printed":
        params["jaumann"] = 1
    elif variant == "yield_sqrt3":
        params["yield_norm"] = 1
    elif variant == "shear_eq30":
        # Eq. 30: Gamma = 0.6 rho c^2 per particle (Poisson ratio 0.25)
        mats = [dict(m, shear_G=-1.0) for m in mats]
    else:
        mats = [dict(m, thermal_softening=0) for m in mats]
    _prime_check(w.arrays, mats, params, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_of_many_tiny_systems(precision):
    rng = np.random.default_rng(64)
    sizes = rng.integers(1, 41, size=120)
    parts, systems, off = [], [], 0
    for k, nk in enumerate(sizes):
        a = cloud(int(nk), seed=100 + k, jitter=0.2, spacing=100.0, vsig=10.0, ssig=1e6)
        a["x"] += 1.0e5 * k
        parts.append(a)
        systems.append((off, int(nk)))
        off += int(nk)
    arr = {f: np.concatenate([a[f] for a in parts]) for f in parts[0]}
    arr["id"] = np.arange(off, dtype=np.int64)
    mats = [wl.basalt_material()]
    p = _p(wl.default_params(), precision)
    sim = sph.Simulation(arr, mats, p, systems=systems)
    sim.prime()
    infos = sim.batch_info()
    g = sim.by_id()
    sim.close()
    capped = 0
    for k, (o, nk) in enumerate(systems):
        sl = slice(o, o + nk)
        a = {f: v[sl].copy() for f, v in arr.items()}
        a["id"] = np.arange(nk, dtype=np.int64)
        ref, rinfo = oracle.derivatives(p, mats, a)
        gk = {f: v[sl] for f, v in g.items()}
        _compare(gk, ref, p, mats, dict(a), precision)
        capped += rinfo["n_capped"]
        # per-system reports carry the system's own time step and sums
        assert infos[k]["dt_next"] == pytest.approx(rinfo["dt_next"],
                                                    rel=1e-6 if precision == 0 else 1e-4)
        assert infos[k]["e_kin"] == pytest.approx(rinfo["e_kin"], rel=1e-9)
    # the counters are batch totals
    assert infos[0]["n_capped"] == capped


@pytest.mark.parametrize("precision", [0, 1])
def test_rod_with_four_sort_passes(precision):
    rng = wl.SplitMix64(71)
    mat = wl.basalt_material()
    nx, ny, nz, sp = 2000, 4, 4, 100.0
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                 -1).reshape(-1, 3).astype(np.float64) * sp
    n = g.shape[0]
    g = g + rng.uniform(3 * n, -0.2 * sp, 0.2 * sp).reshape(n, 3)
    a = wl._empty_arrays(n)
    a["x"], a["y"], a["z"] = g[:, 0].copy(), g[:, 1].copy(), g[:, 2].copy()
    a["m"][:] = mat["rho0"] * sp ** 3
    a["h"][:] = wl.lattice_h(mat, a["m"])
    v = rng.normal(3 * n, 10.0).reshape(n, 3)
    a["vx"], a["vy"], a["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    a["u"][:] = rng.uniform(n, 0.0, 2.0e6)
    # the first sort's grid (cell edge: the largest H) needs 10 bits per axis
    cells_x = int(np.floor((a["x"].max() - a["x"].min()) / a["h"].max())) + 1
    assert 512 < cells_x <= 1024
    _prime_check(a, [mat], wl.default_params(), precision)

