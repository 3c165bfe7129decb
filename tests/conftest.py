"""Shared fixtures. GPU tests carry the ``gpu`` marker; the rest run on CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def _oracle_built():
    import oracle
    oracle.build()
    yield


def cloud(n, seed=7, spacing=1.0, jitter=0.25, mat=None, vsig=0.0, ssig=0.0, shape="ball"):
    """Jittered lattice blob with seeded velocities and stresses (test input)."""
    from paper_2603_19764_b300 import workloads as wl
    rng = wl.SplitMix64(seed)
    mat = mat or wl.basalt_material()
    if shape == "ball":
        pos = wl.lattice_sphere(n, spacing)
    else:
        k = int(round(n ** (1 / 3)))
        g = np.stack(np.meshgrid(*(np.arange(k),) * 3, indexing="ij"), -1).reshape(-1, 3)
        pos = g[:n].astype(np.float64) * spacing
    pos = pos + rng.uniform(3 * n, -jitter * spacing, jitter * spacing).reshape(n, 3)
    a = wl._empty_arrays(n)
    a["x"], a["y"], a["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    a["m"][:] = mat["rho0"] * spacing ** 3 * (1.0 + 0.2 * rng.uniform(n, -1, 1))
    a["h"][:] = wl.lattice_h(mat, a["m"])
    if vsig:
        v = rng.normal(3 * n, vsig).reshape(n, 3)
        a["vx"], a["vy"], a["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    if ssig:
        s = rng.normal(5 * n, ssig).reshape(n, 5)
        for q, f in enumerate(("sxx", "syy", "sxy", "sxz", "syz")):
            a[f] = s[:, q].copy()
    a["u"][:] = rng.uniform(n, 0.0, 2.0e6)
    return a


def check_density_solve(g, ref, p, mats, arrays, rho_tol):
    """Density solve of the CUDA path against the FP64 oracle.

    * Eq. 1 at the CUDA path's own H: its density is the FP64 kernel sum
      there to the form's rounding (rho_tol), and its count is the exact
      count there.
    * Eq. 2: that H meets the constraint to h_tol, up to the same rounding in
      the path's own evaluation of it, unless it sits at the cap with too few
      neighbours; Eq. 3 there gives its Omega to 10 rho_tol, relative.
    * Against the oracle's own solve: both stop at the first radius with
      |(4 pi / 3) H^3 rho / (n_ngb m) - 1| <= h_tol, so two valid radii differ
      by up to 2 h_tol / (3 Omega) in ln H and their densities by up to
      2 h_tol |1 - Omega| / Omega in ln rho (Eq. 3 gives d ln rho / d ln H =
      3 (Omega - 1)). For a particle with few neighbours Omega is small and
      this window can exceed the form's rounding."""
    import oracle
    st = dict(arrays, h=g["h"])
    rho, om, cnt = oracle.density_given_h(p, st)
    assert np.array_equal(cnt, g["nngb"])
    assert np.max(np.abs(g["rho"] / rho - 1)) < rho_tol
    m = np.asarray(arrays["m"])
    rho0 = np.array([mats[k]["rho0"] for k in np.asarray(arrays["mat"])])
    hcap = p["h_cap_factor"] * np.cbrt(3.0 * p["n_ngb"] * m / (4.0 * np.pi * rho0))
    gq = 4.0 * np.pi / 3.0 * g["h"] ** 3 * rho / (p["n_ngb"] * m) - 1.0
    capped = (g["h"] >= hcap * (1 - 1e-6)) & (gq < 0)
    assert np.all(capped | (np.abs(gq) <= p["h_tol"] + rho_tol)), np.max(np.abs(gq[~capped]))
    # Eq. 3 at that H (a capped particle takes Omega = 1); relative, as the
    # forces carry 1 / Omega
    nc = ~capped
    rel_om = np.abs(g["omega"][nc] / om[nc] - 1)
    assert np.all(rel_om < 10 * rho_tol), np.max(rel_om)
    win = (2.0 * p["h_tol"] + rho_tol) * np.abs(1.0 - om) / np.maximum(om, 1e-12)
    rel = np.abs(g["rho"] / ref["rho"] - 1)
    assert np.all(rel < rho_tol + win), np.max(rel - win)
