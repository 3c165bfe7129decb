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
