"""Angular momentum of a spinning elastic sphere (§3.2, the rotation test of
the correction tensor, Eq. 20-22).

* Without strength the pair forces act along the line of centres and are
  antisymmetric, so sum m r x a vanishes and L is kept to round-off.
* With strength the force of Eq. 7 is not central; the deviatoric stress
  grows from the strain rate of Eq. 18-19. A rigid rotation has no strain
  rate, but the uncorrected SPH gradient of a rotating field near the free
  surface reports one, and the stress it builds exerts a spurious torque.
  The correction tensor makes the gradient of a linear field (a rigid
  rotation is one) exact, so L drifts far less with C than with C = I.
  The paper finds the uncorrected error above 1 % after one turn and the
  corrected one below 1e-3; the test runs a small fraction of a turn and
  asks for the same order: C at least five times better than C = I.
"""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import workloads as wl

NSTEPS = 200


def _dl(n, strength, correction, nsteps=NSTEPS):
    w = wl.spinning_sphere(n, correction=correction)
    mats = [dict(m, strength=strength) for m in w.materials]
    p = dict(w.params, precision=0)
    st, info0 = oracle.derivatives(p, mats, w.arrays)
    L0 = np.array(info0["L"])
    P0 = np.array(info0["p"])
    info = oracle.step(p, mats, st, w.dt, nsteps=nsteps)[1][-1] if nsteps else info0
    L = np.array(info["L"])
    P = np.array(info["p"])
    m = w.arrays["m"]
    vscale = float(np.sum(m * np.hypot(w.arrays["vx"], w.arrays["vy"])))
    return (np.linalg.norm(L - L0) / np.linalg.norm(L0), np.linalg.norm(P - P0) / vscale, L0)


def test_spin_is_about_z():
    _, _, L0 = _dl(1000, 1, 1, nsteps=0)
    assert L0[2] > 0 and np.hypot(L0[0], L0[1]) < 1e-2 * L0[2]


@pytest.mark.parametrize("correction", [0, 1])
def test_without_strength_angular_momentum_is_exact(correction):
    dl, dp, _ = _dl(1000, 0, correction)
    assert dl < 1e-12, dl
    assert dp < 1e-12, dp


def test_correction_tensor_keeps_angular_momentum():
    dl_c, dp_c, _ = _dl(1000, 1, 1)
    dl_i, dp_i, _ = _dl(1000, 1, 0)
    # linear momentum stays exact either way (Eq. 7 is antisymmetric)
    assert dp_c < 1e-12 and dp_i < 1e-12, (dp_c, dp_i)
    assert dl_c < 1e-4, dl_c
    assert dl_i > 5 * dl_c, (dl_i, dl_c)
