"""Artificial viscosity (Eq. 5-8) and the time step (Eq. 38-39) of the
oracle against their closed forms for one pair.

Two particles on the x axis inside each other's support. The viscous terms
are the difference between the oracle's derivatives with (alpha, beta) on
and off: the density solve, the EOS and the pressure and strength terms do
not depend on them. The test restates Eq. 5-8 for the pair from the
kernel derivative (pinned in test_oracle_pointwise.py) and the oracle's own
state (H, rho, c_s): an approaching pair gets a_i = -m_j Pi grad W_bar and
du_i = 1/2 m_j Pi v_ij . grad W_bar, with mu from the averaged support
radius; a receding pair gets nothing. A dropped 1/2, a wrong sign of the
approach test, W(H_i) in place of the averaged kernel, or epsilon on the
wrong term each fail it. The time step is restated the same way: the
smaller of the acceleration and CFL criteria, the latter with the
longitudinal sound speed and the pair's mu where it approaches."""
import numpy as np
import pytest

import oracle
from paper_2603_19764_b300 import workloads as wl


def _pair(v, d=3.0):
    mat = wl.basalt_material()
    a = wl._empty_arrays(2)
    a["m"][:] = mat["rho0"] * 1.0
    a["x"][:] = [0.0, d]
    a["vx"][:] = [v, -v]          # v > 0: the two approach each other
    a["vy"][:] = [0.3 * v, 0.0]   # a transverse part: only v . r enters mu
    a["u"][:] = 1.0e5
    a["h"][:] = wl.lattice_h(mat, a["m"])
    return a, [mat]


def _derivs(a, mats, alpha, beta):
    p = dict(wl.default_params(0), av_alpha=alpha, av_beta=beta)
    st, _ = oracle.derivatives(p, mats, a)
    return st, p


@pytest.mark.parametrize("v", [50.0, 400.0])
def test_approaching_pair_matches_eq_5_to_8(v):
    a, mats = _pair(v)
    on, p = _derivs(a, mats, 1.0, 2.0)
    off, _ = _derivs(a, mats, 0.0, 0.0)
    H, rho, cs, m = on["h"], on["rho"], on["cs"], a["m"]
    assert np.array_equal(H, off["h"]) and np.array_equal(rho, off["rho"])
    for i, j in ((0, 1), (1, 0)):
        rij = np.array([a["x"][i] - a["x"][j], a["y"][i] - a["y"][j], a["z"][i] - a["z"][j]])
        vij = np.array([a["vx"][i] - a["vx"][j], a["vy"][i] - a["vy"][j],
                        a["vz"][i] - a["vz"][j]])
        r = np.linalg.norm(rij)
        assert r < min(H[i], H[j]) and vij @ rij < 0
        hb = 0.5 * (H[i] + H[j])
        mu = hb * (vij @ rij) / (r * r + p["av_eps"] * hb * hb)
        Pi = (-p["av_alpha"] * 0.5 * (cs[i] + cs[j]) * mu + p["av_beta"] * mu * mu) \
            / (0.5 * (rho[i] + rho[j]))
        gradWbar = 0.5 * (oracle.dWdr(r, H[i]) + oracle.dWdr(r, H[j])) * rij / r
        da = -m[j] * Pi * gradWbar
        du = 0.5 * m[j] * Pi * (vij @ gradWbar)
        got_a = np.array([on[f][i] - off[f][i] for f in ("ax", "ay", "az")])
        assert got_a == pytest.approx(da, rel=1e-10, abs=1e-12 * np.abs(da).max())
        assert on["dudt"][i] - off["dudt"][i] == pytest.approx(du, rel=1e-10)
        assert Pi > 0 and du > 0   # viscosity heats an approaching pair


def test_receding_pair_has_no_viscosity():
    a, mats = _pair(-200.0)
    on, _ = _derivs(a, mats, 1.0, 2.0)
    off, _ = _derivs(a, mats, 0.0, 0.0)
    for f in ("ax", "ay", "az", "dudt"):
        assert np.array_equal(on[f], off[f]), f


def test_viscous_momentum_and_energy_balance():
    """Eq. 7-8 for an equal-mass pair: the viscous forces cancel, and the
    heating equals the kinetic energy they remove."""
    a, mats = _pair(300.0)
    on, _ = _derivs(a, mats, 1.0, 2.0)
    off, _ = _derivs(a, mats, 0.0, 0.0)
    m = a["m"]
    da = {f: on[f] - off[f] for f in ("ax", "ay", "az", "dudt")}
    for f in ("ax", "ay", "az"):
        assert m[0] * da[f][0] + m[1] * da[f][1] == pytest.approx(0.0, abs=1e-9 * abs(m[0] * da[f][0]))
    dke = sum(m[k] * (a["vx"][k] * da["ax"][k] + a["vy"][k] * da["ay"][k]
                      + a["vz"][k] * da["az"][k]) for k in range(2))
    heat = m[0] * da["dudt"][0] + m[1] * da["dudt"][1]
    assert heat == pytest.approx(-dke, rel=1e-10)


def _dt_by_hand(a, st, p, mats, approach):
    """Eq. 38-39 for the pair, restated: eps = H (the reading of the
    softening length), c the longitudinal speed sqrt(c^2 + 4 Gamma / (3 rho))
    of a material with strength, mu_ij of Eq. 6 where the pair approaches."""
    G = mats[0]["shear_G"]
    out = []
    for i, j in ((0, 1), (1, 0)):
        acc = np.sqrt(st["ax"][i] ** 2 + st["ay"][i] ** 2 + st["az"][i] ** 2)
        ta = p["eta_a"] * np.sqrt(st["h"][i] / acc) if acc > 0 else np.inf
        rij = np.array([a["x"][i] - a["x"][j], a["y"][i] - a["y"][j], a["z"][i] - a["z"][j]])
        vij = np.array([a["vx"][i] - a["vx"][j], a["vy"][i] - a["vy"][j], a["vz"][i] - a["vz"][j]])
        hb = 0.5 * (st["h"][i] + st["h"][j])
        mu = hb * (vij @ rij) / (rij @ rij + p["av_eps"] * hb * hb)
        assert (mu < 0) == approach
        cl = np.sqrt(st["cs"][i] ** 2 + 4.0 / 3.0 * G / st["rho"][i])
        vsig = (1 + 0.6 * p["av_alpha"]) * cl + 0.6 * p["av_beta"] * abs(min(0.0, mu))
        out.append(min(ta, p["eta_c"] * st["h"][i] / vsig))
    return min(out)


@pytest.mark.parametrize("v", [300.0, -300.0])
def test_time_step_cfl_bound(v):
    a, mats = _pair(v)
    p = wl.default_params(0)
    st, info = oracle.derivatives(p, mats, a)
    assert info["dt_next"] == pytest.approx(_dt_by_hand(a, st, p, mats, v > 0), rel=1e-12)


def test_time_step_acceleration_bound():
    """A strong uniform field makes the acceleration criterion bind."""
    a, mats = _pair(300.0)
    p = dict(wl.default_params(0), gravity=1, g_uniform=(0.0, 0.0, -1.0e12))
    st, info = oracle.derivatives(p, mats, a)
    acc = np.sqrt(st["ax"] ** 2 + st["ay"] ** 2 + st["az"] ** 2)
    ta = p["eta_a"] * np.sqrt(st["h"] / acc)
    assert info["dt_next"] == pytest.approx(ta.min(), rel=1e-12)
    assert info["dt_next"] == pytest.approx(_dt_by_hand(a, st, p, mats, True), rel=1e-12)
