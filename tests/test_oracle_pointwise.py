"""Pins of the oracle's point functions against closed forms and limits.

Kernel (§3, Wendland C2), EOS (linear, Tillotson), yield (§2.3, Eq. 34-37),
radial return (Eq. 31-33), stress rate (Eq. 13, 23-29), 3x3 inverse and the
given external field. None of these tests retypes the oracle's formula: each
checks a property the mathematics or the paper fixes.
"""
import math

import numpy as np
import pytest
from scipy import integrate, linalg

import oracle
from paper_2603_19764_b300 import workloads as wl


# ---------------------------------------------------------------- kernel ---
@pytest.mark.parametrize("H", [1.0, 0.37, 2.7e3])
def test_kernel_normalised(H):
    """4 pi int_0^H W r^2 dr = 1 (exact for Wendland C2)."""
    val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * oracle.lib().ref_W(r, H), 0, H,
                            epsabs=0, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-11


def test_kernel_compact_and_smooth():
    H = 1.3
    assert oracle.lib().ref_W(H, H) == 0.0 and oracle.lib().ref_W(1.5 * H, H) == 0.0
    # C2 at the support edge: W ~ (1 - q)^4, so W(H - d) / d^3 -> 0
    for d in (1e-2, 1e-3):
        assert oracle.lib().ref_W(H - d, H) / d ** 3 < 50 * d
    # maximum at r = 0 and monotone decreasing
    r = np.linspace(0, H, 200)
    w = oracle.W(r, H)
    assert np.all(np.diff(w) <= 0)


@pytest.mark.parametrize("q", [0.05, 0.3, 0.5, 0.77, 0.95])
def test_kernel_derivatives_fd(q):
    H = 1.7
    r = q * H
    e = 1e-6
    fd_r = (oracle.lib().ref_W(r + e, H) - oracle.lib().ref_W(r - e, H)) / (2 * e)
    fd_h = (oracle.lib().ref_W(r, H + e) - oracle.lib().ref_W(r, H - e)) / (2 * e)
    assert abs(oracle.lib().ref_dWdr(r, H) - fd_r) < 1e-7 * max(1.0, abs(fd_r))
    assert abs(oracle.lib().ref_dWdH(r, H) - fd_h) < 1e-7 * max(1.0, abs(fd_h))


def test_kernel_scaling_identity():
    """H dW/dH = -3 W - r dW/dr for any kernel of the form H^-3 f(r/H)."""
    H = 0.9
    for q in np.linspace(0.01, 0.99, 23):
        r = q * H
        lhs = H * oracle.lib().ref_dWdH(r, H)
        rhs = -3 * oracle.lib().ref_W(r, H) - r * oracle.lib().ref_dWdr(r, H)
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


# ------------------------------------------------------------------- EOS ---
def test_linear_eos():
    m = dict(wl.granular_material(), p_min=-math.inf)
    P, c = oracle.eos(m, np.array([1600.0, 1700.0, 1500.0]), np.zeros(3))
    assert np.allclose(P, [0.0, 100.0 ** 2 * 100, -100.0 ** 2 * 100], rtol=0, atol=1e-9)
    assert np.all(c == 100.0)
    # the granular medium carries no tension: P floored at zero, c unchanged
    P, c = oracle.eos(wl.granular_material(), np.array([1500.0, 1700.0]), np.zeros(2))
    assert np.array_equal(P, [0.0, 100.0 ** 2 * 100]) and np.all(c == 100.0)


def test_pressure_floor_tillotson():
    m = wl.basalt_material()
    P0, c0 = oracle.eos(m, 0.9 * m["rho0"], 0.0)
    assert P0 < 0
    P1, c1 = oracle.eos(dict(m, p_min=-1e6), 0.9 * m["rho0"], 0.0)
    assert P1 == -1e6 and c1 == c0


def test_tillotson_reference_state():
    m = wl.basalt_material()
    P, c = oracle.eos(m, m["rho0"], 0.0)
    assert abs(P) < 1e-6
    # at (rho0, 0) only the A mu term has a density derivative: c^2 = A / rho0
    assert abs(c ** 2 - m["A"] / m["rho0"]) < 1e-9 * m["A"] / m["rho0"]


def test_tillotson_cold_curve_and_gas_limit():
    m = wl.basalt_material()
    # u = 0: P = A mu + B mu^2 (cold compression curve)
    for eta in (1.05, 1.3, 2.0):
        P, _ = oracle.eos(m, eta * m["rho0"], 0.0)
        mu = eta - 1
        assert abs(P - (m["A"] * mu + m["B"] * mu * mu)) < 1e-9 * abs(P)
    # very low density, hot: the expanded form tends to the ideal gas a rho u
    rho, u = 1e-3 * m["rho0"], 5 * m["Ecv"]
    P, _ = oracle.eos(m, rho, u)
    assert abs(P - m["a"] * rho * u) < 1e-6 * m["a"] * rho * u


def test_tillotson_continuity():
    m = wl.basalt_material()
    for rho in (0.6 * m["rho0"], 0.9 * m["rho0"]):
        for ub in (m["Eiv"], m["Ecv"]):
            Pa, _ = oracle.eos(m, rho, ub * (1 - 1e-10))
            Pb, _ = oracle.eos(m, rho, ub * (1 + 1e-10))
            assert abs(Pa - Pb) < 1e-6 * (abs(Pa) + 1e3)
    # across rho0 at fixed u (condensed on both sides below Eiv)
    Pa, _ = oracle.eos(m, m["rho0"] * (1 - 1e-12), 1e6)
    Pb, _ = oracle.eos(m, m["rho0"] * (1 + 1e-12), 1e6)
    assert abs(Pa - Pb) < 1e-3 * abs(Pa)


@pytest.mark.parametrize("rho_f,u", [(1.2, 1e6), (1.0, 3e6), (0.8, 2e6), (0.8, 30e6),
                                     (0.7, 10e6), (1.5, 40e6)])
def test_tillotson_sound_speed_fd(rho_f, u):
    """c^2 = dP/drho|_u + P / rho^2 dP/du|_rho against central differences."""
    m = wl.basalt_material()
    rho = rho_f * m["rho0"]
    P, c = oracle.eos(m, rho, u)
    er, eu = rho * 1e-6, u * 1e-6
    dPr = (oracle.eos(m, rho + er, u)[0] - oracle.eos(m, rho - er, u)[0]) / (2 * er)
    dPu = (oracle.eos(m, rho, u + eu)[0] - oracle.eos(m, rho, u - eu)[0]) / (2 * eu)
    c2 = max(dPr + P / rho ** 2 * dPu, 0.01 * m["A"] / m["rho0"])
    assert abs(c ** 2 - c2) < 1e-5 * c2


# ----------------------------------------------------------------- yield ---
def test_yield_limits():
    m = wl.basalt_material()
    m.update(thermal_softening=0, mu_d=1e9)       # damaged branch out of the way for P >= 1
    # intercept Y0 (read at P = 1 Pa, where mu_d P already exceeds the intact curve)
    assert abs(oracle.yield_strength(m, 1.0, 0.0) - m["Y0"]) < 2 * m["mu_i"]
    assert abs(oracle.yield_strength(m, 1e16, 0.0) - m["Ym"]) < 1e-3 * m["Ym"]
    # initial slope mu_i
    slope = oracle.yield_strength(m, 2.0, 0.0) - oracle.yield_strength(m, 1.0, 0.0)
    assert abs(slope - m["mu_i"]) < 1e-6
    P = np.linspace(1.0, 1e10, 50)
    assert np.all(np.diff(oracle.yield_strength(m, P, 0.0)) > 0)


def test_yield_damaged_and_min():
    m = wl.basalt_material()
    m["thermal_softening"] = 0
    P = np.array([1e5, 1e7, 1e9, 1e10])
    Y = oracle.yield_strength(m, P, 0.0)
    Yd = m["mu_d"] * P
    assert np.all(Y <= Yd * (1 + 1e-15))
    assert Y[0] == pytest.approx(Yd[0], rel=1e-15)   # low P: damaged branch binds
    # negative pressure is clipped to zero: Y = min(Y0, 0) = 0
    assert oracle.yield_strength(m, -1e8, 0.0) == 0.0


def test_yield_paper_quartz_values():
    """Quartz strength set printed in §3 (Y0 = 0, Ym = 3.5 GPa, mu_i = 2, mu_d = 0.8)."""
    m = wl.basalt_material()
    m.update(Y0=0.0, Ym=3.5e9, mu_i=2.0, mu_d=0.8, thermal_softening=0)
    # with Y0 = 0 the intact curve passes through Ym / 2 at P = Ym / mu_i
    m2 = dict(m, mu_d=1e9)
    assert oracle.yield_strength(m2, 3.5e9 / 2.0, 0.0) == pytest.approx(1.75e9, rel=1e-14)
    # the two branches cross where mu_i P / (1 + mu_i P / Ym) = mu_d P
    Pc = (m["mu_i"] / m["mu_d"] - 1) * m["Ym"] / m["mu_i"]
    assert oracle.yield_strength(m, Pc, 0.0) == pytest.approx(m["mu_d"] * Pc, rel=1e-12)


def test_thermal_softening():
    m = wl.basalt_material()
    P = 1e8
    base = dict(m, thermal_softening=0)
    Y0 = oracle.yield_strength(base, P, 0.0)
    u_melt = (m["Tm"] - m["T0"]) * m["cv"]
    assert oracle.yield_strength(m, P, u_melt) == pytest.approx(0.0, abs=1e-6 * Y0)
    assert oracle.yield_strength(m, P, 2 * u_melt) == 0.0
    # cold: factor tanh(xi (Tm / T0 - 1)) lies in (0, 1) and is below 1
    Yc = oracle.yield_strength(m, P, 0.0)
    assert 0 < Yc < Y0
    assert Yc / Y0 == pytest.approx(math.tanh(m["xi"] * (m["Tm"] / m["T0"] - 1)), rel=1e-12)


# --------------------------------------------------------- radial return ---
def _full(S):
    return np.array([[S[0], S[2], S[3]], [S[2], S[1], S[4]], [S[3], S[4], -S[0] - S[1]]])


@pytest.mark.parametrize("norm", [0, 1])
def test_radial_return(norm):
    rng = np.random.default_rng(3)
    for _ in range(20):
        S = rng.normal(size=5) * 1e8
        T = _full(S)
        J2 = 0.5 * np.trace(T @ T)
        Y = 0.3 * math.sqrt(J2)
        out, f = oracle.radial_return(S, Y, norm)
        To = _full(out)
        J2o = 0.5 * np.trace(To @ To)
        if norm == 0:
            assert math.sqrt(J2o) == pytest.approx(Y, rel=1e-13)
        else:
            assert J2o == pytest.approx(Y * Y / 3.0, rel=1e-13)     # J2 = Y^2 / 3
        assert np.allclose(out, f * S, rtol=1e-15, atol=0)
        # below yield: identity
        same, f1 = oracle.radial_return(S, 10 * math.sqrt(J2), norm)
        assert f1 == 1.0 and np.array_equal(same, S)


# ----------------------------------------------------------- stress rate ---
def _spin(w):
    """G for v = w x r: G_ab = dv_a / dx_b = -eps_abc w_c."""
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], dtype=float)


def _rk4(S0, G, Gm, jaumann, T, nstep):
    S = np.array(S0, float)
    h = T / nstep
    f = lambda s: oracle.stress_rate(s, G, Gm, jaumann)
    for _ in range(nstep):
        k1 = f(S); k2 = f(S + 0.5 * h * k1); k3 = f(S + 0.5 * h * k2); k4 = f(S + h * k3)
        S = S + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return S


@pytest.mark.parametrize("jaumann", [0, 1])
def test_jaumann_pure_spin_closed_form(jaumann):
    """Rigid spin: edot = 0. The objective rate co-rotates S with the body,
    S(t) = Q S0 Q^T; the printed component form gives Q^T S0 Q."""
    w = np.array([0.3, -0.5, 0.8])
    G = _spin(w)
    S0 = np.array([1.0, -0.4, 0.3, 0.2, -0.7]) * 1e7
    T = 1.1
    S = _rk4(S0, G, 5e9, jaumann, T, 400)
    Q = linalg.expm(G * T)          # dQ/dt = G Q for v = G x
    target = Q @ _full(S0) @ Q.T if jaumann == 0 else Q.T @ _full(S0) @ Q
    assert np.allclose(_full(S), target, rtol=0, atol=1e-9 * 1e7)
    other = Q.T @ _full(S0) @ Q if jaumann == 0 else Q @ _full(S0) @ Q.T
    assert not np.allclose(_full(S), other, rtol=0, atol=1e-3 * 1e7)


def test_stress_rate_pure_strain():
    """Symmetric G (no rotation): Sdot = 2 Gamma (edot - tr(edot) / 3 I)."""
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3))
    G = 0.5 * (A + A.T)
    Gm = 3e9
    S = rng.normal(size=5) * 1e7
    for j in (0, 1):
        dS = oracle.stress_rate(S, G, Gm, j)
        dev = G - np.trace(G) / 3 * np.eye(3)
        ref = 2 * Gm * dev
        assert np.allclose(dS, [ref[0, 0], ref[1, 1], ref[0, 1], ref[0, 2], ref[1, 2]],
                           rtol=1e-13, atol=1e-6)


def test_stress_rate_forms_differ_only_in_rotation_sign():
    """The component form (Eq. 25-29) equals Eq. 13 read as S R - R S; the
    objective form is R S - S R: the two rotation parts are opposite."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        G = rng.normal(size=(3, 3))
        S = rng.normal(size=5)
        Gm = 0.7
        a = oracle.stress_rate(S, G, Gm, 0)
        b = oracle.stress_rate(S, G, Gm, 1)
        E = 0.5 * (G + G.T)
        dev = 2 * Gm * (E - np.trace(E) / 3 * np.eye(3))
        d5 = np.array([dev[0, 0], dev[1, 1], dev[0, 1], dev[0, 2], dev[1, 2]])
        assert np.allclose(a - d5, -(b - d5), rtol=0, atol=1e-13)
        R = 0.5 * (G - G.T)
        T = _full(S)
        rot = R @ T - T @ R
        assert np.allclose(a - d5, [rot[0, 0], rot[1, 1], rot[0, 1], rot[0, 2], rot[1, 2]],
                           atol=1e-13)


# ---------------------------------------------------------- 3x3 inverse ---
def test_inv3_matches_numpy():
    rng = np.random.default_rng(2)
    for _ in range(20):
        A = rng.normal(size=(3, 3)) + 2 * np.eye(3)
        inv, det = oracle.inv3(A)
        assert np.allclose(inv, np.linalg.inv(A), rtol=1e-12, atol=1e-12)
        assert det == pytest.approx(np.linalg.det(A), rel=1e-12)


# --------------------------------------------------------- external field ---
def test_radial_table_lookup():
    w = wl.basalt_sphere(20000)
    p = w.params
    r_k = p["g_rmin"] * (p["g_rmax"] / p["g_rmin"]) ** (np.arange(4096) / 4095)
    c = np.array(p["g_center"])
    rng = np.random.default_rng(0)
    for r in rng.uniform(p["g_rmin"] * 1.001, p["g_rmax"] * 0.999, 50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        g = oracle.gravity(p, *(c + r * d))
        gm = np.interp(r, r_k, p["g_table"])
        assert np.allclose(g, -gm * d, rtol=1e-9, atol=1e-15)
        assert oracle.potential(p, *(c + r * d)) == pytest.approx(
            np.interp(r, r_k, p["phi_table"]), rel=1e-9)
    # outside the table: point mass
    r = 3 * p["g_rmax"]
    g = oracle.gravity(p, *(c + np.array([r, 0, 0])))
    assert g[0] == pytest.approx(-p["g_gm"] / r ** 2, rel=1e-14)
    u = oracle.gravity(dict(p, gravity=1, g_uniform=(0, 0, -9.81)), 1.0, 2.0, 3.0)
    assert np.array_equal(u, [0, 0, -9.81])
