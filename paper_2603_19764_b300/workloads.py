"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds particle sets only: lattices, jitter, seeded velocities
and stresses, material constants and the external-field table. It holds none
of the SPH method's arithmetic, and both the CUDA path and the CPU oracle
take their inputs from it.

The paper (§3-§4) runs M-ANEOS bodies, a granular cliff and Q_RD* impact
series whose initial conditions are not public; the stand-ins here are:

* ``granular_column`` -- a 16x8x32 column of granular material on three
  layers of fixed floor particles (the cliff-collapse set-up of §3.1 at
  laboratory scale, linear EOS, Drucker-Prager friction);
* ``basalt_sphere`` -- a jittered simple-cubic lattice sphere of Tillotson
  basalt with seeded Gaussian velocities and deviatoric stresses;
* ``impact`` -- a basalt target and impactor at 45 degrees (the oblique
  impacts of §3.2-§3.4);
* ``impact_batch`` -- many independent impacts of uneven size, the shape of
  a Q_RD* bisection series (§3.2, Appendix tables).

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014), uniform
doubles from its top 53 bits and normals by Box-Muller.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20260319
G_NEWTON = 6.674e-11

# --------------------------------------------------------------------------
# SplitMix64 counter-based stream
# --------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64: output k is mix(seed + (k + 1) * golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def next_u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.seed + k * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return sigma * out[:n]


# --------------------------------------------------------------------------
# Materials and run-time parameters (plain dicts mirroring the C structs)
# --------------------------------------------------------------------------
EOS_LINEAR = 0
EOS_TILLOTSON = 1


def granular_material() -> dict:
    """Cohesionless granular medium: linear EOS without tension, Y = tan(30 deg) P."""
    mu = math.tan(math.radians(30.0))
    return dict(eos=EOS_LINEAR, rho0=1600.0, c0=100.0, A=1600.0 * 100.0 ** 2, B=0.0,
                E0=1.0, a=0.0, b=0.0, alpha=0.0, beta=0.0, Eiv=0.0, Ecv=1.0,
                shear_G=5.0e6, Y0=0.0, mu_i=mu, Ym=math.inf, mu_d=mu,
                thermal_softening=0, xi=0.0, Tm=0.0, T0=293.0, cv=790.0, strength=1,
                p_min=0.0)


def basalt_material() -> dict:
    """Tillotson basalt with pressure-dependent strength and softening."""
    return dict(eos=EOS_TILLOTSON, rho0=2700.0, c0=0.0, A=26.7e9, B=26.7e9,
                E0=487.0e6, a=0.5, b=1.5, alpha=5.0, beta=5.0, Eiv=4.72e6, Ecv=18.2e6,
                shear_G=22.7e9, Y0=10.0e6, mu_i=1.5, Ym=3.5e9, mu_d=0.6,
                thermal_softening=1, xi=1.2, Tm=1373.0, T0=293.0, cv=790.0, strength=1,
                p_min=-math.inf)


def default_params(precision: int = 0) -> dict:
    """Run-time parameters; tolerance depends on the precision form."""
    return dict(n_ngb=64, av_alpha=1.0, av_beta=2.0, av_eps=0.01, eta_c=0.3, eta_a=0.3,
                h_tol=1e-10 if precision == 0 else 1e-6, max_sweeps=32, h_cap_factor=4.0,
                precision=precision, jaumann=0, yield_norm=0, correction_tensor=1,
                gradient_form=0, max_rung=0,
                gravity=0, g_uniform=(0.0, 0.0, 0.0), g_table=None, phi_table=None,
                g_rmin=1.0, g_rmax=2.0, g_center=(0.0, 0.0, 0.0), g_gm=0.0,
                periodic=0, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0))


FIELDS_F64 = ("x", "y", "z", "vx", "vy", "vz", "u", "m", "h",
              "sxx", "syy", "sxy", "sxz", "syz",
              "rho", "omega", "pres", "cs",
              "ax", "ay", "az", "dudt", "dsxx", "dsyy", "dsxy", "dsxz", "dsyz", "eps_ii")
FIELDS_I32 = ("nngb", "mat", "flags")
FIELDS_I64 = ("id",)


@dataclasses.dataclass
class Workload:
    """A particle set with its materials, parameters and fixed time step."""

    name: str
    arrays: dict
    materials: list
    params: dict
    dt: float
    systems: list | None = None   # (offset, count) per independent system
    dts: list | None = None       # fixed step of each system

    @property
    def n(self) -> int:
        return int(self.arrays["x"].shape[0])

    def copy(self) -> "Workload":
        return Workload(self.name, {k: v.copy() for k, v in self.arrays.items()},
                        [dict(m) for m in self.materials], dict(self.params), self.dt,
                        None if self.systems is None else list(self.systems),
                        None if self.dts is None else list(self.dts))

    def system(self, k: int) -> "Workload":
        """System k of a batch on its own, ids renumbered from 0."""
        off, cnt = self.systems[k]
        a = {key: v[off:off + cnt].copy() for key, v in self.arrays.items()}
        a["id"] = a["id"] - off
        return Workload("%s_sys%d" % (self.name, k), a, [dict(m) for m in self.materials],
                        dict(self.params), self.dts[k] if self.dts else self.dt)


def _empty_arrays(n: int) -> dict:
    a = {k: np.zeros(n, np.float64) for k in FIELDS_F64}
    a.update({k: np.zeros(n, np.int32) for k in FIELDS_I32})
    a["id"] = np.arange(n, dtype=np.int64)
    return a


def lattice_h(mat: dict, m: np.ndarray, n_ngb: int = 64) -> np.ndarray:
    """Support radius holding n_ngb masses in a medium at rho0 (first guess)."""
    return np.cbrt(3.0 * n_ngb * m / (4.0 * np.pi * mat["rho0"]))


def longitudinal_speed(mat: dict) -> float:
    c = mat["c0"] if mat["eos"] == EOS_LINEAR else math.sqrt(mat["A"] / mat["rho0"])
    return math.sqrt(c * c + 4.0 / 3.0 * mat["shear_G"] / mat["rho0"])


# --------------------------------------------------------------------------
# Geometry helpers
# --------------------------------------------------------------------------
def lattice_sphere(n: int, spacing: float) -> np.ndarray:
    """The n simple-cubic lattice points nearest the origin (ties by index)."""
    side = int(math.ceil((6.0 * n / math.pi) ** (1.0 / 3.0))) + 4
    k = np.arange(side, dtype=np.float64) - (side - 1) / 2.0
    gz, gy, gx = np.meshgrid(k, k, k, indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1) * spacing
    r2 = np.einsum("ij,ij->i", pts, pts)
    order = np.argsort(r2, kind="stable")[:n]
    return pts[order]


def radial_field_table(pos: np.ndarray, m: np.ndarray, nbins: int = 4096,
                       rmin: float | None = None) -> dict:
    """Given radial field about the centre of mass, built once at t = 0.

    g(r_k) = G M(<r_k) / r_k^2 and Phi(r_k) on log-spaced r_k, with
    Phi(r_max) = -G M / r_max and Phi integrated inward by the trapezoid
    rule. Self-gravity is outside the SPH step; this table is an input.
    """
    com = (pos * m[:, None]).sum(0) / m.sum()
    r = np.sqrt(((pos - com) ** 2).sum(1))
    order = np.argsort(r, kind="stable")
    rs, cm = r[order], np.cumsum(m[order])
    rmax = float(rs[-1]) * 1.0001 + 1e-9
    if rmin is None:
        rmin = max(rmax * 1e-3, 1e-9)
    rk = rmin * (rmax / rmin) ** (np.arange(nbins) / (nbins - 1))
    idx = np.searchsorted(rs, rk, side="left")
    menc = np.where(idx > 0, cm[np.maximum(idx - 1, 0)], 0.0)
    g = G_NEWTON * menc / rk ** 2
    phi = np.empty(nbins)
    gm = G_NEWTON * float(m.sum())
    phi[-1] = -gm / rk[-1]
    for k in range(nbins - 2, -1, -1):
        phi[k] = phi[k + 1] - 0.5 * (g[k] + g[k + 1]) * (rk[k + 1] - rk[k])
    return dict(gravity=2, g_table=g, phi_table=phi, g_rmin=float(rmin), g_rmax=rmax,
                g_center=tuple(float(c) for c in com), g_gm=gm)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def granular_column(seed: int = BASE_SEED + 1, nx: int = 16, ny: int = 8, nz: int = 32,
                    spacing: float = 0.0125, floor_layers: int = 3, margin: int = 3,
                    precision: int = 0) -> Workload:
    """Granular column on a fixed floor, uniform gravity, particles at rest."""
    rng = SplitMix64(seed)
    mat = granular_material()
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    col = np.stack([(ix.ravel() + 0.5), (iy.ravel() + 0.5), (iz.ravel() + 0.5)], 1) * spacing
    fx, fy, fz = np.meshgrid(np.arange(-margin, nx + margin), np.arange(-margin, ny + margin),
                             np.arange(floor_layers), indexing="ij")
    flo = np.stack([fx.ravel() + 0.5, fy.ravel() + 0.5, -(fz.ravel() + 0.5)], 1) * spacing
    pos = np.concatenate([col, flo])
    n = pos.shape[0]
    pos = pos + rng.uniform(3 * n, -0.01 * spacing, 0.01 * spacing).reshape(n, 3)
    a = _empty_arrays(n)
    a["x"], a["y"], a["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    a["m"][:] = mat["rho0"] * spacing ** 3
    a["h"][:] = lattice_h(mat, a["m"])
    a["flags"][col.shape[0]:] = 1
    p = default_params(precision)
    p.update(gravity=1, g_uniform=(0.0, 0.0, -9.81))
    return Workload("granular_column_%d" % n, a, [mat], p, _dt_for(mat, float(a["h"][0]), 0.0))


def _body(rng: SplitMix64, n: int, spacing: float, mat: dict, v_sigma: float,
          s_sigma: float) -> dict:
    pos = lattice_sphere(n, spacing)
    pos = pos + rng.uniform(3 * n, -0.01 * spacing, 0.01 * spacing).reshape(n, 3)
    a = _empty_arrays(n)
    a["x"], a["y"], a["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    a["m"][:] = mat["rho0"] * spacing ** 3
    a["h"][:] = lattice_h(mat, a["m"])
    v = rng.normal(3 * n, v_sigma).reshape(n, 3)
    a["vx"], a["vy"], a["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    s = rng.normal(5 * n, s_sigma).reshape(n, 5)
    for k, f in enumerate(("sxx", "syy", "sxy", "sxz", "syz")):
        a[f] = s[:, k].copy()
    return a


def _concat(parts: list) -> dict:
    out = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    out["id"] = np.arange(out["x"].shape[0], dtype=np.int64)
    return out


def _dt_for(mat: dict, h: float, v_bulk: float) -> float:
    """Fixed step under the CFL form of Eq. 39 (eta_C = 0.3, alpha = 1, beta = 2)."""
    return 0.3 * h / (1.6 * longitudinal_speed(mat) + 1.2 * v_bulk)


def basalt_sphere(n: int = 1_000_000, radius: float = 10.0e3, seed: int = BASE_SEED + 2,
                  precision: int = 0) -> Workload:
    """Jittered lattice sphere of Tillotson basalt, seeded v and S, radial g."""
    rng = SplitMix64(seed)
    mat = basalt_material()
    spacing = (4.0 * math.pi * radius ** 3 / 3.0 / n) ** (1.0 / 3.0)
    a = _body(rng, n, spacing, mat, 10.0, 1.0e6)
    p = default_params(precision)
    pos = np.stack([a["x"], a["y"], a["z"]], 1)
    p.update(radial_field_table(pos, a["m"]))
    return Workload("basalt_sphere_%d" % n, a, [mat], p, _dt_for(mat, float(a["h"][0]), 50.0))


def impact(n_target: int = 1_800_000, n_imp: int = 200_000, radius: float = 10.0e3,
           v_imp: float = 5.0e3, angle_deg: float = 45.0, seed: int = BASE_SEED + 3,
           precision: int = 0, spacing: float | None = None) -> Workload:
    """Basalt target and impactor at the same lattice spacing, in the COM frame.

    The impactor centre starts at 1.02 (R_t + R_i) from the target centre,
    the line of centres at angle_deg to the impact velocity.
    """
    rng = SplitMix64(seed)
    mat = basalt_material()
    if spacing is None:
        spacing = (4.0 * math.pi * radius ** 3 / 3.0 / n_target) ** (1.0 / 3.0)
    tgt = _body(rng, n_target, spacing, mat, 10.0, 1.0e6)
    imp = _body(rng, n_imp, spacing, mat, 10.0, 1.0e6)
    r_t = (3.0 * n_target / (4.0 * math.pi)) ** (1.0 / 3.0) * spacing
    r_i = (3.0 * n_imp / (4.0 * math.pi)) ** (1.0 / 3.0) * spacing
    d = 1.02 * (r_t + r_i)
    th = math.radians(angle_deg)
    imp["x"] += d * math.cos(th)
    imp["y"] += d * math.sin(th)
    imp["vx"] += -v_imp
    a = _concat([tgt, imp])
    mtot = a["m"].sum()
    for c in ("x", "y", "z", "vx", "vy", "vz"):
        a[c] -= (a["m"] * a[c]).sum() / mtot
    p = default_params(precision)
    pos = np.stack([a["x"], a["y"], a["z"]], 1)
    p.update(radial_field_table(pos, a["m"]))
    n = n_target + n_imp
    return Workload("impact_%d" % n, a, [mat], p, _dt_for(mat, float(a["h"][0]), v_imp),
                    systems=[(0, n)])


def impact_batch(n_systems: int = 64, seed: int = BASE_SEED + 4, spacing: float = 161.2,
                 nt_range: tuple = (2.0e3, 2.0e5), precision: int = 0,
                 scale: float = 1.0) -> Workload:
    """Independent impacts of uneven size (a Q_RD*-style series).

    Per system: N_t log-uniform in nt_range (times scale), mass ratio gamma
    uniform in [0.01, 0.5], N_i = max(341, round(gamma N_t)), speed uniform
    in [1, 20] km/s, angle uniform in [0, 60] degrees. Systems are placed
    far apart along x so that no pair of particles from different systems
    is ever within a kernel radius. Each system keeps its own fixed step
    (dts); dt is the smallest of them.
    """
    rng = SplitMix64(seed)
    lo, hi = math.log(nt_range[0] * scale), math.log(nt_range[1] * scale)
    nts = np.rint(np.exp(rng.uniform(n_systems, lo, hi))).astype(np.int64)
    gam = rng.uniform(n_systems, 0.01, 0.5)
    vel = rng.uniform(n_systems, 1.0e3, 20.0e3)
    ang = rng.uniform(n_systems, 0.0, 60.0)
    parts, systems, off, x0 = [], [], 0, 0.0
    dts = []
    for s in range(n_systems):
        nt = int(nts[s])
        ni = max(int(round(341 * scale)) if scale < 1 else 341, int(round(gam[s] * nt)))
        w = impact(nt, ni, v_imp=float(vel[s]), angle_deg=float(ang[s]),
                   seed=seed * 1000 + s, precision=precision, spacing=spacing)
        a = w.arrays
        ext = float(a["x"].max() - a["x"].min())
        shift = x0 - float(a["x"].min())
        a["x"] += shift
        x0 += ext + 20.0 * spacing
        parts.append(a)
        systems.append((off, w.n))
        off += w.n
        dts.append(w.dt)
    arr = _concat(parts)
    p = default_params(precision)
    return Workload("impact_batch_%d" % n_systems, arr, [basalt_material()], p, min(dts),
                    systems=systems, dts=dts)


def periodic_wave_box(nx: int = 64, ny: int = 8, nz: int = 8, spacing: float = 1.0,
                      amp: float = 1.0e-3, precision: int = 0) -> Workload:
    """Perfect lattice in a periodic box with v_x = amp sin(2 pi x / L_x).

    Linear EOS, constant shear modulus, no yield, no viscosity: a
    longitudinal standing wave that must travel at sqrt((K + 4/3 G) / rho).
    """
    mat = dict(eos=EOS_LINEAR, rho0=1000.0, c0=100.0, A=1000.0 * 100.0 ** 2, B=0.0, E0=1.0,
               a=0.0, b=0.0, alpha=0.0, beta=0.0, Eiv=0.0, Ecv=1.0, shear_G=3.0e6, Y0=1e30,
               mu_i=0.0, Ym=math.inf, mu_d=1e30, thermal_softening=0, xi=0.0, Tm=0.0,
               T0=293.0, cv=790.0, strength=1, p_min=-math.inf)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    n = nx * ny * nz
    a = _empty_arrays(n)
    a["x"] = (ix.ravel() + 0.5) * spacing
    a["y"] = (iy.ravel() + 0.5) * spacing
    a["z"] = (iz.ravel() + 0.5) * spacing
    a["m"][:] = mat["rho0"] * spacing ** 3
    a["h"][:] = lattice_h(mat, a["m"])
    lx = nx * spacing
    a["vx"] = amp * np.sin(2.0 * np.pi * a["x"] / lx)
    p = default_params(precision)
    p.update(av_alpha=0.0, av_beta=0.0, periodic=1, box_lo=(0.0, 0.0, 0.0),
             box_hi=(lx, ny * spacing, nz * spacing))
    dt = 0.2 * float(a["h"][0]) / longitudinal_speed(mat)
    return Workload("wave_box_%d" % n, a, [mat], p, dt)


def elastic_material() -> dict:
    """Linear EOS with a constant shear modulus and no yield (elastic)."""
    return dict(eos=EOS_LINEAR, rho0=1000.0, c0=100.0, A=1000.0 * 100.0 ** 2, B=0.0, E0=1.0,
                a=0.0, b=0.0, alpha=0.0, beta=0.0, Eiv=0.0, Ecv=1.0, shear_G=3.0e6, Y0=1e30,
                mu_i=0.0, Ym=math.inf, mu_d=1e30, thermal_softening=0, xi=0.0, Tm=0.0,
                T0=293.0, cv=790.0, strength=1, p_min=-math.inf)


def spinning_sphere(n: int = 4000, spacing: float = 1.0, surface_speed: float = 0.5,
                    seed: int = BASE_SEED + 6, precision: int = 0,
                    correction: int = 1) -> Workload:
    """Elastic lattice sphere in rigid rotation about z (the angular-momentum
    check of the correction tensor): v = omega x r with the equator moving
    at surface_speed, +-1 % jitter, no gravity. The EOS carries no tension
    and is soft (c0 = 10 m/s), so the free surface neither pulls the body
    apart nor pushes it out much, while the shear modulus makes any
    spurious strain rate of the rotation build deviatoric stress."""
    rng = SplitMix64(seed)
    mat = elastic_material()
    mat.update(c0=10.0, A=1000.0 * 10.0 ** 2, p_min=0.0)
    pos = lattice_sphere(n, spacing)
    pos = pos + rng.uniform(3 * n, -0.01 * spacing, 0.01 * spacing).reshape(n, 3)
    a = _empty_arrays(n)
    a["x"], a["y"], a["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    a["m"][:] = mat["rho0"] * spacing ** 3
    a["h"][:] = lattice_h(mat, a["m"])
    radius = float(np.sqrt((pos[:, :2] ** 2).sum(1)).max())
    om = surface_speed / radius
    a["vx"] = -om * a["y"]
    a["vy"] = om * a["x"]
    p = default_params(precision)
    p.update(correction_tensor=correction)
    dt = 0.2 * float(a["h"][0]) / longitudinal_speed(mat)
    return Workload("spinning_sphere_%d" % n, a, [mat], p, dt)


def config(index: int, precision: int | None = None, scale: float = 1.0) -> Workload:
    """The five benchmark configurations (index 1..5); scale < 1 shrinks N.

    1 granular column (4096 + 924 fixed), 2 basalt sphere (1M),
    3 impact (1.8M + 0.2M), 4 64 impacts (about 3.5M in total),
    5 impact (7.2M + 0.8M).
    """
    if index == 1:
        return granular_column(precision=0 if precision is None else precision)
    if index == 2:
        return basalt_sphere(int(1_000_000 * scale), precision=0 if precision is None else precision)
    if index == 3:
        return impact(int(1_800_000 * scale), int(200_000 * scale),
                      precision=1 if precision is None else precision)
    if index == 4:
        return impact_batch(64, precision=0 if precision is None else precision, scale=scale)
    if index == 5:
        return impact(int(7_200_000 * scale), int(800_000 * scale),
                      precision=1 if precision is None else precision)
    raise ValueError("config index must be 1..5")


# --------------------------------------------------------------------------
# Initial weights of the smoothing-length network (6-64-64-1)
# --------------------------------------------------------------------------
MLP_NIN, MLP_NHID = 6, 64
MLP_NPARAM = MLP_NHID * MLP_NIN + MLP_NHID + MLP_NHID * MLP_NHID + MLP_NHID + MLP_NHID + 1


def mlp_init(seed: int = BASE_SEED + 7) -> np.ndarray:
    """Seeded initial parameter vector: weights uniform in +-sqrt(6 / (fan_in
    + fan_out)) (Glorot and Bengio 2010), biases zero. Order: W1[64][6], b1,
    W2[64][64], b2, W3[64], b3."""
    rng = SplitMix64(seed)

    def glorot(fan_out, fan_in):
        a = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(fan_out * fan_in, -a, a)

    nh, ni = MLP_NHID, MLP_NIN
    theta = np.concatenate([glorot(nh, ni), np.zeros(nh), glorot(nh, nh), np.zeros(nh),
                            glorot(1, nh), np.zeros(1)])
    assert theta.shape[0] == MLP_NPARAM
    return theta
