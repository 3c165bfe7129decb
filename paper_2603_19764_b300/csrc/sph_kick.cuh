// sph_kick.cuh -- the per-particle closing kick, radial return and opening
// kick of §2.4 (Eq. 40-43), with the particle's terms of the step's FP64
// sums (Eq. 46) and of the time-step minimum (Eq. 38-39). Shared by the
// kick kernel and by the force pass, whose epilogue kicks each particle
// of a global step as soon as its derivatives are formed.
#pragma once

#include "sph_internal.cuh"

namespace sphk {

constexpr int kNSum = 9;   // e_kin (doubled), e_int, e_pot, p[3], L[3]
// Slots of the step's reductions: the nine sums, then the time-step
// minimum of Eq. 38-39
constexpr int kSlotDt = kNSum, kNSlot = kNSum + 1;
// Reduction tiles: 64 buckets (2048 sorted positions) of one system
constexpr int kRedTile = 64;

// Derivatives of particle i at time i, as the force pass wrote them (FP64
// values; the FP32 form's are exact widenings of FP32 results).
struct KickIn {
  double a[3], dudt, dS[5];
  double edot2;   // 1/2 edot:edot
  double vsig;    // CFL signal speed of Eq. 39
};

// Time-step criterion of a moving particle, min(Eq. 38 with eps = H, Eq.
// 39), in the form's arithmetic type: from its acceleration, its H and the
// CFL signal speed of the force pass.
template <typename T>
__device__ __forceinline__ T crit_t(const KParams &P, const double a[3], double h, double vsig) {
  const T eta_a = to_t<T>(P.eta_a), eta_c = to_t<T>(P.eta_c);
  const T H = to_t<T>(h);
  const T ax = to_t<T>(a[0]), ay = to_t<T>(a[1]), az = to_t<T>(a[2]);
  const T am = root(ax * ax + ay * ay + az * az);
  const T ta = am > T(0) ? eta_a * root(quot(H, am)) : T(INFINITY);   // Eq. 38, eps = H
  const T tc = quot(eta_c * H, to_t<T>(vsig));                        // Eq. 39
  return tmin_(ta, tc);
}

// Particle i of system sy: with kick, moving particles whose own step ends
// with this substep are closed to i (v, u, S alike), S is rescaled with Y
// at (rho_i, u_i), the strain invariant gains dt 1/2 edot:edot and the
// state is opened to i + 1/2; the others are copied from the read view when
// copy is set. Returns the particle's terms of the step's sums (at time i;
// e_kin doubled) in term[] and its time-step criterion in *tcr (infinite
// for a fixed particle). sub: length of the substep (the step without
// rungs); last: every particle's step ends with this substep.
template <typename T>
__device__ __forceinline__ void kick_particle(const sph_state &s, const sph_state &src,
                                              const Work &w, const KParams &P, int64_t i,
                                              bool kick, double sub, bool last, bool copy,
                                              const KickIn &d, double term[kNSum], double *tcr,
                                              int &updates, int *hist) {
  const bool fixed = s.flags[i] & SPH_FLAG_FIXED;
  const double m = s.m[i];
  const double *a = d.a;
  double v[3] = {src.vx[i], src.vy[i], src.vz[i]};
  double u = src.u[i];
  if (kick && !fixed && rung_active(P, i)) {
    // the particle's own step (no conversion on the FP64 unit without rungs)
    const double dt = P.max_rung ? sub * (double)rung_len(P, i) : sub, hdt = 0.5 * dt;
    const MatT<T> &M = mat_t<T>(P, s.mat[i]);
    double S[5] = {src.sxx[i], src.syy[i], src.sxy[i], src.sxz[i], src.syz[i]};
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] += hdt * a[k];
    u += hdt * d.dudt;
#pragma unroll
    for (int k = 0; k < 5; ++k) S[k] += hdt * d.dS[k];
    if (M.strength) {
      const EosT<T> e = eos_t<T>(M, s.rho[i], u);
      const T St[5] = {to_t<T>(S[0]), to_t<T>(S[1]), to_t<T>(S[2]), to_t<T>(S[3]), to_t<T>(S[4])};
      const T ft = radial_factor_t<T>(St, yield_t<T>(M, e.P, to_t<T>(u)), P.yield_norm);
      if (ft < T(1)) {   // below the yield surface f is exactly 1
        const double f = from_t(ft);
#pragma unroll
        for (int k = 0; k < 5; ++k) S[k] *= f;
      }
    } else {
      S[0] = S[1] = S[2] = S[3] = S[4] = 0.0;
    }
    s.eps_ii[i] = src.eps_ii[i] + dt * d.edot2;
    // opening kick from the state at i; with rungs over the next step of
    // the rung the criteria ask for, no coarser than the coarsest rung
    // whose steps start at the next substep
    double ho = hdt;
    if (P.max_rung) {
      // the rung from the criterion in the form's type (the FP32 form's FP64
      // square roots and divisions here cost the kick a third of its time)
      int r = rung_want(P, sub, from_t(crit_t<T>(P, a, s.h[i], d.vsig)));
      int r_al = P.max_rung;
      for (int q = P.substep + 1; r_al > 0 && (q & 1) == 0; q >>= 1) --r_al;
      r = r > r_al ? r : r_al;
      w.rung[i] = r;
      ho = 0.5 * sub * (double)(1 << (P.max_rung - r));
      if (last) atomicAdd(&hist[r], 1);
    }
    ++updates;
    s.vx[i] = v[0] + ho * a[0];
    s.vy[i] = v[1] + ho * a[1];
    s.vz[i] = v[2] + ho * a[2];
    s.u[i] = u + ho * d.dudt;
    s.sxx[i] = S[0] + ho * d.dS[0];
    s.syy[i] = S[1] + ho * d.dS[1];
    s.sxy[i] = S[2] + ho * d.dS[2];
    s.sxz[i] = S[3] + ho * d.dS[3];
    s.syz[i] = S[4] + ho * d.dS[4];
  } else if (copy) {   // not kicked: the state as read
    s.vx[i] = v[0];
    s.vy[i] = v[1];
    s.vz[i] = v[2];
    s.u[i] = u;
    s.sxx[i] = src.sxx[i];
    s.syy[i] = src.syy[i];
    s.sxy[i] = src.sxy[i];
    s.sxz[i] = src.sxz[i];
    s.syz[i] = src.syz[i];
    s.eps_ii[i] = src.eps_ii[i];
  }
  const double x = s.x[i], y = s.y[i], z = s.z[i];
  T g[3], phi;
  ext_field_t<T>(P, x, y, z, g, &phi);
  // momentum first; kinetic energy (doubled, halved when summed) and
  // angular momentum from it
  term[3] = m * v[0];
  term[4] = m * v[1];
  term[5] = m * v[2];
  term[0] = v[0] * term[3] + v[1] * term[4] + v[2] * term[5];
  term[1] = m * u;
  term[2] = m * from_t(phi);
  term[6] = y * term[5] - z * term[4];
  term[7] = z * term[3] - x * term[5];
  term[8] = x * term[4] - y * term[3];
  *tcr = fixed ? double(INFINITY) : from_t(crit_t<T>(P, a, s.h[i], d.vsig));
}

// The smaller of two time-step criteria: non-negative doubles or +inf,
// whose bit patterns order like their values (integer compare, no FP64
// instruction).
__device__ __forceinline__ double min_crit(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ia < ib ? a : b;
}

}  // namespace sphk
