// sph_internal.cuh -- device-side types and functions shared by the CUDA
// translation units of libsph. Not part of the public ABI (include/sph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "sph.h"

namespace sphk {

constexpr int kWarpsPerBlock = 4;      // pair kernels: one warp per bucket
constexpr int kBlock = 256;            // per-particle kernels
constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846;

// Wendland C2 in 3-D with support H (§3; Dehnen & Aly 2012):
//   W      = cW / H^3 (1-q)^4 (1+4q)
//   W'/r   = cG / H^5 (1-q)^3                 (radial derivative over r)
//   dW/dH  = cW / H^4 (1-q)^3 (-3 - 9q + 32q^2)
constexpr double cW = 21.0 / (2.0 * kPi);
constexpr double cG = -210.0 / kPi;

enum : unsigned {
  ERR_NOCONV = 1u,
  ERR_NONFINITE = 2u,
  ERR_CAPACITY = 4u,
  ERR_TIMEOUT = 8u,
  ERR_BOUNDS = 16u   // checked builds: an index check failed
};

// Checked builds (-DSPH_BOUNDS_CHECK): every index that comes from data
// (cell ranges, sort positions, candidate lists, the active list) is tested
// before its access. A failed test latches ERR_BOUNDS in the status word
// and the access goes to index 0 instead -- never a trap -- and the
// synchronising call reports SPH_E_INTERNAL. Release builds compile the
// tests out: checked(i, n, err) is i.
__device__ __forceinline__ int64_t checked(int64_t i, int64_t n, unsigned *err) {
#ifdef SPH_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    atomicOr(err, ERR_BOUNDS);
    return 0;
  }
#else
  (void)n;
  (void)err;
#endif
  return i;
}

// Uniform cell grid of one system for one step, written on the device by
// k_grid_setup. Global cell index = cell_off + (z * dims[1] + y) * dims[0] + x.
struct Grid {
  double lo[3];
  double L;          // cell edge
  double invL;       // 1 / L, and both rounded to FP32: formed once per step,
  float Lf, invLf;   // since FP64 division and conversion run on the FP64 unit
  int dims[3];
  int ncells;
  int cell_off;
};
template <typename T> __device__ __forceinline__ T grid_L(const Grid &g);
template <> __device__ __forceinline__ float grid_L<float>(const Grid &g) { return g.Lf; }
template <> __device__ __forceinline__ double grid_L<double>(const Grid &g) { return g.L; }
template <typename T> __device__ __forceinline__ T grid_invL(const Grid &g);
template <> __device__ __forceinline__ float grid_invL<float>(const Grid &g) { return g.invLf; }
template <> __device__ __forceinline__ double grid_invL<double>(const Grid &g) { return g.invL; }


// One independent particle system of a context (a context holds one system,
// or a batch of them that never interact). Its particles occupy the sorted
// positions [begin, end), which are also its range of caller ids. Encoded
// min/max use the order-preserving map of doubles to unsigned 64-bit
// integers (enc_d / dec_d).
struct SysRec {
  unsigned long long lo_enc[3], hi_enc[3], hmax_enc, hmax2_enc, dtmin_enc;
  unsigned long long disp_enc;   // largest coordinate change of this drift
  Grid grid;
  // staging skin: how far a particle may have moved from the cell it was
  // sorted into (0 right after a sort); a candidate search covers the cells
  // within its radius + skin, its membership tests use current positions
  double skin;
  float skinf;                   // rounded up
  int begin, end;      // sorted positions (= ids) of the system's particles
  int bucket_off;      // first 32-particle bucket of the system
  int cell_cap;        // cells the system may use
  double sums[9];      // e_kin, e_int, e_pot, p[3], L[3]
};

template <typename T> __device__ __forceinline__ T sys_skin(const SysRec &r);
template <> __device__ __forceinline__ float sys_skin<float>(const SysRec &r) { return r.skinf; }
template <> __device__ __forceinline__ double sys_skin<double>(const SysRec &r) { return r.skin; }

// Device-resident step record shared by all systems of a context.
struct Status {
  unsigned int err;
  int max_sweeps, n_unconv, n_capped, n_cfallback;
  int pad_;
  unsigned long long pairs_density, pairs_force;
  unsigned long long cand_density, cand_force;   // staged candidates
  unsigned long long groups_density, groups_force;
  unsigned long long sweeps_total;              // Newton sweeps summed over particles
  int n_expanded;                               // solves closed by the expansion
  int pad3_;
  unsigned next_bucket[2];                      // persistent-warp work counters
  int total_cells;                              // cells of all systems this step
  int pad2_;
  unsigned long long updates;                   // particles kicked in the step
  int rung_hist[16];                            // rungs of the moving particles at its end
  int n_active;                                 // entries of KParams::act this substep
  int key_shift;                                // sort keys: system index << key_shift
  unsigned key_or;                              // OR of this step's sort keys
  int pad5_;
};

// Radix passes of 8 bits that the sort runs for keys whose OR is o: those
// with a nonzero digit at or above their own (a pass whose digit and every
// higher one are zero for all keys would leave the order as it is).
__device__ __forceinline__ int sort_passes(unsigned o) {
  return (o != 0u) + ((o >> 8) != 0u) + ((o >> 16) != 0u) + ((o >> 24) != 0u);
}




// Material parameters in the arithmetic type of a form, with the derived
// constants the evaluations need; the FP32 copies are made once on the host
// so that an evaluation converts nothing. FP64 copies of the values that
// region tests and mu = rho / rho0 - 1 use in FP64.
template <typename T> struct MatT {
  int eos, strength, thermal_softening, pad_;
  double rho0_d, Eiv_d, Ecv_d, c0sq_d, p_min_d;
  T rho0, inv_rho0, c0, c0sq, A, B, E0, a, b, alpha, beta, inv_dE, floor2;
  T shear_G, Y0, mu_i, Ym, mu_d, xi, Tm, T0, inv_cv, p_min;
  // the smoothing-length cap of the density solve: hcap_f (the run's
  // h_cap_factor) times (hcap_k m)^(1/3), hcap_k = 3 n_ngb / (4 pi rho0),
  // both rounded from FP64 once on the host
  T hcap_k, hcap_f;
};

// Kernel-side copy of the run-time parameters.
struct KParams {
  int n_ngb;
  double av_alpha, av_beta, av_eps, eta_c, eta_a, h_tol;
  int max_sweeps;
  double h_cap_factor;
  int precision, jaumann, yield_norm, correction;
  int gravity;
  double g_uniform[3];
  const double *g_table, *phi_table, *g_radii;
  int g_n;
  double g_rmin, g_rmax, g_center[3], g_gm, g_inv_log_ratio;
  // FP32 copies of the field's constants and tables (rounded once on the
  // host), so that the FP32 form's evaluations convert nothing
  const float *g_table_f, *phi_table_f, *g_radii_f;
  float g_rmin_f, g_rmax_f, g_gm_f, g_inv_log_ratio_f, g_uniform_f[3];
  const sph_material *mats;
  const MatT<float> *matf;     // the materials for the FP32 / FP64 forms
  const MatT<double> *matd;
  // systems
  int nsys, axis_bits;         // Morton bits per axis below the system bits
  int nbuckets;
  SysRec *sys;                 // nsys records (device)
  const int *sys_begin;        // nsys + 1 sorted-position boundaries (device)
  const int *sys_bucket;       // nsys + 1 bucket boundaries (device)
  // reduction tiles of the per-bucket partial sums: tile t covers buckets
  // [red_tile[t], red_tile_end[t]) of one system; the tiles of system s are
  // [sys_tile[s], sys_tile[s + 1])
  const int *red_tile, *red_tile_end, *sys_tile;
  int nred_tiles;
  const double *dt;            // current step of every system (device)
  int span_d, span_f;          // group span of the density / force kernels
  // FP32 copies of the constants the FP32 pair loops use, so that a
  // constant the compiler reloads inside a loop needs no FP64 conversion
  float av_alpha_f, av_beta_f, av_eps_f, h_tol_f;
  float lattice_k_f;           // 3 n_ngb / (4 pi): H_bar^3 = lattice_k m / rho0
  // weights of the H_i and H_j terms of Eq. 20-21: -1/2 and -1/2
  // (symmetric), -1 and 0 (one-sided form)
  double grad_wi, grad_wj;
  float grad_wi_f, grad_wj_f;
  const double *h_guess;       // starting radius of the solve (sorted order), or null
  // hierarchical steps: dt[] holds each system's big step; this launch
  // belongs to substep `substep` of 2^max_rung, of length dt * sub_scale
  int max_rung, substep;
  double sub_scale;            // 2^-max_rung (exact)
  const int *rung;             // per particle (sorted order), or null
  // hierarchical steps of one system: the sorted positions of the particles
  // active in the current substep, in sorted order (Status::n_active of
  // them); the pair kernels take their buckets from this list. Null: the
  // buckets are 32 consecutive sorted positions and inactive lanes idle.
  const int *act;
  // periodic box [box_lo, box_hi) on every axis (one system only): drifted
  // positions wrap into it, the cell grid tiles it from box_lo, and pairs
  // take the minimum image
  int periodic;
  double box_lo[3], box_hi[3], box_len[3];
};

// Minimum-image separation along one periodic axis of length `box`, the
// image nearest to d = x_i - x_j (the FP64 arithmetic of the neighbour
// predicate in a periodic box).
__device__ __forceinline__ double min_image(double d, double box) {
  if (d > 0.5 * box) return d - box;
  if (d < -0.5 * box) return d + box;
  return d;
}

// Hierarchical steps: a particle on rung r steps 2^(R - r) substeps and is
// active (solved, given derivatives, kicked) at the end of each of them.
__device__ __forceinline__ int rung_len(const KParams &P, int64_t i) {
  return P.max_rung == 0 ? 1 : 1 << (P.max_rung - P.rung[i]);
}
__device__ __forceinline__ bool rung_active(const KParams &P, int64_t i) {
  return P.max_rung == 0 || ((P.substep + 1) & (rung_len(P, i) - 1)) == 0;
}
// Half-step offset of the predictor at the end of the current substep:
// q(t) = q_half + k dq with k = t - t_mid of the particle's current step
// (dt / 2 of its own step when the step ends there; dt / 2 without rungs).
__device__ __forceinline__ double predict_offset(const KParams &P, int64_t i, double sub_dt) {
  if (P.max_rung == 0) return 0.5 * sub_dt;
  const int len = rung_len(P, i);
  const int start = P.substep & ~(len - 1);
  return ((double)(P.substep + 1 - start) - 0.5 * (double)len) * sub_dt;
}
// The rung a particle's criteria ask for: the smallest r with
// big_dt / 2^r <= crit, at most R (big_dt / 2^r = sub_dt 2^(R - r) exactly).
__device__ __forceinline__ int rung_want(const KParams &P, double sub_dt, double crit) {
  int r = 0;
  while (r < P.max_rung && sub_dt * (double)(1 << (P.max_rung - r)) > crit) ++r;
  return r;
}

// A run-time constant in the pair loops' arithmetic type.
template <typename T> __device__ __forceinline__ T pconst(double d, float f);
template <> __device__ __forceinline__ float pconst<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pconst<double>(double d, float) { return d; }

// Group spans the tuner chooses among.
constexpr int kNumSpans = 3;
constexpr int kSpans[kNumSpans] = {1, 2, 3};
// Staging depths of the FP32 form's pair kernels (chunks of 32 candidate
// positions located and loaded at once; compiled variants), the tuner's
// second knob, and the defaults (the FP64 form runs the defaults only).
constexpr int kNumDepths = 2;
constexpr int kDepths[kNumDepths] = {3, 4};
constexpr int kDepthDensity = 3, kDepthForces = 4;


// System owning a sorted position / an id / a bucket: the last
// boundary not above the value (bounds has nsys + 1 entries).
__device__ __forceinline__ int sys_lookup(const int *bounds, int nsys, int64_t v) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bounds[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Lane `lane` of bucket bk of a pair kernel: its sorted position i (valid
// lanes only), a position safe to read for every lane (ic), and the system.
// From the active list when there is one (n_act entries), else 32
// consecutive positions of the bucket's system.
struct BucketLane {
  int64_t i, ic;
  bool valid;
  int sy;
};
__device__ __forceinline__ int bucket_count(const KParams &P, int n_act) {
  return P.act ? (n_act + 31) >> 5 : P.nbuckets;
}
__device__ __forceinline__ BucketLane bucket_lane(const KParams &P, int n_act, unsigned bk,
                                                  int lane, int64_t n, unsigned *err) {
  BucketLane b;
  if (P.act) {
    const int k = (int)bk * 32 + lane;
    b.valid = k < n_act;
    b.i = checked(P.act[checked(b.valid ? k : (int)bk * 32, n, err)], n, err);
    b.ic = b.i;
    b.sy = 0;
    return b;
  }
  b.sy = P.nsys > 1 ? sys_lookup(P.sys_bucket, P.nsys, bk) : 0;
  const SysRec &R = P.sys[b.sy];
  const int64_t base = R.begin + (int64_t)(bk - R.bucket_off) * 32;
  b.i = base + lane;
  b.valid = b.i < R.end;
  b.ic = b.valid ? b.i : base;
  return b;
}

template <typename T> __device__ __forceinline__ const MatT<T> &mat_t(const KParams &P, int k);
template <> __device__ __forceinline__ const MatT<float> &mat_t<float>(const KParams &P, int k) {
  return P.matf[k & (SPH_MAX_MATERIALS - 1)];
}
template <> __device__ __forceinline__ const MatT<double> &mat_t<double>(const KParams &P, int k) {
  return P.matd[k & (SPH_MAX_MATERIALS - 1)];
}

// FP64 <-> FP32 conversions on the integer pipe. On this part the
// conversion instructions run on the FP64 unit, at 1/64 of the FP32 rate,
// and the per-particle kernels convert tens of values per particle. Built
// from the IEEE 754 binary64 / binary32 layouts: round to nearest even for
// results in the binary32 normal range, and zeros, in integer arithmetic;
// the other cases (subnormal results, overflow to infinity, infinities,
// NaN) call the conversion instruction out of line. (Written inline, that
// call was evaluated for every value by the compiler, which runs both
// sides of a short branch; written in integer arithmetic inline, the rare
// cases took registers from every kernel that converts.)
static __device__ __noinline__ float d2f_rare(double d) { return __double2float_rn(d); }
static __device__ __noinline__ double f2d_rare(float v) { return (double)v; }
__device__ __forceinline__ float d2f(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;   // biased binary64 exponent
  if (e - 897u > 253u) {
    if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi);   // +-0
    return d2f_rare(d);
  }
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 fraction bits
  const unsigned rest = lo & 0x1fffffffu;                    // the 29 dropped bits
  unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
  // a carry out of the fraction raises the exponent (2^128: infinity)
  f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(f);
}
__device__ __forceinline__ double f2d(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u > 253u) {
    if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)u, 0);   // +-0
    return f2d_rare(v);
  }
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
template <typename T> __device__ __forceinline__ T to_t(double d);
template <> __device__ __forceinline__ float to_t<float>(double d) { return d2f(d); }
template <> __device__ __forceinline__ double to_t<double>(double d) { return d; }
__device__ __forceinline__ double from_t(float v) { return f2d(v); }
__device__ __forceinline__ double from_t(double v) { return v; }

// Library-owned per-particle work arrays (sorted order).
struct Work {
  double *vsig, *edot2, *yld;   // CFL signal, 1/2 edot:edot, yield strength
  int *cc;                      // packed cell coordinates x | y << 10 | z << 20
  float4 *pos32;                // cell-relative x, y, z and m (FP32 form)
  double4_32a *pos64;           // absolute x, y, z and m (FP64 form)
  float4 *posh32;               // positions with H (force pass)
  double4_32a *posh64;
  float4 *fj32;                 // force-side neighbour records, 4 vectors per
  double4_32a *fj64;            // particle, contiguous (FP32 / FP64 form)
  float4 *fs32[3];              // own stress, shear modulus, c_L, external g
  double4_32a *fs64[3];
  float *divv;                  // tr of the corrected velocity gradient (learned form)
  double *terms[9];             // each particle's terms of the step's sums (Eq. 46)
  double *tcrit;                // and its time-step criterion (Eq. 38-39)
  int *rung;                    // hierarchical steps: rung of every particle, or null
  int *act;                     // hierarchical steps of one system: active list (n)
  int *act_tiles;               // and its per-tile counts / offsets
};

// Arrays of the learned form. hprev, hprop and feat are per-particle
// arrays in sorted order that the sort permutes with the state; the
// recorded samples are indexed by particle id.
struct LearnArgs {
  int guess, record;
  const float *divv;            // tr G of the last force pass
  double *hprev;                // H of the last solve
  double *hprop;                // starting radius proposed for the next solve
  float2 *feat[3];              // features of the last step (record)
  float *x_out, *y_out;         // samples of the last step, by id (record)
};

// ---------------------------------------------------------------- helpers
// Ask L2 to fetch the line holding p (no register is written).
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned long long enc_d(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double dec_d(unsigned long long e) {
  unsigned long long b = (e & 0x8000000000000000ull) ? (e & 0x7fffffffffffffffull) : ~e;
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}
__host__ inline unsigned long long enc_h(double d) {
  unsigned long long b;
  memcpy(&b, &d, sizeof(b));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T> __device__ __forceinline__ T wmax(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    T w = __shfl_xor_sync(kFull, v, o);
    v = v > w ? v : w;
  }
  return v;
}
template <typename T> __device__ __forceinline__ T wmin(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    T w = __shfl_xor_sync(kFull, v, o);
    v = v < w ? v : w;
  }
  return v;
}
template <typename T> __device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename T> __device__ __forceinline__ T tmax_(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T tmin_(T a, T b) { return a < b ? a : b; }

// Spread the low 10 bits of v to every third bit (Morton interleave).
__host__ __device__ inline unsigned part1by2(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ inline unsigned compact1by2(unsigned v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x000003ffu;
  return v;
}
__host__ __device__ inline unsigned morton3(unsigned x, unsigned y, unsigned z) {
  return part1by2(x) | (part1by2(y) << 1) | (part1by2(z) << 2);
}

// Square root of x >= 0 and a quotient: correctly rounded in FP64; in FP32
// through the hardware reciprocal square root and the fast divide (a few
// ulp; root gives 0 for x <= 0 or NaN), which the FP32 form's tolerances
// absorb. The FP32 form's pair loops and per-particle material model use
// them; a correctly rounded FP32 divide or root costs a refinement sequence,
// a check and a branch to a slow path. root0: the same root through PTX's
// approximate square root (exact 0 at 0, so no zero test); the density walk
// takes it (1.7 % faster there; in the force walk it cost 2.8 %, through
// that kernel's register allocation).
template <typename T> __device__ __forceinline__ T root(T x);
template <> __device__ __forceinline__ float root<float>(float x) {
  return x > 0.f ? x * rsqrtf(x) : 0.f;
}
template <> __device__ __forceinline__ double root<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T root0(T x);
template <> __device__ __forceinline__ float root0<float>(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <> __device__ __forceinline__ double root0<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T quot(T a, T b);
template <> __device__ __forceinline__ float quot<float>(float a, float b) {
  return __fdividef(a, b);
}
template <> __device__ __forceinline__ double quot<double>(double a, double b) { return a / b; }

// -------------------------------------------------------- material model
// Equation of state, evaluated in T (FP64 form: double; FP32 form: float).
// Linear: P = c0^2 (rho - rho0), c = c0. Tillotson (Tillotson 1962; regions
// as in Melosh 1989): condensed or cold states, hot expanded states and a
// linear-in-u blend in between, with c^2 = P_rho + P P_u / rho^2 floored at
// 0.01 A / rho0. mu = rho / rho0 - 1 is formed from an FP64 difference so
// that the FP32 form keeps its relative accuracy near rho0. The returned P
// is floored at the material's p_min; c is that of the unfloored EOS.
template <typename T> struct EosT {
  T P, c;
};

template <typename T>
__device__ inline void till_dense_t(const MatT<T> &M, T eta, T mu, T rho, T u, T &P, T &Pr, T &Pu) {
  const T e0e2 = M.E0 * eta * eta;
  const T w = quot(u, e0e2) + T(1);
  const T bw = quot(M.b, w), bw2 = quot(bw, w);   // b / w, b / w^2
  P = (M.a + bw) * rho * u + mu * (M.A + M.B * mu);
  // dw/drho = -2 (w - 1) / rho, dw/du = 1 / (E0 eta^2)
  Pr = (M.a + bw) * u + bw2 * u * T(2) * (w - T(1)) + (M.A + T(2) * M.B * mu) * M.inv_rho0;
  Pu = (M.a + bw) * rho - quot(bw2 * rho * u, e0e2);
}

template <typename T>
__device__ inline void till_vapour_t(const MatT<T> &M, T eta, T mu, T rho, T u, T &P, T &Pr,
                                     T &Pu) {
  const T A = M.A, a = M.a, b = M.b, al = M.alpha, be = M.beta;
  const T e0e2 = M.E0 * eta * eta;
  const T w = quot(u, e0e2) + T(1);
  const T z = quot(-mu, eta);                  // rho0 / rho - 1
  const T zr = quot(T(-1), eta * rho);         // dz / drho
  const T eb = exp(-be * z), ea = exp(-al * z * z);
  const T brw = quot(b * rho * u, w);
  const T q = brw + A * mu * eb;
  const T qr = quot(b * u, w) + quot(quot(brw, w) * T(2) * (w - T(1)), rho) +
               A * M.inv_rho0 * eb - A * mu * eb * be * zr;
  const T qu = quot(b * rho, w) - quot(quot(brw, w), e0e2);
  P = a * rho * u + q * ea;
  Pr = a * u + (qr - q * T(2) * al * z * zr) * ea;
  Pu = a * rho + qu * ea;
}

// a >= b and a <= b on the integer pipe when b > 0 (IEEE-754 bit patterns
// of a positive b order like the values; a negative a has a negative
// pattern); the FP64 comparison otherwise.
__device__ __forceinline__ bool ge_d(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ib > 0 ? ia >= ib : a >= b;
}
__device__ __forceinline__ bool le_d(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ib > 0 ? ia <= ib : a <= b;
}

template <typename T>
__device__ inline EosT<T> eos_t(const MatT<T> &M, double rhod, double ud) {
  EosT<T> o;
  if (M.eos == SPH_EOS_LINEAR) {
    o.P = tmax_(M.c0sq * to_t<T>(rhod - M.rho0_d), M.p_min);
    o.c = M.c0;
    return o;
  }
  const T u = to_t<T>(ud), rho = to_t<T>(rhod);
  const T mu = to_t<T>(rhod - M.rho0_d) * M.inv_rho0;
  const T eta = T(1) + mu;
  T P, Pr, Pu;
  if (ge_d(rhod, M.rho0_d) || le_d(ud, M.Eiv_d)) {
    till_dense_t<T>(M, eta, mu, rho, u, P, Pr, Pu);
  } else if (ge_d(ud, M.Ecv_d)) {
    till_vapour_t<T>(M, eta, mu, rho, u, P, Pr, Pu);
  } else {
    T P1, Pr1, Pu1, P2, Pr2, Pu2;
    till_dense_t<T>(M, eta, mu, rho, u, P1, Pr1, Pu1);
    till_vapour_t<T>(M, eta, mu, rho, u, P2, Pr2, Pu2);
    const T wv = to_t<T>(ud - M.Eiv_d) * M.inv_dE, wd = to_t<T>(M.Ecv_d - ud) * M.inv_dE;
    P = wv * P2 + wd * P1;
    Pr = wv * Pr2 + wd * Pr1;
    Pu = wv * Pu2 + wd * Pu1 + (P2 - P1) * M.inv_dE;
  }
  T c2 = Pr + quot(P * Pu, rho * rho);
  if (!(c2 >= M.floor2)) c2 = M.floor2;
  o.P = tmax_(P, M.p_min);
  o.c = root(c2);
  return o;
}

// Shear modulus: constant, or Eq. 30 with nu = 0.25 (Gamma = 0.6 rho c^2).
template <typename T> __device__ __forceinline__ T shear_mod_t(const MatT<T> &M, T rho, T c) {
  return M.shear_G >= T(0) ? M.shear_G : T(0.6) * rho * c * c;
}

// Yield strength (Eq. 34-37) with the pressure clipped at zero.
template <typename T> __device__ inline T yield_t(const MatT<T> &M, T P, T u) {
  const T p = tmax_(P, T(0));
  const T yi = M.Y0 + quot(M.mu_i * p, T(1) + quot(M.mu_i * p, M.Ym - M.Y0));
  T y = tmin_(yi, M.mu_d * p);
  if (M.thermal_softening) {
    const T Tk = M.T0 + u * M.inv_cv;
    if (!(Tk > T(0))) return T(0);
    y *= tmax_(tanh(M.xi * (quot(M.Tm, Tk) - T(1))), T(0));
  }
  return y;
}

// Radial-return factor (Eq. 31-33) of S = {xx, yy, xy, xz, yz}.
template <typename T> __device__ inline T radial_factor_t(const T S[5], T Y, int norm) {
  const T zz = -(S[0] + S[1]);
  const T j2 = T(0.5) * (S[0] * S[0] + S[1] * S[1] + zz * zz) + S[2] * S[2] + S[3] * S[3] +
               S[4] * S[4];
  if (!(j2 > T(0))) return T(1);
  const T f = quot(Y, root(norm ? T(3) * j2 : j2));
  return f < T(1) ? f : T(1);
}

// The field's constants and tables in the arithmetic type of a form.
template <typename T> struct FieldT {
  const T *g, *phi, *r;
  T rmin, rmax, gm, inv_log_ratio, gu[3];
};
__device__ __forceinline__ FieldT<float> field_t(const KParams &P, float) {
  return {P.g_table_f, P.phi_table_f, P.g_radii_f, P.g_rmin_f, P.g_rmax_f, P.g_gm_f,
          P.g_inv_log_ratio_f, {P.g_uniform_f[0], P.g_uniform_f[1], P.g_uniform_f[2]}};
}
__device__ __forceinline__ FieldT<double> field_t(const KParams &P, double) {
  return {P.g_table, P.phi_table, P.g_radii, P.g_rmin, P.g_rmax, P.g_gm,
          P.g_inv_log_ratio, {P.g_uniform[0], P.g_uniform[1], P.g_uniform[2]}};
}

// External field at an absolute position (uniform, or radial table with
// linear interpolation between log-spaced radii). The offset from the
// centre, and the uniform field's potential, are formed in FP64.
template <typename T>
__device__ inline void ext_field_t(const KParams &P, double x, double y, double z, T g[3], T *phi) {
  g[0] = g[1] = g[2] = T(0);
  if (phi) *phi = T(0);
  if (P.gravity == SPH_GRAVITY_UNIFORM) {
    const FieldT<T> F = field_t(P, T(0));
    g[0] = F.gu[0];
    g[1] = F.gu[1];
    g[2] = F.gu[2];
    if (phi) *phi = to_t<T>(-(P.g_uniform[0] * x + P.g_uniform[1] * y + P.g_uniform[2] * z));
    return;
  }
  if (P.gravity != SPH_GRAVITY_RADIAL) return;
  const FieldT<T> F = field_t(P, T(0));
  const T dx = to_t<T>(x - P.g_center[0]), dy = to_t<T>(y - P.g_center[1]),
          dz = to_t<T>(z - P.g_center[2]);
  const T r = root(dx * dx + dy * dy + dz * dz);
  if (!(r > T(0))) return;
  const T rmin = F.rmin, rmax = F.rmax;
  T gm, ph;
  if (r >= rmax) {
    gm = quot(F.gm, r * r);
    ph = quot(-F.gm, r);
  } else if (r <= rmin) {
    const T g0 = F.g[0];
    gm = quot(g0 * r, rmin);
    ph = F.phi[0] + quot(T(0.5) * g0, rmin) * (r * r - rmin * rmin);
  } else {
    int k = (int)floorf(log2f((float)quot(r, rmin)) * (float)F.inv_log_ratio);
    k = max(0, min(k, P.g_n - 2));
    if (r < F.r[k] && k > 0) --k;
    else if (r >= F.r[k + 1] && k < P.g_n - 2) ++k;
    const T r0 = F.r[k], r1 = F.r[k + 1];
    const T w = quot(r - r0, r1 - r0);
    const T ga = F.g[k], gb = F.g[k + 1];
    gm = ga + w * (gb - ga);
    const T pa = F.phi[k], pb = F.phi[k + 1];
    ph = pa + w * (pb - pa);
  }
  g[0] = quot(-gm * dx, r);
  g[1] = quot(-gm * dy, r);
  g[2] = quot(-gm * dz, r);
  if (phi) *phi = ph;
}

// Lattice support radius of a particle (first-guess scale and cap base).
__device__ __forceinline__ double lattice_radius(int n_ngb, double m, double rho0) {
  return cbrt(3.0 * n_ngb * m / (4.0 * kPi * rho0));
}

}  // namespace sphk

// --------------------------------------------------------------- context
struct sph_ctx {
  sph_params params;
  sph_material mats[SPH_MAX_MATERIALS];
  int nmat;
  sph_state st;
  int64_t n;
  cudaStream_t stream;
  sphk::KParams kp;
  sph_material *d_mats;
  sphk::MatT<float> *d_matf;
  sphk::MatT<double> *d_matd;
  double *d_gtab, *d_phitab, *d_radii;
  float *d_gtab_f;       // FP32 copies: g, phi, radii (3 x g_n)
  sphk::Work w;
  // sort and cell list
  unsigned *keys, *keys_alt;
  int *vals, *vals_alt;
  unsigned *hist, *scan_tot;
  int ntiles;
  int *cell_start, *cell_end;
  int max_cells;
  void *tmp;            // permutation scratch: tmp_words words of 8 bytes per particle
  int tmp_words;
  // global steps: the force pass kicks every particle in its epilogue (no
  // separate kick kernel); set only while such a step is enqueued
  int fuse_kick;
  // sph_step_host with global steps: the force pass runs as copy_chunks
  // launches over consecutive bucket ranges, alternating between fstream[0]
  // and fstream[1] (so that one launch's tail overlaps the next one's
  // start), and each range's final state is copied back as soon as its
  // launch completes (chunk_ev); chunked_out marks a step enqueued so
  int copy_chunks;
  int out_done;                 // the step's last group is already being copied back
  cudaStream_t fstream[2];
  cudaEvent_t chunk_ev[SPH_MAX_COPY_CHUNKS], ev_pre;
  unsigned *d_chunk_ctr;        // one bucket counter per launch
  int nsys;
  int64_t *sys_first;   // host copy of the system boundaries (nsys + 1)
  int *d_sys_begin, *d_sys_bucket;
  int *d_red_tile;          // tile starts, tile ends, per-system tile offsets
  double *tile_partials;    // per reduction tile
  sphk::SysRec *d_sys;
  sphk::SysRec *h_sys;      // pinned mirror
  double *d_dt;             // device copy of the current dt of every system
  sphk::Status *d_status;
  sphk::Status *h_status;   // pinned mirror
  double *h_dt;             // pinned dt staging (nsys)
  double *dt_next;          // host, per system
  int occ_density, occ_forces;   // resident blocks per SM of the pair kernels
  void *dens_spill;              // overflow of the density kernel's candidate lists
  int spill_warps;               // warps it has room for
  int num_sms;
  int timing;
  int use_graph;
  int capturing;                // the step is being captured into a graph
  cudaStream_t gstream;         // library stream that graphs are captured on
  cudaEvent_t fence;            // caller stream -> library stream ordering
  // sph_step_host: each group of state arrays is copied back on cstream as
  // soon as the step has finished writing it (host_out != null only then)
  const sph_state *host_out;
  int rungs;                    // sph_params.max_rung
  cudaStream_t cstream;
  cudaEvent_t out_ev[5];
  // sph_step_host's split copy-in: the arrays the sort and the density
  // solve read come first on the context's stream; the rest follow on
  // istream (after ev_a) while those kernels run, and in_ev marks their
  // arrival (split_in: the step waits for it before the predictor)
  cudaStream_t istream;
  cudaEvent_t ev_a, in_ev;
  int split_in;
  // Read view of the state between a step's sort and the kernels that
  // rewrite it (lazy = 1: steps without hierarchical rungs). The arrays
  // that a later kernel of the step rewrites for every particle (v, u, S
  // and the strain invariant by the kicks, H by the density solve, the
  // derivatives by the force pass) are not copied back after the
  // permutation: src points at their permuted copies in the scratch block
  // and the first readers take them from there; the rest of src is the
  // caller's arrays. Outside a lazy step src equals st.
  sph_state src;
  int lazy;
  cudaGraphExec_t graph_exec;   // captured step
  cudaEvent_t ev[SPH_NUM_PHASES + 1];
  // online tuning of the group spans over the coming steps
  sphk::LearnArgs learn;        // learned form (hprev == null: off)
  const struct sph_mlp *net;    // network of the learned guess
  int nlaunch;                  // kernels enqueued by the current call
  int graph_nlaunch;            // kernels in the captured step
  int tune_left;                // steps still to be timed (0: not tuning)
  int tune_idx;                 // tuning steps taken so far
  int tune_now;                 // the step being enqueued is timed
  cudaEvent_t tev[4];           // density start / end, forces start / end
  double tune_ms_d[sphk::kNumSpans], tune_ms_f[sphk::kNumSpans];
  int tune_n[sphk::kNumSpans];
  // staging depths in use (FP32 form) and the tuner's depth phase
  int depth_d, depth_f;
  int tune_phase, tune_rounds;   // 0: spans, 1: depths at the chosen spans
  double tune_dms_d[sphk::kNumDepths], tune_dms_f[sphk::kNumDepths];
  int tune_dn[sphk::kNumDepths];
  double phase_ms[SPH_NUM_PHASES];
  int timed_steps;
  int primed;
  int broken;
  int fail_after;               // injected failure: the fail_after-th checked call (0: none)
  char err[512];
};

// Grid of a persistent pair kernel: as many blocks as stay resident, at
// most one warp per bucket of 32 particles.
template <typename K> inline int resident_grid(const sph_ctx *c, K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * sphk::kWarpsPerBlock,
                                                    0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int64_t need = ((int64_t)c->kp.nbuckets + sphk::kWarpsPerBlock - 1) / sphk::kWarpsPerBlock;
  const int64_t have = (int64_t)per_sm * c->num_sms;
  return (int)(need < have ? need : have);
}

// Launch helpers implemented in the .cu files (all stream-ordered).
namespace sphk {
cudaError_t launch_drift_bbox(sph_ctx *c, int do_drift);
cudaError_t launch_grid_setup(sph_ctx *c, int keep);
// all = 0: leave out the arrays a step recomputes before reading them;
// part 1: only what the drift, sort and density solve read (the rest
// follows with launch_permute_rest once it has been copied in)
cudaError_t launch_sort_permute(sph_ctx *c, int all, int part);
cudaError_t launch_permute_rest(sph_ctx *c);
// parts: bit 0 the evaluation (predicted) state, bit 1 the packed positions
cudaError_t launch_pack(sph_ctx *c);
cudaError_t launch_density(sph_ctx *c, int expand);
cudaError_t launch_eos_pack(sph_ctx *c, int predict);
cudaError_t launch_forces(sph_ctx *c);
cudaError_t launch_forces_range(sph_ctx *c, int b0, int b1, unsigned *ctr, cudaStream_t stream);
cudaError_t launch_kick(sph_ctx *c, int kick);
// the step's sums from the per-particle terms the kicks left (per tile, then
// per system)
cudaError_t launch_reduce_buckets(sph_ctx *c);
cudaError_t launch_reset_status(sph_ctx *c, int full);
cudaError_t launch_rung_init(sph_ctx *c);
// hierarchical steps: the list of the substep's active particles (KParams::act)
cudaError_t launch_compact_active(sph_ctx *c);
cudaError_t launch_learn(sph_ctx *c);
cudaError_t alloc_density_spill(sph_ctx *c);
}  // namespace sphk
