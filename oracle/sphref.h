/*
 * sphref.h -- interface of the FP64 CPU oracle for the SPH particle step with
 * material strength (Meier et al., "SPH in pkdgrav3 for Shock Physics
 * Simulations. II. Shear Strength", §2).
 *
 * TEST INFRASTRUCTURE. This header and sphref.c are used only by the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark. The CUDA
 * library never includes, links or calls anything here, and nothing here
 * includes the CUDA library's headers: the two implementations are
 * independent and are compared against each other.
 *
 * All arrays are host arrays of length n in structure-of-arrays layout,
 * owned by the caller. All floating point is IEEE double. The oracle works
 * in the order the arrays are given; neighbour sums run over j in ascending
 * array index, so callers pass arrays ordered by original particle id.
 */
#ifndef SPHREF_H
#define SPHREF_H
#include <stdint.h>

/* Equation of state selector. */
#define REF_EOS_LINEAR 0
#define REF_EOS_TILLOTSON 1

/* Per-material constants (§2.2 shear modulus, §2.3 yield model). */
typedef struct {
  int32_t eos;            /* REF_EOS_LINEAR or REF_EOS_TILLOTSON */
  double rho0;            /* reference density [kg/m^3] */
  double c0;              /* linear EOS sound speed [m/s] */
  double A, B, E0, a, b, alpha, beta, Eiv, Ecv; /* Tillotson constants */
  double shear_G;         /* Gamma [Pa]; < 0 selects Eq. 30 with nu = 0.25 */
  double Y0, mu_i, Ym, mu_d; /* Eq. 34-35 */
  int32_t thermal_softening; /* Eq. 37 on/off */
  double xi, Tm, T0, cv;  /* Eq. 37 and T = T0 + u / cv */
  int32_t strength;       /* 0: fluid, S stays zero */
  double p_min;           /* pressure floor of the EOS (-inf: none) */
} ref_material;

/* Run-time parameters. */
typedef struct {
  int32_t n_ngb;          /* target neighbour number (constant kernel mass) */
  double av_alpha, av_beta, av_eps; /* Eq. 5-6 */
  double eta_c, eta_a;    /* Eq. 38-39 */
  double h_tol;           /* Newton tolerance on |g| / (n_ngb m) */
  int32_t max_sweeps;     /* Newton sweeps before giving up */
  double h_cap_factor;    /* H never exceeds h_cap_factor * lattice H */
  int32_t jaumann;        /* 0 objective (R S - S R), 1 as printed (Eq. 25-29) */
  int32_t yield_norm;     /* 0: f = min(Y / sqrt(J2), 1); 1: min(Y / sqrt(3 J2), 1) */
  int32_t correction_tensor; /* 1: G = F C (Eq. 22); 0: C = I */
  int32_t gravity;        /* 0 none, 1 uniform, 2 radial table */
  double g_uniform[3];
  const double *g_table;  /* radial table g(r_k) [m/s^2], k = 0..g_n-1 */
  const double *phi_table;/* potential Phi(r_k) [J/kg] on the same radii */
  int32_t g_n;
  double g_rmin, g_rmax;  /* r_k log-spaced from g_rmin to g_rmax */
  double g_center[3];
  double g_gm;            /* G * M_total for r > g_rmax */
  int32_t periodic;       /* 1: periodic box [box_lo, box_hi) in x, y and z */
  double box_lo[3], box_hi[3];
  int32_t brute_force;    /* 1: O(N^2) neighbour search; 0: uniform grid */
  int32_t gradient_form;  /* 0: F, C^-1 as Eq. 20-21; 1: their H_i term alone */
} ref_params;

/* Particle state. Any output pointer the caller does not need may be NULL
 * where the function documents it. */
typedef struct {
  double *x, *y, *z;
  double *vx, *vy, *vz;
  double *u, *m, *h;                 /* h = kernel support radius H */
  double *sxx, *syy, *sxy, *sxz, *syz;
  double *rho, *omega, *pres, *cs, *yld;
  double *ax, *ay, *az, *dudt;
  double *dsxx, *dsyy, *dsxy, *dsxz, *dsyz;
  double *eps_ii;                    /* integral of 1/2 edot:edot dt (Eq. 43) */
  double *vsig;                      /* CFL denominator of Eq. 39 */
  int32_t *nngb, *mat, *flags;       /* flags bit 0: fixed boundary particle */
} ref_state;

/* Per-step diagnostics (Eq. 46 and energy / momentum sums). */
typedef struct {
  double dt_next, e_kin, e_int, e_pot, p[3], L[3];
  int32_t max_sweeps, n_unconverged, n_capped, n_cfallback;
} ref_info;

#ifdef __cplusplus
extern "C" {
#endif

/* Wendland C2 kernel in 3-D, support radius H (§3, Dehnen & Aly form). */
double ref_W(double r, double H);
double ref_dWdr(double r, double H);
double ref_dWdH(double r, double H);

/* Equation of state: pressure and sound speed from (rho, u). */
void ref_eos(const ref_material *mt, double rho, double u, double *P, double *cs);
/* Yield strength Y from pressure and internal energy (Eq. 34-37). */
double ref_yield(const ref_material *mt, double P, double u);
/* Radial return of one deviatoric stress (Eq. 31-33); returns f. */
double ref_radial_return(double S[5], double Y, int32_t yield_norm);
/* Stress rate from the corrected gradient G (row-major 3x3, Eq. 23-29). */
void ref_stress_rate(const double S[5], const double G[9], double shear_G,
                     int32_t jaumann, double dS[5]);
/* 3x3 inverse; returns the determinant of the input. */
double ref_inv3(const double A[9], double Ainv[9]);
/* Given radial or uniform field at a point. */
void ref_gravity(const ref_params *p, double x, double y, double z, double g[3]);
double ref_potential(const ref_params *p, double x, double y, double z);

/* Neighbours of particle i in ascending index order. mode 0: r < H_i
 * (gather, self included); mode 1: r < max(H_i, H_j) (union, self
 * excluded). Returns the count, writes at most cap indices. */
int64_t ref_neighbours(const ref_params *p, int64_t n, const double *x,
                       const double *y, const double *z, const double *h,
                       int64_t i, int32_t mode, int64_t *out, int64_t cap);

/* Neighbour counts #{j != i : r_ij < H_i} with the given H, for the listed
 * particles (idx NULL: all n). */
void ref_count_neighbours(const ref_params *p, int64_t n, const ref_state *s,
                          int64_t nsel, const int64_t *idx, int32_t *count);

/* Kernel sums at the given H (no Newton): rho (Eq. 1), Omega (Eq. 3),
 * count, for the listed particles. */
void ref_density_given_h(const ref_params *p, int64_t n, const ref_state *s,
                         int64_t nsel, const int64_t *idx, double *rho,
                         double *omega, int32_t *count);

/* Smoothing-length solve for every particle: Newton on
 * g(H) = (4 pi / 3) H^3 rho(H) - n_ngb m (Eq. 1-3). Updates h, rho, omega,
 * nngb. Returns the largest sweep count; *n_unconv, *n_capped receive
 * counts. */
int32_t ref_density_solve(const ref_params *p, const ref_material *mats,
                          int64_t n, ref_state *s, int32_t *n_unconv,
                          int32_t *n_capped);

/* EOS, yield and radial return of the evaluation stress (Eq. 31-37). Reads
 * rho and u_eval; writes pres, cs, yld; rescales the given S arrays. */
void ref_eos_yield(const ref_params *p, const ref_material *mats, int64_t n,
                   ref_state *s, const double *u_eval, double *sxx, double *syy,
                   double *sxy, double *sxz, double *syz);

/* Pair sums and per-particle finalize (Eq. 4-8, 18-29) for the listed
 * particles (idx NULL: all). Positions, h, m, rho, omega, pres, cs, nngb,
 * flags, mat come from s; velocities and stress are the evaluation state
 * passed separately. Writes ax..az, dudt, ds*, vsig. If G and Cm are not
 * NULL, the corrected gradient and the correction tensor are written there
 * (9 values per listed particle, row-major). */
void ref_forces(const ref_params *p, const ref_material *mats, int64_t n,
                ref_state *s, const double *vx, const double *vy,
                const double *vz, const double *sxx, const double *syy,
                const double *sxy, const double *sxz, const double *syz,
                int64_t nsel, const int64_t *idx, double *G, double *Cm,
                int32_t *n_cfallback);

/* One full step of length dt (§2.4): drift, predict, density, EOS + yield,
 * forces, closing kick + rescale, opening kick. The state holds x at i-1,
 * v, u, S at i-1/2 and the derivatives at i-1 on entry; x at i, v, u, S at
 * i+1/2 and derivatives at i on return. Returns 0, or 3 when the density
 * solve did not converge for some particle. */
int32_t ref_step(const ref_params *p, const ref_material *mats, int64_t n,
                 ref_state *s, double dt, ref_info *info);
/* Hierarchical individual steps over one big step dt with 2^R substeps;
 * rung (n, out) receives each particle's rung at the end. The state must
 * carry vsig from the last derivatives. Returns 4 for R outside 0..15 or a
 * missing vsig / rung, 3 if a solve did not converge. */
int32_t ref_step_rungs(const ref_params *p, const ref_material *mats, int64_t n,
                       ref_state *s, double dt, int32_t R, int32_t *rung,
                       int64_t *active_updates, ref_info *info);

/* Derivatives of the given state without moving it (predict with dt = 0):
 * density, EOS + yield on a copy of S, forces. Used to start a run. */
int32_t ref_derivatives(const ref_params *p, const ref_material *mats,
                        int64_t n, ref_state *s, ref_info *info);

/* Global sums at the current state (Eq. 46 and energies). */
void ref_diagnostics(const ref_params *p, int64_t n, const ref_state *s,
                     ref_info *info);

/* Threads used by the OpenMP loops. */
int32_t ref_threads(void);
int32_t ref_set_threads(int32_t n);

#ifdef __cplusplus
}
#endif
#endif
