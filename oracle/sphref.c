/*
 * sphref.c -- FP64 CPU oracle for the SPH particle step with material
 * strength (Meier et al., "SPH in pkdgrav3 for Shock Physics Simulations. II.
 * Shear Strength", §2.1-§2.4).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this code. It is the plain, slow reference the
 * CUDA path is compared against: every per-pair sum is written as the paper
 * prints it, per particle, in FP64, over neighbours j in ascending array
 * index. It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Readings of points the paper leaves open are marked "Reading:" where they
 * are used. Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include "sphref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

int32_t ref_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* Thread count of the following parallel regions (timing runs only; the
 * results do not depend on it). Returns the count now in effect. */
int32_t ref_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads((int)n);
  return (int32_t)omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel: Wendland C2 in three dimensions (§3: "Wendland C2 kernel",        */
/* Dehnen & Aly 2012). Reading: h in Eq. 1-3 is the compact support radius  */
/* H, W(r, H) = 21 / (2 pi H^3) (1 - q)^4 (1 + 4 q), q = r / H < 1.          */
/* ------------------------------------------------------------------------ */
double ref_W(double r, double H) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double t = 1.0 - q;
  return 21.0 / (2.0 * PI * H * H * H) * t * t * t * t * (1.0 + 4.0 * q);
}

/* dW/dr = 21 / (2 pi H^4) d/dq[(1-q)^4 (1+4q)] = -(210 / pi) q (1-q)^3 / H^4 */
double ref_dWdr(double r, double H) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double t = 1.0 - q;
  return -210.0 / PI * q * t * t * t / (H * H * H * H);
}

/* dW/dH at fixed r: W = H^-3 f(r/H) gives dW/dH = -(3 W + q f'(q) H^-3) / H
 * = -21 / (2 pi H^4) (1-q)^3 (3 + 9 q - 32 q^2). */
double ref_dWdH(double r, double H) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double t = 1.0 - q;
  return -21.0 / (2.0 * PI * H * H * H * H) * t * t * t * (3.0 + 9.0 * q - 32.0 * q * q);
}

/* ------------------------------------------------------------------------ */
/* Equations of state. The paper uses M-ANEOS through EOSlib (§2.3); the    */
/* workloads here use a linear EOS and the Tillotson EOS instead.           */
/* Reading (Tillotson): region split as in Melosh (1989): compressed or     */
/* cold states use the condensed form, hot expanded states the vapour form, */
/* and states between Eiv and Ecv a linear blend in u. Sound speed          */
/* c^2 = dP/drho|_u + P / rho^2 dP/du|_rho, floored at 0.01 A / rho0.       */
/* ------------------------------------------------------------------------ */
static void till_condensed(const ref_material *mt, double rho, double u,
                           double *P, double *dPdr, double *dPdu) {
  double eta = rho / mt->rho0, mu = eta - 1.0;
  double w0 = u / (mt->E0 * eta * eta) + 1.0;
  double dw_dr = -2.0 * (w0 - 1.0) / rho;
  double dw_du = 1.0 / (mt->E0 * eta * eta);
  *P = (mt->a + mt->b / w0) * rho * u + mt->A * mu + mt->B * mu * mu;
  *dPdr = (mt->a + mt->b / w0) * u - mt->b * rho * u / (w0 * w0) * dw_dr +
          (mt->A + 2.0 * mt->B * mu) / mt->rho0;
  *dPdu = (mt->a + mt->b / w0) * rho - mt->b * rho * u / (w0 * w0) * dw_du;
}

static void till_expanded(const ref_material *mt, double rho, double u,
                          double *P, double *dPdr, double *dPdu) {
  double eta = rho / mt->rho0, mu = eta - 1.0;
  double w0 = u / (mt->E0 * eta * eta) + 1.0;
  double dw_dr = -2.0 * (w0 - 1.0) / rho;
  double dw_du = 1.0 / (mt->E0 * eta * eta);
  double z = 1.0 / eta - 1.0, dz_dr = -mt->rho0 / (rho * rho);
  double eb = exp(-mt->beta * z), ez = exp(-mt->alpha * z * z);
  double inner = mt->b * rho * u / w0 + mt->A * mu * eb;
  double dinner_dr = mt->b * u / w0 - mt->b * rho * u / (w0 * w0) * dw_dr +
                     mt->A / mt->rho0 * eb + mt->A * mu * eb * (-mt->beta * dz_dr);
  double dinner_du = mt->b * rho / w0 - mt->b * rho * u / (w0 * w0) * dw_du;
  *P = mt->a * rho * u + inner * ez;
  *dPdr = mt->a * u + dinner_dr * ez + inner * ez * (-2.0 * mt->alpha * z * dz_dr);
  *dPdu = mt->a * rho + dinner_du * ez;
}

/* Reading: a material may floor its pressure (p_min; a cohesionless
 * granular medium carries no tension, p_min = 0). The floor applies to P
 * only; the sound speed is that of the unfloored EOS. */
void ref_eos(const ref_material *mt, double rho, double u, double *P, double *cs) {
  if (mt->eos == REF_EOS_LINEAR) {
    double pl = mt->c0 * mt->c0 * (rho - mt->rho0);
    *P = pl < mt->p_min ? mt->p_min : pl;
    *cs = mt->c0;
    return;
  }
  double p, pr, pu;
  if (rho >= mt->rho0 || u <= mt->Eiv) {
    till_condensed(mt, rho, u, &p, &pr, &pu);
  } else if (u >= mt->Ecv) {
    till_expanded(mt, rho, u, &p, &pr, &pu);
  } else {
    double pc, prc, puc, pe, pre, pue, dE = mt->Ecv - mt->Eiv;
    till_condensed(mt, rho, u, &pc, &prc, &puc);
    till_expanded(mt, rho, u, &pe, &pre, &pue);
    p = ((u - mt->Eiv) * pe + (mt->Ecv - u) * pc) / dE;
    pr = ((u - mt->Eiv) * pre + (mt->Ecv - u) * prc) / dE;
    pu = ((u - mt->Eiv) * pue + pe + (mt->Ecv - u) * puc - pc) / dE;
  }
  double c2 = pr + p / (rho * rho) * pu;
  double c2min = 0.01 * mt->A / mt->rho0;
  if (!(c2 >= c2min)) c2 = c2min;
  *P = p < mt->p_min ? mt->p_min : p;
  *cs = sqrt(c2);
}

/* Shear modulus: a material constant, or Eq. 30 with nu = 0.25 and the bulk
 * modulus K = rho c^2. */
static double shear_modulus(const ref_material *mt, double rho, double cs) {
  if (mt->shear_G >= 0.0) return mt->shear_G;
  double nu = 0.25;
  return 3.0 * (1.0 - 2.0 * nu) / (2.0 * (1.0 + nu)) * rho * cs * cs;
}

/* Yield strength, §2.3: intact Eq. 34, damaged Eq. 35, Y = min (Eq. 36),
 * thermal softening Eq. 37. Pressures below zero are clipped to zero (§2.3).
 * Reading: T = T0 + u / cv with a constant melt temperature Tm; the softening
 * factor is clipped at zero above Tm and Y = 0 for T <= 0. */
double ref_yield(const ref_material *mt, double P, double u) {
  double Pc = P > 0.0 ? P : 0.0;
  double Yi = mt->Y0 + mt->mu_i * Pc / (1.0 + mt->mu_i * Pc / (mt->Ym - mt->Y0));
  double Yd = mt->mu_d * Pc;
  double Y = Yi < Yd ? Yi : Yd;
  if (mt->thermal_softening) {
    double T = mt->T0 + u / mt->cv;
    if (T <= 0.0) return 0.0;
    double s = tanh(mt->xi * (mt->Tm / T - 1.0));
    Y *= s > 0.0 ? s : 0.0;
  }
  return Y;
}

/* Radial return, Eq. 31-33: J2 = 1/2 S:S with S_zz = -S_xx - S_yy (Eq. 11),
 * f = min(Y / sqrt(J2), 1). yield_norm = 1 reads the criterion as
 * sqrt(3 J2) <= Y instead. */
double ref_radial_return(double S[5], double Y, int32_t yield_norm) {
  double szz = -S[0] - S[1];
  double J2 = 0.5 * (S[0] * S[0] + S[1] * S[1] + szz * szz +
                     2.0 * (S[2] * S[2] + S[3] * S[3] + S[4] * S[4]));
  if (!(J2 > 0.0)) return 1.0;
  double root = yield_norm ? sqrt(3.0 * J2) : sqrt(J2);
  double f = Y / root;
  if (!(f < 1.0)) return 1.0;
  for (int k = 0; k < 5; ++k) S[k] *= f;
  return f;
}

/* Deviatoric stress rate from the corrected gradient G (row-major,
 * G[3a+b] = dv^a/dx^b, Eq. 22). S = {xx, yy, xy, xz, yz}.
 * jaumann = 1: the component form exactly as printed, Eq. 25-29.
 * jaumann = 0: Eq. 13 with rotation terms R S - S R (R from Eq. 23, edot from
 * Eq. 24), the frame-indifferent Jaumann rate of Benz & Asphaug (1994). */
void ref_stress_rate(const double S[5], const double G[9], double Gm,
                     int32_t jaumann, double dS[5]) {
  double Gxx = G[0], Gxy = G[1], Gxz = G[2];
  double Gyx = G[3], Gyy = G[4], Gyz = G[5];
  double Gzx = G[6], Gzy = G[7], Gzz = G[8];
  double Sxx = S[0], Syy = S[1], Sxy = S[2], Sxz = S[3], Syz = S[4];
  if (jaumann == 1) {
    dS[0] = Sxy * (Gyx - Gxy) + Sxz * (Gzx - Gxz) -
            2.0 / 3.0 * Gm * (Gyy + Gzz - 2.0 * Gxx);
    dS[1] = Sxy * (Gxy - Gyx) + Syz * (Gzy - Gyz) -
            2.0 / 3.0 * Gm * (Gxx + Gzz - 2.0 * Gyy);
    dS[2] = Gm * (Gxy + Gyx) +
            0.5 * (Sxx * (Gxy - Gyx) + Syy * (Gyx - Gxy) + Syz * (Gzx - Gxz) +
                   Sxz * (Gzy - Gyz));
    dS[3] = Gm * (Gxz + Gzx) +
            0.5 * ((Sxx + Syy) * (Gxz - Gzx) + Sxx * (Gxz - Gzx) +
                   Syz * (Gyx - Gxy) + Sxy * (Gyz - Gzy));
    dS[4] = Gm * (Gyz + Gzy) +
            0.5 * ((Sxx + Syy) * (Gyz - Gzy) + Sxz * (Gxy - Gyx) +
                   Sxy * (Gxz - Gzx) + Syy * (Gyz - Gzy));
    return;
  }
  double Sm[3][3] = {{Sxx, Sxy, Sxz}, {Sxy, Syy, Syz}, {Sxz, Syz, -Sxx - Syy}};
  double E[3][3], R[3][3], out[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      E[a][b] = 0.5 * (G[3 * a + b] + G[3 * b + a]);
      R[a][b] = 0.5 * (G[3 * a + b] - G[3 * b + a]);
    }
  double tr = E[0][0] + E[1][1] + E[2][2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double rot = 0.0;
      for (int c = 0; c < 3; ++c) rot += R[a][c] * Sm[c][b] - Sm[a][c] * R[c][b];
      out[a][b] = 2.0 * Gm * (E[a][b] - (a == b ? tr / 3.0 : 0.0)) + rot;
    }
  dS[0] = out[0][0];
  dS[1] = out[1][1];
  dS[2] = out[0][1];
  dS[3] = out[0][2];
  dS[4] = out[1][2];
}

/* 3x3 inverse by cofactors; returns det(A). */
double ref_inv3(const double A[9], double Ainv[9]) {
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  double id = 1.0 / det;
  Ainv[0] = c00 * id;
  Ainv[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  Ainv[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  Ainv[3] = c01 * id;
  Ainv[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  Ainv[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  Ainv[6] = c02 * id;
  Ainv[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  Ainv[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return det;
}

/* ------------------------------------------------------------------------ */
/* External field. Self-gravity is not part of this step; it enters as a    */
/* given uniform field or a given radial table g(r) about a centre, linear  */
/* in r between log-spaced table radii, g = G M / r^2 beyond the table and  */
/* g proportional to r inside the first radius.                             */
/* ------------------------------------------------------------------------ */
static double table_interp(const ref_params *p, const double *tab, double r) {
  double lr = log(r / p->g_rmin) / log(p->g_rmax / p->g_rmin) * (double)(p->g_n - 1);
  int64_t k = (int64_t)floor(lr);
  if (k < 0) k = 0;
  if (k > p->g_n - 2) k = p->g_n - 2;
  double r0 = p->g_rmin * pow(p->g_rmax / p->g_rmin, (double)k / (double)(p->g_n - 1));
  double r1 = p->g_rmin * pow(p->g_rmax / p->g_rmin, (double)(k + 1) / (double)(p->g_n - 1));
  double w = (r - r0) / (r1 - r0);
  return tab[k] + w * (tab[k + 1] - tab[k]);
}

void ref_gravity(const ref_params *p, double x, double y, double z, double g[3]) {
  g[0] = g[1] = g[2] = 0.0;
  if (p->gravity == 1) {
    g[0] = p->g_uniform[0];
    g[1] = p->g_uniform[1];
    g[2] = p->g_uniform[2];
  } else if (p->gravity == 2) {
    double dx = x - p->g_center[0], dy = y - p->g_center[1], dz = z - p->g_center[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r > 0.0)) return;
    double gm;
    if (r >= p->g_rmax) gm = p->g_gm / (r * r);
    else if (r <= p->g_rmin) gm = p->g_table[0] * r / p->g_rmin;
    else gm = table_interp(p, p->g_table, r);
    g[0] = -gm * dx / r;
    g[1] = -gm * dy / r;
    g[2] = -gm * dz / r;
  }
}

double ref_potential(const ref_params *p, double x, double y, double z) {
  if (p->gravity == 1) return -(p->g_uniform[0] * x + p->g_uniform[1] * y + p->g_uniform[2] * z);
  if (p->gravity != 2) return 0.0;
  double dx = x - p->g_center[0], dy = y - p->g_center[1], dz = z - p->g_center[2];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  if (r >= p->g_rmax) return -p->g_gm / r;
  if (r <= p->g_rmin)
    return p->phi_table[0] + 0.5 * p->g_table[0] / p->g_rmin * (r * r - p->g_rmin * p->g_rmin);
  return table_interp(p, p->phi_table, r);
}

/* ------------------------------------------------------------------------ */
/* Neighbour search. The membership predicate is evaluated in FP64 as       */
/* dx = x_i - x_j (minimum image in a periodic box), r^2 = (dx dx + dy dy)  */
/* + dz dz without fused multiply-add, and r^2 < R^2 (strict). Two searches */
/* give the same sets: O(N^2) brute force, and a uniform grid whose cells   */
/* are visited in any order, after which the candidates are sorted by      */
/* index so that every sum runs over j in ascending index.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int brute;
  int64_t dims[3];
  double lo[3], cell[3], box[3];
  int periodic;
  int64_t *head, *next;
} grid_t;

static inline double min_image(double d, double box, int periodic) {
  if (periodic) {
    if (d > 0.5 * box) d -= box;
    else if (d < -0.5 * box) d += box;
  }
  return d;
}

static inline double dist2(const grid_t *g, const double *x, const double *y,
                           const double *z, int64_t i, int64_t j) {
  double dx = min_image(x[i] - x[j], g->box[0], g->periodic);
  double dy = min_image(y[i] - y[j], g->box[1], g->periodic);
  double dz = min_image(z[i] - z[j], g->box[2], g->periodic);
  return (dx * dx + dy * dy) + dz * dz;
}

static void grid_free(grid_t *g) {
  free(g->head);
  free(g->next);
  g->head = g->next = NULL;
}

/* Cell size at least R; cell count capped near 2^24. */
static void grid_build(grid_t *g, const ref_params *p, int64_t n, const double *x,
                       const double *y, const double *z, double R) {
  memset(g, 0, sizeof(*g));
  g->periodic = p->periodic;
  for (int a = 0; a < 3; ++a) g->box[a] = p->box_hi[a] - p->box_lo[a];
  g->brute = p->brute_force || n < 2;
  if (g->brute) return;
  const double *c[3] = {x, y, z};
  double ext[3];
  for (int a = 0; a < 3; ++a) {
    double lo, hi;
    if (p->periodic) {
      lo = p->box_lo[a];
      hi = p->box_hi[a];
    } else {
      lo = hi = c[a][0];
      for (int64_t i = 1; i < n; ++i) {
        if (c[a][i] < lo) lo = c[a][i];
        if (c[a][i] > hi) hi = c[a][i];
      }
    }
    g->lo[a] = lo;
    ext[a] = hi - lo;
    g->cell[a] = R > 0.0 ? R : 1.0;
  }
  for (;;) {
    for (int a = 0; a < 3; ++a) {
      g->dims[a] = (int64_t)floor(ext[a] / g->cell[a]);
      if (!p->periodic) g->dims[a] += 1;
      if (g->dims[a] < 1) g->dims[a] = 1;
    }
    if (g->dims[0] * g->dims[1] * g->dims[2] <= (1 << 24)) break;
    for (int a = 0; a < 3; ++a) g->cell[a] *= 1.26;
  }
  if (p->periodic)
    for (int a = 0; a < 3; ++a) g->cell[a] = ext[a] / (double)g->dims[a];
  int64_t nc = g->dims[0] * g->dims[1] * g->dims[2];
  g->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
  g->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t k = 0; k < nc; ++k) g->head[k] = -1;
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t ci[3];
    for (int a = 0; a < 3; ++a) {
      double t = (c[a][i] - g->lo[a]) / g->cell[a];
      int64_t k = (int64_t)floor(t);
      if (k < 0) k = p->periodic ? ((k % g->dims[a]) + g->dims[a]) % g->dims[a] : 0;
      if (k >= g->dims[a]) k = p->periodic ? k % g->dims[a] : g->dims[a] - 1;
      ci[a] = k;
    }
    int64_t cell = (ci[2] * g->dims[1] + ci[1]) * g->dims[0] + ci[0];
    g->next[i] = g->head[cell];
    g->head[cell] = i;
  }
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

/* Collect j with dist2 < R_ij^2; mode 0: R = H_i (self included), mode 1:
 * R = max(H_i, H_j), j != i. Hq overrides H_i when >= 0 (the Newton sweeps
 * evaluate trial radii). Output sorted ascending; returns the count. */
static int64_t collect(const grid_t *g, int64_t n, const double *x, const double *y,
                       const double *z, const double *h, int64_t i, double Hq,
                       double Rsearch, int mode, int64_t **buf, int64_t *cap) {
  double Hi = Hq >= 0.0 ? Hq : h[i];
  int64_t cnt = 0;
  int brute = g->brute;
  int64_t span[3] = {0, 0, 0};
  if (!brute) {
    for (int a = 0; a < 3; ++a) {
      span[a] = (int64_t)ceil(Rsearch / g->cell[a]);
      if (g->periodic && 2 * span[a] + 1 > g->dims[a]) brute = 1;
    }
  }
#define PUSH(j)                                                         \
  do {                                                                  \
    if (cnt == *cap) {                                                  \
      *cap = *cap * 2 + 64;                                             \
      *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * (size_t)*cap);  \
    }                                                                   \
    (*buf)[cnt++] = (j);                                                \
  } while (0)
  if (brute) {
    for (int64_t j = 0; j < n; ++j) {
      double r2 = dist2(g, x, y, z, i, j);
      if (mode == 0) {
        if (r2 < Hi * Hi) PUSH(j);
      } else if (j != i) {
        double R = Hi > h[j] ? Hi : h[j];
        if (r2 < R * R) PUSH(j);
      }
    }
    return cnt;
  }
  const double *c[3] = {x, y, z};
  int64_t ci[3];
  for (int a = 0; a < 3; ++a) {
    int64_t k = (int64_t)floor((c[a][i] - g->lo[a]) / g->cell[a]);
    if (g->periodic) k = ((k % g->dims[a]) + g->dims[a]) % g->dims[a];
    else if (k < 0) k = 0;
    else if (k >= g->dims[a]) k = g->dims[a] - 1;
    ci[a] = k;
  }
  for (int64_t oz = -span[2]; oz <= span[2]; ++oz)
    for (int64_t oy = -span[1]; oy <= span[1]; ++oy)
      for (int64_t ox = -span[0]; ox <= span[0]; ++ox) {
        int64_t k[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz};
        int skip = 0;
        for (int a = 0; a < 3; ++a) {
          if (g->periodic) k[a] = ((k[a] % g->dims[a]) + g->dims[a]) % g->dims[a];
          else if (k[a] < 0 || k[a] >= g->dims[a]) skip = 1;
        }
        if (skip) continue;
        int64_t cell = (k[2] * g->dims[1] + k[1]) * g->dims[0] + k[0];
        for (int64_t j = g->head[cell]; j >= 0; j = g->next[j]) {
          double r2 = dist2(g, x, y, z, i, j);
          if (mode == 0) {
            if (r2 < Hi * Hi) PUSH(j);
          } else if (j != i) {
            double R = Hi > h[j] ? Hi : h[j];
            if (r2 < R * R) PUSH(j);
          }
        }
      }
#undef PUSH
  qsort(*buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
  return cnt;
}

static double max_of(const double *a, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i)
    if (a[i] > m) m = a[i];
  return m;
}

int64_t ref_neighbours(const ref_params *p, int64_t n, const double *x,
                       const double *y, const double *z, const double *h,
                       int64_t i, int32_t mode, int64_t *out, int64_t cap) {
  grid_t g;
  double hmax = max_of(h, n);
  grid_build(&g, p, n, x, y, z, hmax);
  int64_t bcap = 256, *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)bcap);
  int64_t cnt = collect(&g, n, x, y, z, h, i, -1.0, mode == 0 ? h[i] : hmax, mode, &buf, &bcap);
  for (int64_t k = 0; k < cnt && k < cap; ++k) out[k] = buf[k];
  free(buf);
  grid_free(&g);
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Density (Eq. 1), the grad-h term (Eq. 3) and the neighbour count at a    */
/* given H. Reading: the sum includes j = i; the count excludes it.         */
/* ------------------------------------------------------------------------ */
static void density_sums(const grid_t *g, int64_t n, const ref_state *s, int64_t i,
                         double H, int64_t **buf, int64_t *cap, double *rho,
                         double *rhoH, int32_t *count) {
  int64_t cnt = collect(g, n, s->x, s->y, s->z, s->h, i, H, H, 0, buf, cap);
  double r_sum = 0.0, rh_sum = 0.0;
  int32_t c = 0;
  for (int64_t k = 0; k < cnt; ++k) {
    int64_t j = (*buf)[k];
    double r = sqrt(dist2(g, s->x, s->y, s->z, i, j));
    r_sum += s->m[j] * ref_W(r, H);
    rh_sum += s->m[j] * ref_dWdH(r, H);
    if (j != i) ++c;
  }
  *rho = r_sum;
  *rhoH = rh_sum;
  *count = c;
}

void ref_count_neighbours(const ref_params *p, int64_t n, const ref_state *s,
                          int64_t nsel, const int64_t *idx, int32_t *count) {
  grid_t g;
  grid_build(&g, p, n, s->x, s->y, s->z, max_of(s->h, n));
  int64_t nl = idx ? nsel : n;
#pragma omp parallel
  {
    int64_t cap = 256, *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < nl; ++k) {
      int64_t i = idx ? idx[k] : k;
      int64_t cnt = collect(&g, n, s->x, s->y, s->z, s->h, i, -1.0, s->h[i], 0, &buf, &cap);
      count[k] = (int32_t)(cnt - 1);
    }
    free(buf);
  }
  grid_free(&g);
}

void ref_density_given_h(const ref_params *p, int64_t n, const ref_state *s,
                         int64_t nsel, const int64_t *idx, double *rho,
                         double *omega, int32_t *count) {
  grid_t g;
  grid_build(&g, p, n, s->x, s->y, s->z, max_of(s->h, n));
  int64_t nl = idx ? nsel : n;
#pragma omp parallel
  {
    int64_t cap = 256, *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < nl; ++k) {
      int64_t i = idx ? idx[k] : k;
      double r, rh;
      int32_t c;
      density_sums(&g, n, s, i, s->h[i], &buf, &cap, &r, &rh, &c);
      rho[k] = r;
      omega[k] = 1.0 + s->h[i] / (3.0 * r) * rh; /* Eq. 3 */
      count[k] = c;
    }
    free(buf);
  }
  grid_free(&g);
}

/* Lattice support radius of a particle: the H at which a uniform medium of
 * density rho0 holds n_ngb particle masses, (4 pi / 3) H^3 rho0 = n_ngb m. */
static double lattice_h(const ref_params *p, const ref_material *mt, double m) {
  return cbrt(3.0 * p->n_ngb * m / (4.0 * PI * mt->rho0));
}

/* Smoothing-length solve (§2.1, Eq. 2-3). Newton-Raphson on
 * g(H) = (4 pi / 3) H^3 rho(H) - n_ngb m_i with g'(H) = 4 pi H^2 rho Omega.
 * Reading of what the paper leaves open: start from the current H; stop at
 * |g| <= h_tol n_ngb m_i, keeping (H, rho, Omega, count) of that evaluation;
 * otherwise H <- H - g / g', limited to [0.75 H, 1.25 H], replaced by the
 * midpoint of the bracket [lo, hi] of the root when it leaves it, and capped
 * at h_cap_factor times the lattice radius (a particle at the cap with
 * g < 0 is accepted and counted as capped). A particle that has not met
 * the tolerance after max_sweeps keeps its last evaluated H.
 * Reading: Eq. 3 leaves the grad-h factor of a capped particle without
 * meaning -- it falls to 0 as the neighbours vanish (a lone particle's
 * rho = m W(0, H) gives exactly 1 + (H / 3 rho)(-3 rho / H) = 0), and every
 * term over Omega rho then divides by zero -- so a capped particle takes
 * Omega = 1. */
static int32_t density_solve_sel(const ref_params *p, const ref_material *mats, int64_t n,
                                 ref_state *s, const unsigned char *active, int32_t *n_unconv,
                                 int32_t *n_capped);

int32_t ref_density_solve(const ref_params *p, const ref_material *mats,
                          int64_t n, ref_state *s, int32_t *n_unconv,
                          int32_t *n_capped) {
  return density_solve_sel(p, mats, n, s, NULL, n_unconv, n_capped);
}

/* The solve for the particles with active[i] != 0 (all when active is
 * NULL); the others keep H, rho, Omega and their count. */
static int32_t density_solve_sel(const ref_params *p, const ref_material *mats, int64_t n,
                                 ref_state *s, const unsigned char *active, int32_t *n_unconv,
                                 int32_t *n_capped) {
  double hmax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double cap = p->h_cap_factor * lattice_h(p, &mats[s->mat[i]], s->m[i]);
    double h0 = s->h[i] < cap ? s->h[i] : cap;
    if (h0 > hmax) hmax = h0;
  }
  grid_t g;
  grid_build(&g, p, n, s->x, s->y, s->z, hmax);
  int32_t worst = 0, unconv = 0, capped = 0;
#pragma omp parallel reduction(max : worst) reduction(+ : unconv, capped)
  {
    int64_t cap = 256, *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
      if (active && !active[i]) continue;
      double target = p->n_ngb * s->m[i];
      double Hcap = p->h_cap_factor * lattice_h(p, &mats[s->mat[i]], s->m[i]);
      double H = s->h[i] < Hcap ? s->h[i] : Hcap;
      double lo = 0.0, hi = INFINITY;
      double rho = 0.0, rhoH = 0.0, Om = 1.0, Heval = H;
      int32_t c = 0, sweep, done = 0;
      for (sweep = 1; sweep <= p->max_sweeps; ++sweep) {
        Heval = H;
        density_sums(&g, n, s, i, H, &buf, &cap, &rho, &rhoH, &c);
        Om = 1.0 + H / (3.0 * rho) * rhoH;
        double gv = 4.0 * PI / 3.0 * H * H * H * rho - target;
        if (fabs(gv) <= p->h_tol * target) {
          done = 1;
          break;
        }
        if (gv < 0.0 && H >= Hcap) {
          done = 2;
          break;
        }
        if (gv < 0.0) lo = H;
        else hi = H;
        double gp = 4.0 * PI * H * H * rho * Om;
        double Hn = gp > 0.0 ? H - gv / gp : (gv < 0.0 ? 1.25 * H : 0.75 * H);
        if (!(Hn >= 0.75 * H)) Hn = 0.75 * H;
        if (!(Hn <= 1.25 * H)) Hn = 1.25 * H;
        if (hi < INFINITY && (Hn <= lo || Hn >= hi)) Hn = 0.5 * (lo + hi);
        if (Hn > Hcap) Hn = Hcap;
        H = Hn;
      }
      if (sweep > p->max_sweeps) sweep = p->max_sweeps;
      if (!done) ++unconv;
      if (done == 2) {
        ++capped;
        Om = 1.0;
      }
      if (sweep > worst) worst = sweep;
      s->h[i] = Heval; /* rho, Omega and the count belong to this H */
      s->rho[i] = rho;
      s->omega[i] = Om;
      s->nngb[i] = c;
    }
    free(buf);
  }
  grid_free(&g);
  if (n_unconv) *n_unconv = unconv;
  if (n_capped) *n_capped = capped;
  return worst;
}

/* EOS at (rho, u_eval), yield (Eq. 34-37) and radial return (Eq. 31-33) of
 * the evaluation stress. Fluid materials keep S = 0. */
void ref_eos_yield(const ref_params *p, const ref_material *mats, int64_t n,
                   ref_state *s, const double *u_eval, double *sxx, double *syy,
                   double *sxy, double *sxz, double *syz) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const ref_material *mt = &mats[s->mat[i]];
    double P, c;
    ref_eos(mt, s->rho[i], u_eval[i], &P, &c);
    s->pres[i] = P;
    s->cs[i] = c;
    double Y = ref_yield(mt, P, u_eval[i]);
    if (s->yld) s->yld[i] = Y;
    double S[5] = {sxx[i], syy[i], sxy[i], sxz[i], syz[i]};
    if (!mt->strength) {
      S[0] = S[1] = S[2] = S[3] = S[4] = 0.0;
    } else {
      ref_radial_return(S, Y, p->yield_norm);
    }
    sxx[i] = S[0];
    syy[i] = S[1];
    sxy[i] = S[2];
    sxz[i] = S[3];
    syz[i] = S[4];
  }
}

/* ------------------------------------------------------------------------ */
/* Pair sums, literally as printed, for particle i over its neighbours j    */
/* with r_ij < max(H_i, H_j), j != i, in ascending j. Conventions:          */
/* x_ij = x_i - x_j, v_ij = v_i - v_j, dW/dx_i = W'(r, H) x_ij / r.          */
/*   hydro acceleration                       Eq. 4                         */
/*   artificial viscosity Pi_ij, mu_ij        Eq. 5-6 (v_ij . x_ij < 0)      */
/*   viscous acceleration and heating         Eq. 7-8, W_bar = (W(H_i) +     */
/*                                            W(H_j)) / 2                   */
/*   stress acceleration                      Eq. 18 (sum term)             */
/*   energy equation                          Eq. 19; du/dt|_H read as      */
/*     P_i / (Omega_i rho_i^2) sum_j m_j v_ij . dW_ij(H_i)/dx_i              */
/*   velocity gradient F, correction C^-1     Eq. 20-21; gradient_form = 1: */
/*     the H_i term of both sums alone, -sum_j m_j v_ij (x) dW(H_i)/dx_i /   */
/*     (Omega_i rho_i) (Reading: the non-symmetric form named in §2.2)       */
/*   corrected gradient, R, strain rate       Eq. 22-24                     */
/*   stress rate                              Eq. 13 / Eq. 25-29            */
/*   CFL signal of Eq. 39                                                   */
/* Readings: h_bar in Eq. 6 averages the support radii H; C = I when fewer  */
/* than 8 neighbours or |det C^-1| < 1e-3; fixed particles get zero         */
/* derivatives; the CFL uses the longitudinal speed sqrt(c^2 + 4/3 G/rho)   */
/* for materials with strength.                                             */
/* ------------------------------------------------------------------------ */
void ref_forces(const ref_params *p, const ref_material *mats, int64_t n,
                ref_state *s, const double *vx, const double *vy,
                const double *vz, const double *sxx, const double *syy,
                const double *sxy, const double *sxz, const double *syz,
                int64_t nsel, const int64_t *idx, double *Gout, double *Cout,
                int32_t *n_cfallback) {
  double hmax = max_of(s->h, n);
  grid_t g;
  grid_build(&g, p, n, s->x, s->y, s->z, hmax);
  int64_t nl = idx ? nsel : n;
  int32_t fallbacks = 0;
  const double al = p->av_alpha, be = p->av_beta, ep = p->av_eps;
#pragma omp parallel reduction(+ : fallbacks)
  {
    int64_t cap = 256, *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t k = 0; k < nl; ++k) {
      int64_t i = idx ? idx[k] : k;
      const ref_material *mt = &mats[s->mat[i]];
      int strength = mt->strength;
      double Hi = s->h[i], rhoi = s->rho[i], Omi = s->omega[i], Pi = s->pres[i];
      double ci = s->cs[i];
      double Si[3][3] = {{sxx[i], sxy[i], sxz[i]},
                         {sxy[i], syy[i], syz[i]},
                         {sxz[i], syz[i], -sxx[i] - syy[i]}};
      if (!strength) memset(Si, 0, sizeof(Si));
      double aH[3] = {0, 0, 0}, aS[3] = {0, 0, 0}, aPi[3] = {0, 0, 0};
      double duH = 0.0, duPi = 0.0, Es[3][3] = {{0}}, F[3][3] = {{0}}, Ci[3][3] = {{0}};
      double muneg = 0.0;
      int64_t cnt = collect(&g, n, s->x, s->y, s->z, s->h, i, -1.0, hmax, 1, &buf, &cap);
      for (int64_t kk = 0; kk < cnt; ++kk) {
        int64_t j = buf[kk];
        const ref_material *mj = &mats[s->mat[j]];
        double Hj = s->h[j], rhoj = s->rho[j], Omj = s->omega[j], Pj = s->pres[j];
        double cj = s->cs[j], m = s->m[j];
        double xij[3] = {min_image(s->x[i] - s->x[j], g.box[0], g.periodic),
                         min_image(s->y[i] - s->y[j], g.box[1], g.periodic),
                         min_image(s->z[i] - s->z[j], g.box[2], g.periodic)};
        double vij[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
        double r2 = (xij[0] * xij[0] + xij[1] * xij[1]) + xij[2] * xij[2];
        double r = sqrt(r2);
        double gWi[3], gWj[3], gWb[3];
        double fi = r > 0.0 ? ref_dWdr(r, Hi) / r : 0.0;
        double fj = r > 0.0 ? ref_dWdr(r, Hj) / r : 0.0;
        for (int a = 0; a < 3; ++a) {
          gWi[a] = fi * xij[a];
          gWj[a] = fj * xij[a];
          gWb[a] = 0.5 * (gWi[a] + gWj[a]);
        }
        double Sj[3][3] = {{sxx[j], sxy[j], sxz[j]},
                           {sxy[j], syy[j], syz[j]},
                           {sxz[j], syz[j], -sxx[j] - syy[j]}};
        if (!mj->strength) memset(Sj, 0, sizeof(Sj));
        /* Eq. 4 */
        for (int a = 0; a < 3; ++a)
          aH[a] -= m * (Pi / (Omi * rhoi * rhoi) * gWi[a] + Pj / (Omj * rhoj * rhoj) * gWj[a]);
        /* Eq. 18, stress term */
        for (int a = 0; a < 3; ++a) {
          double t = 0.0;
          for (int b = 0; b < 3; ++b)
            t += Si[a][b] / (Omi * rhoi * rhoi) * gWi[b] + Sj[a][b] / (Omj * rhoj * rhoj) * gWj[b];
          aS[a] += m * t;
        }
        /* Eq. 5-6 */
        double vr = vij[0] * xij[0] + vij[1] * xij[1] + vij[2] * xij[2];
        double hb = 0.5 * (Hi + Hj), cb = 0.5 * (ci + cj), rb = 0.5 * (rhoi + rhoj);
        double mu = hb * vr / (r2 + ep * hb * hb);
        double PI_ij = vr < 0.0 ? (-al * cb * mu + be * mu * mu) / rb : 0.0;
        if (mu < 0.0 && -mu > muneg) muneg = -mu;
        /* Eq. 7-8 */
        double vgb = vij[0] * gWb[0] + vij[1] * gWb[1] + vij[2] * gWb[2];
        for (int a = 0; a < 3; ++a) aPi[a] -= m * PI_ij * gWb[a];
        duPi += 0.5 * m * PI_ij * vgb;
        /* du/dt|_H */
        duH += Pi / (Omi * rhoi * rhoi) * m * (vij[0] * gWi[0] + vij[1] * gWi[1] + vij[2] * gWi[2]);
        /* Eq. 19 sum, Eq. 20-21 */
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            Es[a][b] += m * vij[a] * gWi[b];
            double w = p->gradient_form ? 2.0 * gWi[b] / (Omi * rhoi)
                                        : gWi[b] / (Omi * rhoi) + gWj[b] / (Omj * rhoj);
            F[a][b] += -0.5 * m * vij[a] * w;
            Ci[a][b] += -0.5 * m * xij[a] * w;
          }
      }
      /* Eq. 19 strength term */
      double duS = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) duS -= Si[a][b] / (Omi * rhoi * rhoi) * Es[a][b];
      /* Eq. 21-22 with the guard */
      double Cm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Cflat[9], Gm[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Cflat[3 * a + b] = Ci[a][b];
      if (p->correction_tensor) {
        double inv[9];
        double det = ref_inv3(Cflat, inv);
        if (s->nngb[i] >= 8 && fabs(det) >= 1e-3) memcpy(Cm, inv, sizeof(Cm));
        else ++fallbacks;
      }
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double t = 0.0;
          for (int c = 0; c < 3; ++c) t += F[a][c] * Cm[3 * c + b];
          Gm[3 * a + b] = t;
        }
      double Sv[5] = {Si[0][0], Si[1][1], Si[0][1], Si[0][2], Si[1][2]};
      double dS[5] = {0, 0, 0, 0, 0};
      if (strength) ref_stress_rate(Sv, Gm, shear_modulus(mt, rhoi, ci), p->jaumann, dS);
      double gx[3];
      ref_gravity(p, s->x[i], s->y[i], s->z[i], gx);
      double cl = ci;
      if (strength) cl = sqrt(ci * ci + 4.0 / 3.0 * shear_modulus(mt, rhoi, ci) / rhoi);
      if (s->vsig) s->vsig[i] = (1.0 + 0.6 * al) * cl + 0.6 * be * muneg;
      int fixed = s->flags[i] & 1;
      s->ax[i] = fixed ? 0.0 : aH[0] + aPi[0] + aS[0] + gx[0];
      s->ay[i] = fixed ? 0.0 : aH[1] + aPi[1] + aS[1] + gx[1];
      s->az[i] = fixed ? 0.0 : aH[2] + aPi[2] + aS[2] + gx[2];
      s->dudt[i] = fixed ? 0.0 : duH + duPi + duS;
      s->dsxx[i] = fixed ? 0.0 : dS[0];
      s->dsyy[i] = fixed ? 0.0 : dS[1];
      s->dsxy[i] = fixed ? 0.0 : dS[2];
      s->dsxz[i] = fixed ? 0.0 : dS[3];
      s->dsyz[i] = fixed ? 0.0 : dS[4];
      if (Gout) memcpy(Gout + 9 * k, Gm, sizeof(Gm));
      if (Cout) memcpy(Cout + 9 * k, Cm, sizeof(Cm));
    }
    free(buf);
  }
  grid_free(&g);
  if (n_cfallback) *n_cfallback = fallbacks;
}

/* Global sums: kinetic, internal and external-field energy, linear momentum
 * and angular momentum L = sum m r x v (Eq. 46). */
void ref_diagnostics(const ref_params *p, int64_t n, const ref_state *s, ref_info *info) {
  double ek = 0, eu = 0, ep = 0, px = 0, py = 0, pz = 0, lx = 0, ly = 0, lz = 0;
  for (int64_t i = 0; i < n; ++i) {
    double m = s->m[i];
    ek += 0.5 * m * (s->vx[i] * s->vx[i] + s->vy[i] * s->vy[i] + s->vz[i] * s->vz[i]);
    eu += m * s->u[i];
    ep += m * ref_potential(p, s->x[i], s->y[i], s->z[i]);
    px += m * s->vx[i];
    py += m * s->vy[i];
    pz += m * s->vz[i];
    lx += m * (s->y[i] * s->vz[i] - s->z[i] * s->vy[i]);
    ly += m * (s->z[i] * s->vx[i] - s->x[i] * s->vz[i]);
    lz += m * (s->x[i] * s->vy[i] - s->y[i] * s->vx[i]);
  }
  info->e_kin = ek;
  info->e_int = eu;
  info->e_pot = ep;
  info->p[0] = px;
  info->p[1] = py;
  info->p[2] = pz;
  info->L[0] = lx;
  info->L[1] = ly;
  info->L[2] = lz;
}

/* Time step of Eq. 38-39, minimum over moving particles. Reading: the
 * softening epsilon of Eq. 38 is the kernel support H_i. */
static double next_dt(const ref_params *p, int64_t n, const ref_state *s) {
  double dt = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    if (s->flags[i] & 1) continue;
    double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
    double ta = a > 0.0 ? p->eta_a * sqrt(s->h[i] / a) : INFINITY;
    double tc = p->eta_c * s->h[i] / s->vsig[i];
    double t = ta < tc ? ta : tc;
    if (t < dt) dt = t;
  }
  return dt;
}

static double *dup(const double *a, int64_t n) {
  double *b = (double *)malloc(sizeof(double) * (size_t)n);
  memcpy(b, a, sizeof(double) * (size_t)n);
  return b;
}

int32_t ref_derivatives(const ref_params *p, const ref_material *mats,
                        int64_t n, ref_state *s, ref_info *info) {
  int32_t unconv = 0, capped = 0, fb = 0;
  int32_t sweeps = ref_density_solve(p, mats, n, s, &unconv, &capped);
  double *S[5] = {dup(s->sxx, n), dup(s->syy, n), dup(s->sxy, n), dup(s->sxz, n), dup(s->syz, n)};
  double *vs = s->vsig ? NULL : (double *)malloc(sizeof(double) * (size_t)n);
  if (vs) s->vsig = vs;
  ref_eos_yield(p, mats, n, s, s->u, S[0], S[1], S[2], S[3], S[4]);
  ref_forces(p, mats, n, s, s->vx, s->vy, s->vz, S[0], S[1], S[2], S[3], S[4], n, NULL,
             NULL, NULL, &fb);
  if (info) {
    ref_diagnostics(p, n, s, info);
    info->dt_next = next_dt(p, n, s);
    info->max_sweeps = sweeps;
    info->n_unconverged = unconv;
    info->n_capped = capped;
    info->n_cfallback = fb;
  }
  if (vs) {
    free(vs);
    s->vsig = NULL;
  }
  for (int k = 0; k < 5; ++k) free(S[k]);
  return unconv ? 3 : 0;
}

/* One step of the predictor-corrector of §2.4 (Eq. 40-43), applied to v, u
 * and S alike (the paper integrates S "with the same predictor-corrector
 * scheme as the internal energy"):
 *   drift      x_i = x_{i-1} + dt v_{i-1/2}
 *   predict    q_pred = q_{i-1/2} + dt/2 dq_{i-1}         (Eq. 40), S rescaled
 *   derivatives at i from the predicted state
 *   close      q_i = q_{i-1/2} + dt/2 dq_i                (Eq. 41), S rescaled
 *              with Y from the EOS at (rho_i, u_i)
 *   open       q_{i+1/2} = q_i + dt/2 dq_i                (Eq. 42)
 *   invariant  eps_ii += dt * 1/2 edot:edot at i           (Eq. 43)
 * Fixed particles are neither drifted nor kicked. Diagnostics use x_i, v_i. */
int32_t ref_step(const ref_params *p, const ref_material *mats, int64_t n,
                 ref_state *s, double dt, ref_info *info) {
  const double hdt = 0.5 * dt;
  for (int64_t i = 0; i < n; ++i) {
    if (s->flags[i] & 1) continue;
    s->x[i] += dt * s->vx[i];
    s->y[i] += dt * s->vy[i];
    s->z[i] += dt * s->vz[i];
  }
  if (p->periodic) {
    double *c[3] = {s->x, s->y, s->z};
    for (int a = 0; a < 3; ++a) {
      double L = p->box_hi[a] - p->box_lo[a];
      for (int64_t i = 0; i < n; ++i) {
        if (c[a][i] >= p->box_hi[a]) c[a][i] -= L;
        else if (c[a][i] < p->box_lo[a]) c[a][i] += L;
      }
    }
  }
  double *vp[3] = {dup(s->vx, n), dup(s->vy, n), dup(s->vz, n)};
  double *up = dup(s->u, n);
  double *Sp[5] = {dup(s->sxx, n), dup(s->syy, n), dup(s->sxy, n), dup(s->sxz, n), dup(s->syz, n)};
  double *dS[5] = {s->dsxx, s->dsyy, s->dsxy, s->dsxz, s->dsyz};
  double *a[3] = {s->ax, s->ay, s->az};
  for (int64_t i = 0; i < n; ++i) {
    if (s->flags[i] & 1) continue;
    for (int c = 0; c < 3; ++c) vp[c][i] += hdt * a[c][i];
    up[i] += hdt * s->dudt[i];
    for (int c = 0; c < 5; ++c) Sp[c][i] += hdt * dS[c][i];
  }
  int32_t unconv = 0, capped = 0, fb = 0;
  int32_t sweeps = ref_density_solve(p, mats, n, s, &unconv, &capped);
  double *vs = s->vsig ? NULL : (double *)malloc(sizeof(double) * (size_t)n);
  if (vs) s->vsig = vs;
  ref_eos_yield(p, mats, n, s, up, Sp[0], Sp[1], Sp[2], Sp[3], Sp[4]);
  double *G = (double *)malloc(sizeof(double) * 9 * (size_t)n);
  ref_forces(p, mats, n, s, vp[0], vp[1], vp[2], Sp[0], Sp[1], Sp[2], Sp[3], Sp[4], n,
             NULL, G, NULL, &fb);
  double *S[5] = {s->sxx, s->syy, s->sxy, s->sxz, s->syz};
  double *v[3] = {s->vx, s->vy, s->vz};
  /* closing kick to i */
  for (int64_t i = 0; i < n; ++i) {
    if (s->flags[i] & 1) continue;
    const ref_material *mt = &mats[s->mat[i]];
    for (int c = 0; c < 3; ++c) v[c][i] += hdt * a[c][i];
    s->u[i] += hdt * s->dudt[i];
    double Sv[5];
    for (int c = 0; c < 5; ++c) Sv[c] = S[c][i] + hdt * dS[c][i];
    if (mt->strength) {
      double P, cs;
      ref_eos(mt, s->rho[i], s->u[i], &P, &cs);
      ref_radial_return(Sv, ref_yield(mt, P, s->u[i]), p->yield_norm);
    } else {
      Sv[0] = Sv[1] = Sv[2] = Sv[3] = Sv[4] = 0.0;
    }
    for (int c = 0; c < 5; ++c) S[c][i] = Sv[c];
    const double *Gi = G + 9 * i;
    double ee = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double e = 0.5 * (Gi[3 * r + c] + Gi[3 * c + r]);
        ee += e * e;
      }
    s->eps_ii[i] += dt * 0.5 * ee;
  }
  if (info) {
    ref_diagnostics(p, n, s, info);
    info->dt_next = next_dt(p, n, s);
    info->max_sweeps = sweeps;
    info->n_unconverged = unconv;
    info->n_capped = capped;
    info->n_cfallback = fb;
  }
  /* opening kick to i + 1/2 */
  for (int64_t i = 0; i < n; ++i) {
    if (s->flags[i] & 1) continue;
    for (int c = 0; c < 3; ++c) v[c][i] += hdt * a[c][i];
    s->u[i] += hdt * s->dudt[i];
    for (int c = 0; c < 5; ++c) S[c][i] += hdt * dS[c][i];
  }
  if (vs) {
    free(vs);
    s->vsig = NULL;
  }
  free(G);
  for (int c = 0; c < 3; ++c) free(vp[c]);
  free(up);
  for (int c = 0; c < 5; ++c) free(Sp[c]);
  return unconv ? 3 : 0;
}

/* ------------------------------------------------------------------------ */
/* Hierarchical individual time steps. §2.4 takes its step sizes from the   */
/* criteria of Eq. 38-39 within the hierarchical scheme of the paper's      */
/* Paper I, which is not printed here. Reading: power-of-two rungs with the */
/* predictor-corrector of ref_step applied per particle:                    */
/*   the big step dt is split into L = 2^R substeps of delta = dt / L; a    */
/*   particle on rung r steps dt_r = dt / 2^r, i.e. len = 2^(R-r) substeps, */
/*   and its steps start at multiples of len;                               */
/*   every substep drifts every moving particle by delta with its half-step */
/*   velocity; the particles whose step ends at the substep's end are       */
/*   active: their density is solved, their derivatives are formed from the */
/*   state predicted to that time, and they are kicked (closing and opening */
/*   kicks of dt_r / 2, rescale, strain invariant over dt_r);               */
/*   the other particles enter as neighbours with v, u, S predicted to the  */
/*   same time, q + (t - t_mid) dq with t_mid the midpoint of their current */
/*   step and dq their last derivatives, and with their last H, rho, Omega; */
/*   the EOS and radial return of the predicted state run for every one;   */
/*   a kicked particle takes the rung its criteria ask for (the smallest r  */
/*   with dt / 2^r <= min(dt_a, dt_CFL), at most R), but no coarser than    */
/*   the coarsest rung whose steps start at the next substep; rungs are set */
/*   from the criteria of the last derivatives at the start of a big step.  */
/* Fixed particles are never kicked; their density is solved at the end of  */
/* the big step (rung 0). R = 0 is ref_step.                                */
/* ------------------------------------------------------------------------ */
static int32_t rung_for(const ref_params *p, const ref_state *s, int64_t i, double dt,
                        int32_t R) {
  double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
  double ta = a > 0.0 ? p->eta_a * sqrt(s->h[i] / a) : INFINITY;
  double tc = p->eta_c * s->h[i] / s->vsig[i];
  double t = ta < tc ? ta : tc;
  int32_t r = 0;
  while (r < R && dt / (double)(1 << r) > t) ++r;
  return r;
}

int32_t ref_step_rungs(const ref_params *p, const ref_material *mats, int64_t n,
                       ref_state *s, double dt, int32_t R, int32_t *rung,
                       int64_t *active_updates, ref_info *info) {
  if (R < 0 || R > 15 || !s->vsig || !rung) return 4;
  const int64_t L = (int64_t)1 << R;
  const double delta = dt / (double)L;
  for (int64_t i = 0; i < n; ++i) rung[i] = (s->flags[i] & 1) ? 0 : rung_for(p, s, i, dt, R);
  double *vp[3] = {dup(s->vx, n), dup(s->vy, n), dup(s->vz, n)};
  double *up = dup(s->u, n);
  double *Sp[5] = {dup(s->sxx, n), dup(s->syy, n), dup(s->sxy, n), dup(s->sxz, n), dup(s->syz, n)};
  double *G = (double *)malloc(sizeof(double) * 9 * (size_t)n);
  unsigned char *act = (unsigned char *)malloc((size_t)n);
  int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  double *S[5] = {s->sxx, s->syy, s->sxy, s->sxz, s->syz};
  double *dS[5] = {s->dsxx, s->dsyy, s->dsxy, s->dsxz, s->dsyz};
  double *v[3] = {s->vx, s->vy, s->vz};
  double *a[3] = {s->ax, s->ay, s->az};
  int32_t unconv = 0, capped = 0, fb = 0, sweeps = 0, worst = 0;
  int64_t updates = 0;
  for (int64_t sub = 0; sub < L; ++sub) {
    for (int64_t i = 0; i < n; ++i) {
      if (s->flags[i] & 1) continue;
      s->x[i] += delta * s->vx[i];
      s->y[i] += delta * s->vy[i];
      s->z[i] += delta * s->vz[i];
    }
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t len = (int64_t)1 << (R - rung[i]);
      const int64_t start = (sub / len) * len;
      act[i] = (unsigned char)((sub + 1) % len == 0);
      if (act[i]) idx[na++] = i;
      const double k = (s->flags[i] & 1) ? 0.0 : ((double)(sub + 1 - start) - 0.5 * (double)len) * delta;
      for (int c = 0; c < 3; ++c) vp[c][i] = v[c][i] + k * a[c][i];
      up[i] = s->u[i] + k * s->dudt[i];
      for (int c = 0; c < 5; ++c) Sp[c][i] = S[c][i] + k * dS[c][i];
    }
    int32_t uc = 0, cp = 0, f = 0;
    sweeps = density_solve_sel(p, mats, n, s, act, &uc, &cp);
    if (sweeps > worst) worst = sweeps;
    unconv += uc;
    capped += cp;
    ref_eos_yield(p, mats, n, s, up, Sp[0], Sp[1], Sp[2], Sp[3], Sp[4]);
    ref_forces(p, mats, n, s, vp[0], vp[1], vp[2], Sp[0], Sp[1], Sp[2], Sp[3], Sp[4], na, idx,
               G, NULL, &f);
    fb += f;
    /* closing kick of the active particles to their step's end */
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = idx[k];
      if (s->flags[i] & 1) continue;
      ++updates;
      const ref_material *mt = &mats[s->mat[i]];
      const double dti = (double)((int64_t)1 << (R - rung[i])) * delta, hdt = 0.5 * dti;
      for (int c = 0; c < 3; ++c) v[c][i] += hdt * a[c][i];
      s->u[i] += hdt * s->dudt[i];
      double Sv[5];
      for (int c = 0; c < 5; ++c) Sv[c] = S[c][i] + hdt * dS[c][i];
      if (mt->strength) {
        double P, cs;
        ref_eos(mt, s->rho[i], s->u[i], &P, &cs);
        ref_radial_return(Sv, ref_yield(mt, P, s->u[i]), p->yield_norm);
      } else {
        Sv[0] = Sv[1] = Sv[2] = Sv[3] = Sv[4] = 0.0;
      }
      for (int c = 0; c < 5; ++c) S[c][i] = Sv[c];
      const double *Gi = G + 9 * k;
      double ee = 0.0;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double e = 0.5 * (Gi[3 * r + c] + Gi[3 * c + r]);
          ee += e * e;
        }
      s->eps_ii[i] += dti * 0.5 * ee;
    }
    if (sub == L - 1 && info) {   /* every particle is at the big step's end */
      ref_diagnostics(p, n, s, info);
      info->dt_next = next_dt(p, n, s);
    }
    /* new rungs, then the opening kicks */
    int32_t r_al = R;   /* coarsest rung whose steps start at sub + 1 */
    for (int64_t m = sub + 1; r_al > 0 && (m & 1) == 0; m >>= 1) --r_al;
    if (sub + 1 == L) r_al = 0;
    for (int64_t k = 0; k < na; ++k) {
      const int64_t i = idx[k];
      if (s->flags[i] & 1) continue;
      int32_t r = rung_for(p, s, i, dt, R);
      if (r < r_al) r = r_al;
      rung[i] = r;
      const double hdt = 0.5 * (double)((int64_t)1 << (R - r)) * delta;
      for (int c = 0; c < 3; ++c) v[c][i] += hdt * a[c][i];
      s->u[i] += hdt * s->dudt[i];
      for (int c = 0; c < 5; ++c) S[c][i] += hdt * dS[c][i];
    }
  }
  if (info) {
    info->max_sweeps = worst;
    info->n_unconverged = unconv;
    info->n_capped = capped;
    info->n_cfallback = fb;
  }
  if (active_updates) *active_updates = updates;
  free(G);
  free(act);
  free(idx);
  for (int c = 0; c < 3; ++c) free(vp[c]);
  free(up);
  for (int c = 0; c < 5; ++c) free(Sp[c]);
  return unconv ? 3 : 0;
}
