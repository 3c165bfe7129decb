/*
 * sph.h -- C ABI of the B300 (sm_103a) SPH particle step with material
 * strength, after Meier et al., "Smoothed Particle Hydrodynamics in pkdgrav3
 * for Shock Physics Simulations. II. Shear Strength" (§2).
 *
 * One step (§2.4) is: drift; cell-list neighbour search; density and
 * smoothing-length solve (§2.1, Eq. 1-3); equation of state, yield strength
 * (§2.3, Eq. 34-37) and radial return of the predicted deviatoric stress
 * (Eq. 31-33); one pair loop for the full-stress momentum and energy
 * equations with artificial viscosity (Eq. 4-8, 18-19) and the corrected
 * velocity gradient (Eq. 20-24); the Jaumann stress rate (Eq. 13, 25-29);
 * and the predictor-corrector kicks with rescaling (Eq. 40-43).
 *
 * Conventions for every call:
 *  - All particle arrays are DEVICE pointers owned by the caller, length n,
 *    structure-of-arrays. The library never frees them. Calls that sort
 *    (sph_neighbours, sph_step) permute every array of sph_state in place
 *    into cell (Morton) order; `id` travels with the particles.
 *  - The library owns its scratch (cell list, sort buffers, packed mirrors,
 *    predicted state) and frees it in sph_destroy.
 *  - All calls are ordered on the CUDA stream given to sph_init and are not
 *    thread-safe for one context. A call returns after enqueueing its work,
 *    except where it says it synchronises.
 *  - Every call returns a status. Device-side conditions (no convergence,
 *    non-finite results) are latched in a device word and reported at the
 *    next synchronising call. After SPH_E_CUDA the context is left in
 *    SPH_E_STATE and can only be destroyed. sph_last_error() gives detail.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH_OK = 0,
  SPH_E_ARG = 1,        /* invalid argument; nothing was enqueued */
  SPH_E_CUDA = 2,       /* a CUDA runtime call failed */
  SPH_E_NOCONV = 3,     /* smoothing-length solve did not converge */
  SPH_E_CAPACITY = 4,   /* a periodic box axis is not wider than twice a
                           search radius (the minimum image would not be the
                           only image in range); the step's results are not
                           valid. Candidate lists that outgrow their buffers
                           never fail: they continue in further segments. */
  SPH_E_NONFINITE = 5,  /* a derivative or density came out NaN or Inf */
  SPH_E_TIMEOUT = 6,    /* reserved: no kernel waits on a flag or on another
                           block, so none can time out */
  SPH_E_STATE = 7,      /* context unusable after an earlier failure */
  SPH_E_INTERNAL = 8    /* checked build only (compiled with
                           -DSPH_BOUNDS_CHECK): an index that came from data
                           fell outside its array; the access was redirected
                           and the call's results are not valid */
} sph_status;

enum { SPH_EOS_LINEAR = 0, SPH_EOS_TILLOTSON = 1 };
enum { SPH_FP64 = 0, SPH_FP32K = 1 };
enum { SPH_JAUMANN_OBJECTIVE = 0, SPH_JAUMANN_PRINTED = 1 };
enum { SPH_GRADIENT_SYMMETRIC = 0, SPH_GRADIENT_ONE_SIDED = 1 };
enum { SPH_YIELD_SQRT_J2 = 0, SPH_YIELD_SQRT_3J2 = 1 };
enum { SPH_GRAVITY_NONE = 0, SPH_GRAVITY_UNIFORM = 1, SPH_GRAVITY_RADIAL = 2 };
#define SPH_MAX_MATERIALS 8
#define SPH_MAX_SYSTEMS 1024
#define SPH_MAX_COPY_CHUNKS 16
#define SPH_FLAG_FIXED 1

typedef struct sph_ctx sph_ctx;

/* Particle state: caller-owned device arrays of length n.
 *   x, y, z        position [m] (x at time i after a step)
 *   vx, vy, vz     velocity at i+1/2 (half-step, §2.4) [m/s]
 *   u              specific internal energy at i+1/2 [J/kg]
 *   m              mass [kg]
 *   h              kernel support radius H [m]; read as the first guess of
 *                  the solve and overwritten with the converged value
 *   sxx..syz       deviatoric stress S at i+1/2, five independent
 *                  components (S_zz = -S_xx - S_yy, Eq. 11) [Pa]
 *   rho, omega     density (Eq. 1) and grad-h term (Eq. 3)      (outputs)
 *   pres, cs       pressure and sound speed from the EOS       (outputs)
 *   ax..az, dudt, dsxx..dsyz
 *                  time derivatives at i (input: at i-1, used by the
 *                  predictor; output: at i)
 *   eps_ii         integral of 1/2 edot:edot dt (Eq. 43)       (in/out)
 *   nngb           #{j != i : r_ij < H_i}                       (output)
 *   mat            material index into the sph_init table
 *   flags          bit 0: fixed boundary particle (never moved, no
 *                  derivatives)
 *   id             caller's particle identifier, permuted with the rest */
typedef struct {
  double *x, *y, *z;
  double *vx, *vy, *vz;
  double *u, *m, *h;
  double *sxx, *syy, *sxy, *sxz, *syz;
  double *rho, *omega, *pres, *cs;
  double *ax, *ay, *az, *dudt;
  double *dsxx, *dsyy, *dsxy, *dsxz, *dsyz;
  double *eps_ii;
  int32_t *nngb, *mat, *flags;
  int64_t *id;
} sph_state;

/* Material constants. Linear EOS P = c0^2 (rho - rho0); Tillotson with
 * (rho0, A, B, E0, a, b, alpha, beta, Eiv, Ecv). Shear modulus shear_G, or
 * Eq. 30 with nu = 0.25 when shear_G < 0. Yield: Eq. 34-36 with (Y0, mu_i,
 * Ym, mu_d); thermal softening Eq. 37 with T = T0 + u / cv when
 * thermal_softening != 0. strength = 0 makes the material a fluid (S = 0).
 * p_min floors the pressure the EOS returns (-INFINITY: no floor; 0 for a
 * cohesionless medium that carries no tension); the sound speed is that of
 * the unfloored EOS. */
typedef struct {
  int32_t eos;
  double rho0, c0;
  double A, B, E0, a, b, alpha, beta, Eiv, Ecv;
  double shear_G;
  double Y0, mu_i, Ym, mu_d;
  int32_t thermal_softening;
  double xi, Tm, T0, cv;
  int32_t strength;
  double p_min;
} sph_material;

/* Run-time parameters.
 *   n_ngb          target neighbour number: (4 pi / 3) H^3 rho = n_ngb m
 *   av_alpha, av_beta, av_eps   artificial viscosity (Eq. 5-6)
 *   eta_c, eta_a   time-step factors (Eq. 38-39)
 *   h_tol          Newton stop: |g| <= h_tol n_ngb m
 *   max_sweeps     Newton sweeps before SPH_E_NOCONV
 *   h_cap_factor   H is capped at h_cap_factor times the lattice radius
 *   precision      SPH_FP64 or SPH_FP32K (FP32 pair arithmetic on
 *                  cell-relative offsets with compensated sums)
 *   jaumann        SPH_JAUMANN_OBJECTIVE (R S - S R) or _PRINTED (Eq. 25-29)
 *   yield_norm     SPH_YIELD_SQRT_J2 (Eq. 32) or _SQRT_3J2
 *   correction_tensor  1: G = F C (Eq. 22); 0: C = I
 *   gravity        none, uniform g_uniform, or radial table: g_table and
 *                  phi_table are HOST arrays of g_n values on radii
 *                  log-spaced from g_rmin to g_rmax about g_center, copied
 *                  at sph_init; g = g_gm / r^2 beyond g_rmax
 *   periodic       0: open space. 1: periodic box [box_lo, box_hi) on all
 *                  three axes (one system, max_rung = 0, no radial table;
 *                  SPH_E_ARG otherwise, or if a position lies outside the
 *                  box at sph_init): drifted positions wrap back into the
 *                  box, and every pair takes the minimum image, in the
 *                  neighbour predicate (x_i - x_j shifted by a box length
 *                  where |x_i - x_j| > box / 2, as FP64) and in every pair
 *                  term. Each box length must exceed twice the largest
 *                  search radius (about 2.1 H_max); a step that finds a
 *                  narrower box returns SPH_E_CAPACITY.
 *   gradient_form  SPH_GRADIENT_SYMMETRIC: F and C^-1 as Eq. 20-21 (the mean
 *                  of the two kernels, each over its own Omega rho);
 *                  SPH_GRADIENT_ONE_SIDED: the H_i term alone,
 *                  F_i = -sum_j m_j v_ij (x) dW(H_i)/dx_i / (Omega_i rho_i)
 *                  and C_i^-1 likewise with x_ij (the non-symmetric form
 *                  §2.2 mentions beside Eq. 20-21). SPH_E_ARG otherwise.
 *   max_rung       0: one global step per sph_step (dt for every particle).
 *                  1..15: hierarchical individual steps -- sph_step's dt is
 *                  a big step of 2^max_rung substeps; a particle on rung r
 *                  steps dt / 2^r (the smallest r with dt / 2^r within its
 *                  Eq. 38-39 criteria, at most max_rung), is drifted every
 *                  substep, and is solved, given derivatives and kicked only
 *                  at the end of its own steps; neighbours between their
 *                  steps enter with v, u, S predicted linearly to the
 *                  substep time and their last H, rho, Omega. Every
 *                  particle is at time t + dt when the call returns. */
typedef struct {
  int32_t n_ngb;
  double av_alpha, av_beta, av_eps;
  double eta_c, eta_a;
  double h_tol;
  int32_t max_sweeps;
  double h_cap_factor;
  int32_t precision, jaumann, yield_norm, correction_tensor;
  int32_t gravity;
  double g_uniform[3];
  const double *g_table, *phi_table;
  int32_t g_n;
  double g_rmin, g_rmax, g_center[3], g_gm;
  int32_t periodic;
  double box_lo[3], box_hi[3];
  int32_t gradient_form;
  int32_t max_rung;
} sph_params;

/* Per-step report (filled by the synchronising calls). Energies and
 * momenta are FP64 sums over all particles at time i (x_i, v_i, u_i);
 * L = sum m r x v (Eq. 46). dt_next is the minimum of Eq. 38-39.
 * pairs_density counts the in-range pairs evaluated over all Newton sweeps,
 * pairs_force the pairs of the force loop; cand_* count the candidates the
 * two pair kernels staged (work done to find those pairs). With
 * hierarchical steps the counters add up over the substeps, and
 * particle_updates counts the particles kicked (n per step otherwise);
 * rung_counts[r] the moving particles on rung r when the step ends. */
typedef struct {
  double dt, dt_next;
  double e_kin, e_int, e_pot;
  double p[3], L[3];
  int32_t sweeps, n_unconverged, n_capped, n_cfallback;
  int64_t pairs_density, pairs_force;
  uint32_t device_flags;
  int64_t cand_density, cand_force;
  int64_t groups_density, groups_force;  /* lane groups the pair kernels formed */
  int32_t kernel_launches;               /* kernels the call launched */
  int64_t sweeps_total;                  /* Newton sweeps summed over particles */
  int32_t n_expanded;                    /* FP32 form: solves closed by the expansion */
  int64_t particle_updates;              /* particle steps taken (kicks) */
  int32_t rung_counts[16];
} sph_step_info;

/* Report of the tuner (sph_autotune). The pair kernels give each warp a
 * bucket of 32 sorted particles; lanes whose cells lie within `span` cells
 * of one another share one staged candidate list (the tile), which the
 * warp stages `depth` chunks of 32 candidate positions at a time (located
 * and loaded before the first is tested; the list itself does not depend
 * on the depth). */
typedef struct {
  int32_t span_density, span_forces;   /* spans in use */
  int32_t steps_left;                  /* tuning steps still to run (both phases) */
  int32_t n_cand;                      /* span candidates (4 at most) */
  int32_t cand[4];                     /* candidate spans */
  int32_t timed[4];                    /* steps timed per span candidate */
  double ms_density[4], ms_forces[4];  /* summed kernel milliseconds */
  int32_t depth_density, depth_forces; /* staging depths in use */
  int32_t n_depth;                     /* depth candidates (2 at most; 1 in the FP64 form) */
  int32_t depth_cand[2];               /* candidate depths */
  int32_t depth_timed[2];              /* steps timed per depth candidate */
  int32_t reserved_;
  double ms_depth_density[2], ms_depth_forces[2];  /* summed kernel milliseconds */
} sph_tune_report;

/* Create a context for n particles in `st` on `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream). Validates the parameters, copies
 * params, materials and the gravity table, allocates scratch. Does not
 * touch the state. Errors: SPH_E_ARG (n < 1, bad pointer, bad enum, n_mat
 * out of 1..SPH_MAX_MATERIALS, periodic not 0 or 1, a periodic box that is
 * empty or not finite, or one combined with max_rung > 0 or the radial
 * table), SPH_E_CUDA. *out is NULL on failure. */
sph_status sph_init(sph_ctx **out, const sph_params *p, const sph_material *mats,
                    int32_t n_mat, const sph_state *st, int64_t n, void *cuda_stream);

/* A batch of n_sys independent systems in one context (the many uneven
 * impacts of a Q_RD* series, §3.2): system k is the particles with ids in
 * [sys_first[k], sys_first[k+1]) (HOST array of n_sys + 1 values, first 0,
 * last n, increasing; ids must be 0..n-1). Systems never interact: each has
 * its own bounding box, cell grid, time step and sums, and work is split
 * into 32-particle buckets that never straddle two systems, so a system's
 * arithmetic does not depend on the batch around it. One launch of each
 * kernel covers all systems. Radial-table gravity needs n_sys = 1. Errors
 * as sph_init, plus SPH_E_ARG for bad system bounds or n_sys out of
 * 1..SPH_MAX_SYSTEMS. sph_init is this call with one system. */
sph_status sph_init_batch(sph_ctx **out, const sph_params *p, const sph_material *mats,
                          int32_t n_mat, const sph_state *st, int64_t n, int32_t n_sys,
                          const int64_t *sys_first, void *cuda_stream);

/* Cell-list build (replaces the paper's tree walk, §2.1): bounding box, cell
 * size L_c = max H, 30-bit Morton keys of cell coordinates, stable radix sort,
 * in-place permutation of every sph_state array, cell start / end. */
sph_status sph_neighbours(sph_ctx *c);

/* Density and smoothing-length solve (Eq. 1-3) from the current h as first
 * guess; writes h, rho, omega, nngb. Requires a cell list of the current
 * positions. Synchronises; *sweeps (may be NULL) receives the largest
 * Newton sweep count. Returns SPH_E_NOCONV if some particle did not meet
 * h_tol within max_sweeps (its last evaluation is kept). */
sph_status sph_density(sph_ctx *c, int32_t *sweeps);

/* Derivatives of the state as it stands (no prediction): EOS at (rho, u),
 * yield and radial return of a copy of S (Eq. 31-37), the pair loop
 * (Eq. 4-8, 18-22) and the stress rate (Eq. 13 / 25-29). Writes pres, cs,
 * ax..az, dudt, dsxx..dsyz. Requires sph_density on the current cell list.
 * The caller's S is not modified. */
sph_status sph_forces_strength(sph_ctx *c);

/* Closing kick to i (Eq. 41; v and u alike), radial return with Y at
 * (rho_i, u_i), strain invariant (Eq. 43), then opening kick to i+1/2
 * (Eq. 42), all with step dt > 0 and the derivatives in the state. */
sph_status sph_stress_update(sph_ctx *c, double dt);

/* One full step of length dt (dt <= 0: the dt_next of the previous call
 * or, on the first call, of the initial derivatives). The state holds
 * x_{i-1}, v/u/S at i-1/2 and derivatives at i-1 on entry; x_i, v/u/S at
 * i+1/2 and derivatives at i on return. Synchronises and fills *info (may
 * be NULL). */
sph_status sph_step(sph_ctx *c, double dt, sph_step_info *info);

/* One step of every system of a batch, system k with step dt[k] (HOST
 * array of n_sys; dt[k] <= 0: that system's dt_next). *info (may be NULL)
 * receives batch totals: sums over systems, the smallest dt_next, dt of
 * system 0. Synchronises. */
sph_status sph_step_batch(sph_ctx *c, const double *dt, sph_step_info *info);

/* Per-system reports of the last synchronising call, systems 0..n-1. */
sph_status sph_batch_info(const sph_ctx *c, sph_step_info *info, int32_t n);

/* Replay every following sph_step / sph_step_batch from one CUDA graph
 * (on = 1) captured at the first such step on a stream the library owns and
 * ordered after the caller's stream. The graph records the pointers and
 * parameters of sph_init; it is dropped by sph_set_graph and
 * sph_set_timing. on = 0 returns to direct launches. */
sph_status sph_set_graph(sph_ctx *c, int32_t on);

/* Tune the two pair kernels' tiles over the next calls of sph_step /
 * sph_step_batch. First the group span (the cell extent that shares one
 * staged candidate list; candidates 1, 2 and 3 cells) over `rounds` x 3
 * steps; then, in the FP32 form, the staging depth (3 or 4 chunks of 32
 * candidate positions in flight) at the chosen spans over `rounds` x 2
 * steps. Each tuning step runs with one candidate and times both kernels
 * with CUDA events; after the last step of a phase each kernel keeps its
 * fastest candidate and any captured graph is dropped so that the next step
 * captures the tuned launch (sph_tune_info's steps_left counts both phases).
 * Tuning steps are ordinary steps: in the FP64 form their results are
 * bit-identical whatever the span; in the FP32 form the span moves the
 * cell-relative frame, within the form's tolerances, and the depth changes
 * no bit. rounds = 0 stops tuning and keeps the current tiles. Returns
 * SPH_E_ARG for rounds outside 0..64. */
sph_status sph_autotune(sph_ctx *c, int32_t rounds);

/* Set the group spans by hand (1..3 cells each; SPH_E_ARG otherwise) and
 * stop any tuning in progress. Drops a captured graph. */
sph_status sph_set_spans(sph_ctx *c, int32_t span_density, int32_t span_forces);

/* Set the staging depths of the FP32 form's pair kernels by hand (3 or 4
 * each; SPH_E_ARG otherwise; the FP64 form runs 3 in the density solve and
 * 4 in the force pass whatever is set) and stop any tuning in progress.
 * Results do not depend on the depth. Drops a captured graph. */
sph_status sph_set_stage_depths(sph_ctx *c, int32_t depth_density, int32_t depth_forces);

/* The tuner's state and timings. */
sph_status sph_tune_info(const sph_ctx *c, sph_tune_report *out);

/* Measured FMA throughput of the current device. */
typedef struct {
  double tflops;    /* FLOP/s / 1e12, an FMA counting 2 FLOP */
  double ms;        /* average launch duration (CUDA events) */
  double sm_mhz;    /* SM clock during the last launch: cycles / elapsed ns
                       of one block spanning the launch */
  double flops;     /* FLOP per launch */
  int32_t n_sm;     /* multiprocessors the launch covered */
  int32_t pad_;
} sph_peak_report;

/* FMA microbenchmark: one warm-up and then `launches` (1..10000) launches
 * of a kernel whose threads run eight independent FMA chains each, in FP32
 * (precision 1) or FP64 (precision 0), over 4 blocks of 256 threads per
 * multiprocessor. Reports the average launch; the throughput is the peak
 * the pair kernels' ALU roofline compares against at the clock the GPU
 * actually holds. Allocates 64 bytes; synchronises `cuda_stream` (NULL =
 * the legacy default stream). SPH_E_ARG for a bad precision, count or a
 * NULL out. */
sph_status sph_measure_fma_peak(int32_t precision, int32_t launches, sph_peak_report *out,
                                void *cuda_stream);

/* Self-check of the library's own FP64 <-> FP32 conversions (the
 * per-particle kernels convert on the integer pipe, since the conversion
 * instructions run on the FP64 unit): for each of the n DEVICE values, the
 * library's double -> float against the hardware round-to-nearest
 * conversion, and float -> double back, bit for bit. *mismatches (HOST)
 * receives the number of values that differ. Synchronises; allocates 8
 * bytes. */
sph_status sph_check_conversions(const double *in, int64_t n, int64_t *mismatches,
                                 void *cuda_stream);

/* ---------------------------------------------------------------------
 * Learned smoothing-length proposal. The paper's solve (§2.1, Eq. 2-3)
 * starts Newton from the previous support radius; this form starts it from
 * a proposal and leaves the exact solve to decide H and the count. The
 * proposal is made per particle at the end of every step from six features
 * of the converged state (f0 = log(H / H_bar), H_bar = (3 N_ngb m / (4 pi
 * rho0))^(1/3); f1 = n / N_ngb - 1; f2 = log(rho / rho0); f3 = dt tr G,
 * the trace of the corrected velocity gradient of Eq. 18-20; f4 =
 * log(H / H_prev), the previous step's H; f5 = Omega - 1) by a 6-64-64-1
 * network with tanh hidden units and a linear output that predicts
 * log(H_next / H), in bf16 weights with FP32 accumulation on the tensor
 * cores. The predicted ratio is limited to [0.8, 1.25].
 * --------------------------------------------------------------------- */
#define SPH_MLP_NIN 6
#define SPH_MLP_NHID 64
#define SPH_MLP_NPARAM 4673   /* W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3 */
#define SPH_MLP_NNORM 14      /* x_mu[6], x_sd[6], y_mu, y_sd */

enum { SPH_GUESS_PREVIOUS = 0, SPH_GUESS_CONTINUITY = 1, SPH_GUESS_NETWORK = 2 };

typedef struct sph_mlp sph_mlp;   /* opaque network on one device */

/* Create a network with zero parameters on `cuda_stream` (NULL: legacy
 * default stream); every call below runs on that stream. Owns its device
 * memory (about 1.5 MB) until sph_mlp_destroy. SPH_E_CUDA on allocation
 * failure. */
sph_status sph_mlp_create(sph_mlp **out, void *cuda_stream);
sph_status sph_mlp_destroy(sph_mlp *net);
const char *sph_mlp_last_error(const sph_mlp *net);

/* Load parameters (HOST, SPH_MLP_NPARAM floats in the order above) and the
 * normalisation (HOST, SPH_MLP_NNORM floats; standard deviations > 0,
 * SPH_E_ARG otherwise); resets the Adam moments. Synchronises. */
sph_status sph_mlp_set(sph_mlp *net, const float *theta, const float *norm);
/* Copy parameters and normalisation to HOST arrays (either may be NULL). */
sph_status sph_mlp_get(const sph_mlp *net, float *theta, float *norm);
/* Set the normalisation to the means and standard deviations (floored at
 * 1e-6) of m DEVICE samples X (m x 6, row-major) and y (m), skipping
 * samples with a non-finite target. Synchronises. */
sph_status sph_mlp_fit_norm(sph_mlp *net, const float *X, const float *y, int64_t m);
/* Predictions log(H_next / H) of m DEVICE feature rows into DEVICE pred. */
sph_status sph_mlp_forward(sph_mlp *net, const float *X, int64_t m, float *pred);
/* Loss L = 1/(2 m') sum (out - (y - y_mu) / y_sd)^2 over the m' samples
 * with finite features and target among rows idx[0..m) (DEVICE, NULL: rows
 * 0..m), into *loss (HOST); its gradient (SPH_MLP_NPARAM floats) into
 * DEVICE grad when not NULL. Deterministic. Synchronises. */
sph_status sph_mlp_loss_grad(sph_mlp *net, const float *X, const float *y, const int64_t *idx,
                             int64_t m, float *loss, float *grad);
/* One Adam update (Kingma & Ba 2015) with DEVICE gradient grad. */
sph_status sph_mlp_adam_step(sph_mlp *net, const float *grad, float lr, float beta1, float beta2,
                             float eps);
/* One epoch of minibatch Adam (beta 0.9, 0.999, eps 1e-8) over the rows in
 * the order perm (DEVICE, m entries), `batch` rows per update (>= 16);
 * *mean_loss (HOST) the mean of the minibatch losses. */
sph_status sph_mlp_train_epoch(sph_mlp *net, const float *X, const float *y, const int64_t *perm,
                               int64_t m, int32_t batch, float lr, float *mean_loss);

/* Starting radius of the context's smoothing-length solves: guess =
 * SPH_GUESS_PREVIOUS (the paper's), SPH_GUESS_CONTINUITY (H exp(-dt tr G /
 * 3), the continuity equation's estimate) or SPH_GUESS_NETWORK (`net`,
 * which must stay alive while in use). record = 1 keeps, after every step,
 * one training sample per particle (sph_learn_samples). Any mode other than
 * (PREVIOUS, 0) needs ids 0..n-1 (checked: SPH_E_ARG) and allocates about
 * 60 bytes per particle; proposals start one step after the call. Drops a
 * captured graph. */
sph_status sph_set_learned_h(sph_ctx *c, int32_t guess, int32_t record, const sph_mlp *net);
/* The samples of the last step, by particle id: X (DEVICE, n x 6) the
 * features of the step before, y (DEVICE, n) log(H / H_before); rows
 * without a previous step are NaN. SPH_E_STATE unless recording. */
sph_status sph_learn_samples(sph_ctx *c, float *X, float *y);

/* The starting radii that the last step proposed for the next solve:
 * n doubles into the DEVICE array h_next, in the particle order the step
 * left the state arrays in (the sorted order); 0 for a particle without a
 * proposal yet (none is made before the first step after
 * sph_set_learned_h). SPH_E_STATE unless a guess mode other than
 * SPH_GUESS_PREVIOUS is set; ordered on the context's stream. */
sph_status sph_learn_proposal(sph_ctx *c, double *h_next);

/* sph_step with HOST state: the caller passes pinned (for overlap) or
 * pageable host arrays in `host`; the library copies to the context's device
 * state every array the step reads (rho, Omega, P, c_s and the counts are
 * recomputed by the step and are not copied in, except rho, Omega and the
 * counts with hierarchical steps), runs one step with direct
 * launches, and copies each group of arrays back as soon as the step has
 * finished writing it, on a library copy stream that overlaps the rest of
 * the step (positions, masses, ids after the sort; H, rho, Omega after the
 * density solve; P, c_s after the EOS; in a global step the derivatives,
 * counts, v, u, S and strain invariant of each range of the force pass as
 * that range completes, see sph_set_copy_chunks; with hierarchical steps
 * derivatives and counts after the force pass and v, u, S, strain
 * invariant after the kicks). Synchronises. h2d / d2h byte counts go to
 * *bytes_in / *bytes_out (may be NULL). */
sph_status sph_step_host(sph_ctx *c, const sph_state *host, double dt, sph_step_info *info,
                         int64_t *bytes_in, int64_t *bytes_out);

/* Copy-back granularity of sph_step_host with global steps (max_rung = 0):
 * the force pass, which in a global step also applies each particle's
 * closing and opening kicks (§2.4) as soon as its derivatives are formed,
 * runs as `chunks` launches over consecutive ranges of 32-particle buckets
 * (sorted order), and the final state of each range (derivatives, counts,
 * v, u, S, strain invariant) is copied back while the next ranges are
 * computed. chunks = 1 copies those arrays after the whole pass. The
 * results do not depend on it. 1 <= chunks <= SPH_MAX_COPY_CHUNKS, else
 * SPH_E_ARG; the default is 8. Takes effect at the next sph_step_host. */
sph_status sph_set_copy_chunks(sph_ctx *c, int32_t chunks);

/* Derivatives of the initial state: sph_neighbours, sph_density and
 * sph_forces_strength in one call, plus the diagnostics and dt_next in
 * *info (may be NULL). Call once before the first sph_step. */
sph_status sph_prime(sph_ctx *c, sph_step_info *info);

/* Phase timing with CUDA events recorded on the context's stream around the
 * phases of every sph_step: 0 neighbours (drift, keys, sort, permutation,
 * cells), 1 position packing, 2 density solve, 3 prediction (Eq. 40), EOS,
 * yield, radial return and packing, 4 pair loop with finalize (in the
 * global steps of sph_step_host also the kicks, applied per particle in its
 * epilogue), 5 kicks and reductions (the reductions only where the pair
 * loop kicked).
 * sph_set_timing(c, 1) enables it and zeroes the accumulators. Steps
 * replayed from a graph (sph_set_graph) are not phase-timed;
 * sph_phase_times copies up to n accumulated milliseconds per phase into
 * ms and the number of timed steps into *steps (may be NULL). Phase 4
 * includes the learned form's per-step kernel. */
#define SPH_NUM_PHASES 6
sph_status sph_set_timing(sph_ctx *c, int32_t on);
sph_status sph_phase_times(const sph_ctx *c, double *ms, int32_t n, int32_t *steps);

/* Global sums of a particle state with no allocation of any kind. The
 * paper has no counterpart; this is a library service for callers that may
 * not allocate device memory: a host application that has committed the
 * whole device heap to its own allocator or a fixed budget, or a monitoring
 * hook that must leave the device's allocation state untouched between
 * steps. Needs no context: reads x, y, z, vx, vy, vz, u, m of `st` (DEVICE
 * arrays of length n, other pointers may be NULL) and writes 8 doubles to
 * the caller-owned DEVICE array `sums`: kinetic energy, internal energy,
 * linear momentum (3) and angular momentum L = sum m r x v (3), each an
 * FP64 sum over all particles OF THE ARRAYS AS STORED. Between steps the
 * state holds x at time i but v and u at i+1/2 (the kick-drift-kick of
 * §2.4), so these are half-step sums, not the time-i sums of
 * sph_step_info; no potential energy is included. Its scratch is a fixed
 * array compiled into the library (partial sums of at most 1184 blocks,
 * 75,776 bytes, held by every GPU that loads the library until the
 * process exits). Every call made outside a stream capture looks up that
 * array's device address on the current device (so the first call on each
 * device must come before any stream capture: SPH_E_STATE otherwise); a
 * captured call uses the address last looked up. Every call on a device
 * shares the array, so calls that overlap on the GPU (different streams,
 * no ordering) race. An error left pending by earlier work is cleared on
 * entry, so SPH_E_CUDA reports this call's own launches. Ordered on
 * `cuda_stream`; returns after enqueueing. Errors: SPH_E_ARG (NULL
 * pointer, n < 1 or n > SPH_NOALLOC_MAX_N), SPH_E_STATE, SPH_E_CUDA. */
#define SPH_NOALLOC_MAX_N ((int64_t)1 << 31)
sph_status sph_diagnostics_noalloc(const sph_state *st, int64_t n, double *sums,
                                   void *cuda_stream);

/* Host-side fault injection for tests of the error paths: the `after`-th
 * CUDA runtime call that the context checks from now on (1 = the next) is
 * reported as failed with cudaErrorUnknown although it succeeded, exactly as
 * a real failure of that call would be: the calling entry point returns
 * SPH_E_CUDA (work it enqueued before that call stays enqueued and runs to
 * completion) and every later call on the context returns SPH_E_STATE until
 * sph_destroy. Nothing is done to the GPU. after = 0 cancels a pending
 * injection; SPH_E_ARG for after < 0. */
sph_status sph_inject_cuda_failure(sph_ctx *c, int32_t after);

/* Free the context and its scratch; the caller's arrays are untouched.
 * Accepts NULL. */
sph_status sph_destroy(sph_ctx *c);

/* Static description of a status code. */
const char *sph_status_string(sph_status s);

/* Detail of the last failure on this context ("" if none). */
const char *sph_last_error(const sph_ctx *c);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
