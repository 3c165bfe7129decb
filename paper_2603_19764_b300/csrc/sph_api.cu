// sph_api.cu -- the extern "C" entry points of include/sph.h: context
// set-up, validation, scratch ownership, the call sequences of one step
// (§2.4) and status reporting.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_internal.cuh"

using namespace sphk;

namespace {

sph_status fail(sph_ctx *c, sph_status s, const char *msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
  return s;
}

sph_status fail_cuda(sph_ctx *c, cudaError_t e, const char *what) {
  if (c) {
    snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
    c->broken = 1;
  }
  return SPH_E_CUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return fail_cuda(c, e_, #call); \
  } while (0)

#define ENTER(c)                                                                 \
  do {                                                                           \
    if (!(c)) return SPH_E_ARG;                                                  \
    if ((c)->broken) return fail(c, SPH_E_STATE, "context unusable after a CUDA error"); \
  } while (0)

template <typename T> cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

bool state_complete(const sph_state *s) {
  const void *p[] = {s->x,    s->y,    s->z,    s->vx,    s->vy,     s->vz,   s->u,    s->m,
                     s->h,    s->sxx,  s->syy,  s->sxy,   s->sxz,    s->syz,  s->rho,  s->omega,
                     s->pres, s->cs,   s->ax,   s->ay,    s->az,     s->dudt, s->dsxx, s->dsyy,
                     s->dsxy, s->dsxz, s->dsyz, s->eps_ii, s->nngb,  s->mat,  s->flags, s->id};
  for (const void *q : p)
    if (!q) return false;
  return true;
}

// Validation of the device state at set-up: material index in range,
// positive mass and H, finite positions.
__global__ void k_validate(sph_state s, int64_t n, int nmat, unsigned *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool ok = s.mat[i] >= 0 && s.mat[i] < nmat && s.m[i] > 0.0 && s.h[i] > 0.0 &&
                    isfinite(s.x[i]) && isfinite(s.y[i]) && isfinite(s.z[i]) && isfinite(s.h[i]);
    if (!ok) atomicOr(bad, 1u);
  }
}

void free_all(sph_ctx *c) {
  void *dev[] = {c->d_mats, c->d_gtab, c->d_phitab, c->d_radii, c->w.vp[0], c->w.vp[1],
                 c->w.vp[2], c->w.up, c->w.sp[0], c->w.sp[1], c->w.sp[2], c->w.sp[3],
                 c->w.sp[4], c->w.vsig, c->w.edot2, c->w.yld, c->w.cc, c->w.pos32, c->w.pos64,
                 c->w.fj32[0], c->w.fj32[1], c->w.fj32[2], c->w.fj32[3], c->w.fj64[0],
                 c->w.fj64[1], c->w.fj64[2], c->w.fj64[3], c->w.posh32, c->w.posh64,
                 c->w.fs32[0], c->w.fs32[1], c->w.fs32[2], c->w.fs64[0], c->w.fs64[1],
                 c->w.fs64[2], c->keys, c->keys_alt, c->vals, c->vals_alt, c->hist, c->scan_tot,
                 c->cell_start, c->cell_end, c->tmp, c->partials, c->d_dt, c->d_status};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_dt) cudaFreeHost(c->h_dt);
}

sph_status status_from_flags(sph_ctx *c, unsigned flags) {
  if (flags & ERR_NONFINITE) return fail(c, SPH_E_NONFINITE, "non-finite density or derivative");
  if (flags & ERR_TIMEOUT) return fail(c, SPH_E_TIMEOUT, "device wait timed out");
  if (flags & ERR_CAPACITY) return fail(c, SPH_E_CAPACITY, "scratch capacity exceeded");
  if (flags & ERR_NOCONV) return fail(c, SPH_E_NOCONV, "smoothing-length solve did not converge");
  return SPH_OK;
}

// Copy the device record to the host, wait, clear the latched error word.
sph_status sync_status(sph_ctx *c, sph_step_info *info, double dt) {
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(Status), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(&c->d_status->err, 0, sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const Status &h = *c->h_status;
  const double dtn = dec_d(h.dtmin_enc);
  if (h.dtmin_enc != ~0ull && dtn > 0.0) c->dt_next = dtn;
  if (info) {
    info->dt = dt;
    info->dt_next = c->dt_next;
    info->e_kin = h.sums[0];
    info->e_int = h.sums[1];
    info->e_pot = h.sums[2];
    for (int k = 0; k < 3; ++k) {
      info->p[k] = h.sums[3 + k];
      info->L[k] = h.sums[6 + k];
    }
    info->sweeps = h.max_sweeps;
    info->n_unconverged = h.n_unconv;
    info->n_capped = h.n_capped;
    info->n_cfallback = h.n_cfallback;
    info->pairs_density = (int64_t)h.pairs_density;
    info->pairs_force = (int64_t)h.pairs_force;
    info->cand_density = (int64_t)h.cand_density;
    info->cand_force = (int64_t)h.cand_force;
    info->groups_density = (int64_t)h.groups_density;
    info->groups_force = (int64_t)h.groups_force;
    info->device_flags = h.err;
  }
  return status_from_flags(c, h.err);
}

sph_status set_dt(sph_ctx *c, double dt) {
  *c->h_dt = dt;
  CK(cudaMemcpyAsync(c->d_dt, c->h_dt, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return SPH_OK;
}

// Phase marker k (0..SPH_NUM_PHASES) when timing is on.
cudaError_t mark(sph_ctx *c, int k) {
  return c->timing ? cudaEventRecord(c->ev[k], c->stream) : cudaSuccess;
}

sph_status run_neighbours(sph_ctx *c, int drift) {
  CK(mark(c, 0));
  CK(launch_reset_status(c, 0));
  CK(launch_drift_bbox(c, drift));
  CK(launch_grid_setup(c));
  CK(launch_sort_permute(c));
  CK(mark(c, 1));
  return SPH_OK;
}

sph_status run_derivatives(sph_ctx *c, int predict) {
  CK(launch_predict_pack(c, predict));
  CK(mark(c, 2));
  CK(launch_density(c));
  CK(mark(c, 3));
  CK(launch_eos_pack(c));
  CK(mark(c, 4));
  CK(launch_forces(c));
  CK(mark(c, 5));
  return SPH_OK;
}

// Accumulate the phase times of the step just synchronised.
sph_status collect_times(sph_ctx *c) {
  if (!c->timing) return SPH_OK;
  for (int k = 0; k < SPH_NUM_PHASES; ++k) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
    c->phase_ms[k] += ms;
  }
  c->timed_steps += 1;
  return SPH_OK;
}

}  // namespace

extern "C" {

const char *sph_status_string(sph_status s) {
  switch (s) {
    case SPH_OK: return "ok";
    case SPH_E_ARG: return "invalid argument";
    case SPH_E_CUDA: return "CUDA error";
    case SPH_E_NOCONV: return "smoothing-length solve did not converge";
    case SPH_E_CAPACITY: return "scratch capacity exceeded";
    case SPH_E_NONFINITE: return "non-finite result";
    case SPH_E_TIMEOUT: return "device wait timed out";
    case SPH_E_STATE: return "context unusable";
  }
  return "unknown status";
}

const char *sph_last_error(const sph_ctx *c) { return c ? c->err : "no context"; }

sph_status sph_init(sph_ctx **out, const sph_params *p, const sph_material *mats, int32_t n_mat,
                    const sph_state *st, int64_t n, void *cuda_stream) {
  if (!out) return SPH_E_ARG;
  *out = nullptr;
  if (!p || !mats || !st || n < 1 || n > (int64_t)1 << 30) return SPH_E_ARG;
  if (n_mat < 1 || n_mat > SPH_MAX_MATERIALS || !state_complete(st)) return SPH_E_ARG;
  if (p->precision != SPH_FP64 && p->precision != SPH_FP32K) return SPH_E_ARG;
  if (p->jaumann != SPH_JAUMANN_OBJECTIVE && p->jaumann != SPH_JAUMANN_PRINTED) return SPH_E_ARG;
  if (p->yield_norm != SPH_YIELD_SQRT_J2 && p->yield_norm != SPH_YIELD_SQRT_3J2) return SPH_E_ARG;
  if (p->gravity < SPH_GRAVITY_NONE || p->gravity > SPH_GRAVITY_RADIAL) return SPH_E_ARG;
  if (p->periodic != 0) return SPH_E_ARG;
  if (!(p->n_ngb >= 1) || !(p->h_tol > 0.0) || p->max_sweeps < 1 || !(p->h_cap_factor > 0.0))
    return SPH_E_ARG;
  if (p->gravity == SPH_GRAVITY_RADIAL &&
      (!p->g_table || !p->phi_table || p->g_n < 2 || !(p->g_rmin > 0.0) || !(p->g_rmax > p->g_rmin)))
    return SPH_E_ARG;
  for (int k = 0; k < n_mat; ++k)
    if (!(mats[k].rho0 > 0.0) || (mats[k].eos != SPH_EOS_LINEAR && mats[k].eos != SPH_EOS_TILLOTSON))
      return SPH_E_ARG;

  sph_ctx *c = (sph_ctx *)calloc(1, sizeof(sph_ctx));
  if (!c) return SPH_E_ARG;
  c->params = *p;
  for (int k = 0; k < SPH_MAX_MATERIALS; ++k) c->mats[k] = mats[k < n_mat ? k : n_mat - 1];
  c->nmat = n_mat;
  c->st = *st;
  c->n = n;
  c->stream = (cudaStream_t)cuda_stream;
  const bool fp32 = p->precision == SPH_FP32K;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        c->num_sms < 1) {
      free(c);
      return SPH_E_CUDA;
    }
  }

#define CKI(call)                          \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) {               \
      free_all(c);                         \
      free(c);                             \
      return SPH_E_CUDA;                   \
    }                                      \
  } while (0)

  CKI(dalloc(&c->d_mats, SPH_MAX_MATERIALS));
  CKI(cudaMemcpy(c->d_mats, c->mats, sizeof(c->mats), cudaMemcpyHostToDevice));
  KParams &kp = c->kp;
  kp.n_ngb = p->n_ngb;
  kp.av_alpha = p->av_alpha;
  kp.av_beta = p->av_beta;
  kp.av_eps = p->av_eps;
  kp.eta_c = p->eta_c;
  kp.eta_a = p->eta_a;
  kp.h_tol = p->h_tol;
  kp.max_sweeps = p->max_sweeps;
  kp.h_cap_factor = p->h_cap_factor;
  kp.precision = p->precision;
  kp.jaumann = p->jaumann;
  kp.yield_norm = p->yield_norm;
  kp.correction = p->correction_tensor;
  kp.gravity = p->gravity;
  for (int a = 0; a < 3; ++a) {
    kp.g_uniform[a] = p->g_uniform[a];
    kp.g_center[a] = p->g_center[a];
  }
  kp.mats = c->d_mats;
  if (p->gravity == SPH_GRAVITY_RADIAL) {
    const int gn = p->g_n;
    double *radii = (double *)malloc(sizeof(double) * gn);
    for (int k = 0; k < gn; ++k)
      radii[k] = p->g_rmin * pow(p->g_rmax / p->g_rmin, (double)k / (double)(gn - 1));
    CKI(dalloc(&c->d_gtab, gn));
    CKI(dalloc(&c->d_phitab, gn));
    CKI(dalloc(&c->d_radii, gn));
    CKI(cudaMemcpy(c->d_gtab, p->g_table, sizeof(double) * gn, cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(c->d_phitab, p->phi_table, sizeof(double) * gn, cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(c->d_radii, radii, sizeof(double) * gn, cudaMemcpyHostToDevice));
    free(radii);
    kp.g_table = c->d_gtab;
    kp.phi_table = c->d_phitab;
    kp.g_radii = c->d_radii;
    kp.g_n = gn;
    kp.g_rmin = p->g_rmin;
    kp.g_rmax = p->g_rmax;
    kp.g_gm = p->g_gm;
    kp.g_inv_log_ratio = (double)(gn - 1) / log2(p->g_rmax / p->g_rmin);
  }
  c->params.g_table = c->d_gtab;
  c->params.phi_table = c->d_phitab;

  Work &w = c->w;
  for (int k = 0; k < 3; ++k) CKI(dalloc(&w.vp[k], n));
  CKI(dalloc(&w.up, n));
  for (int k = 0; k < 5; ++k) CKI(dalloc(&w.sp[k], n));
  CKI(dalloc(&w.vsig, n));
  CKI(dalloc(&w.edot2, n));
  CKI(dalloc(&w.yld, n));
  CKI(dalloc(&w.cc, n));
  if (fp32) {
    CKI(dalloc(&w.pos32, n));
    CKI(dalloc(&w.posh32, n));
    for (int k = 0; k < 4; ++k) CKI(dalloc(&w.fj32[k], n));
    for (int k = 0; k < 3; ++k) CKI(dalloc(&w.fs32[k], n));
  } else {
    CKI(dalloc(&w.pos64, n));
    CKI(dalloc(&w.posh64, n));
    for (int k = 0; k < 4; ++k) CKI(dalloc(&w.fj64[k], n));
    for (int k = 0; k < 3; ++k) CKI(dalloc(&w.fs64[k], n));
  }
  CKI(dalloc(&c->keys, n));
  CKI(dalloc(&c->keys_alt, n));
  CKI(dalloc(&c->vals, n));
  CKI(dalloc(&c->vals_alt, n));
  c->ntiles = (int)((n + 2047) / 2048);
  CKI(dalloc(&c->hist, (size_t)256 * c->ntiles));
  CKI(dalloc(&c->scan_tot, (size_t)(256 * c->ntiles + 1023) / 1024 + 1));
  int64_t mc = 2 * n;
  if (mc < 4096) mc = 4096;
  if (mc > (1 << 24)) mc = 1 << 24;
  c->max_cells = (int)mc;
  CKI(dalloc(&c->cell_start, mc));
  CKI(dalloc(&c->cell_end, mc));
  CKI(cudaMalloc(&c->tmp, (size_t)n * 32 * 8));
  int64_t rb = (n + kBlock - 1) / kBlock;
  if (rb > 148 * 8) rb = 148 * 8;
  c->nred_blocks = (int)rb;
  CKI(dalloc(&c->partials, (size_t)rb * 9));
  CKI(dalloc(&c->d_dt, 1));
  CKI(dalloc(&c->d_status, 1));
  CKI(cudaMemset(c->d_status, 0, sizeof(Status)));
  CKI(cudaMallocHost((void **)&c->h_status, sizeof(Status)));
  CKI(cudaMallocHost((void **)&c->h_dt, sizeof(double)));
  // validate the caller's state once
  unsigned *bad = nullptr;
  CKI(dalloc(&bad, 1));
  CKI(cudaMemset(bad, 0, sizeof(unsigned)));
  k_validate<<<148 * 4, kBlock, 0, c->stream>>>(c->st, n, n_mat, bad);
  unsigned hbad = 0;
  CKI(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CKI(cudaStreamSynchronize(c->stream));
  cudaFree(bad);
  if (hbad) {
    free_all(c);
    free(c);
    return SPH_E_ARG;
  }
  *out = c;
  return SPH_OK;
#undef CKI
}

sph_status sph_set_timing(sph_ctx *c, int32_t on) {
  ENTER(c);
  if (on && !c->timing) {
    for (int k = 0; k <= SPH_NUM_PHASES; ++k) CK(cudaEventCreate(&c->ev[k]));
  }
  if (!on && c->timing) {
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k <= SPH_NUM_PHASES; ++k) cudaEventDestroy(c->ev[k]);
  }
  c->timing = on ? 1 : 0;
  for (int k = 0; k < SPH_NUM_PHASES; ++k) c->phase_ms[k] = 0.0;
  c->timed_steps = 0;
  return SPH_OK;
}

sph_status sph_phase_times(const sph_ctx *c, double *ms, int32_t n, int32_t *steps) {
  if (!c || (!ms && n > 0) || n < 0) return SPH_E_ARG;
  for (int k = 0; k < n && k < SPH_NUM_PHASES; ++k) ms[k] = c->phase_ms[k];
  if (steps) *steps = c->timed_steps;
  return SPH_OK;
}

sph_status sph_destroy(sph_ctx *c) {
  if (!c) return SPH_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->timing)
    for (int k = 0; k <= SPH_NUM_PHASES; ++k) cudaEventDestroy(c->ev[k]);
  free_all(c);
  free(c);
  return SPH_OK;
}

sph_status sph_neighbours(sph_ctx *c) {
  ENTER(c);
  return run_neighbours(c, 0);
}

sph_status sph_density(sph_ctx *c, int32_t *sweeps) {
  ENTER(c);
  CK(launch_predict_pack(c, 0));
  CK(launch_density(c));
  sph_step_info info;
  const sph_status s = sync_status(c, &info, 0.0);
  if (sweeps) *sweeps = info.sweeps;
  return s;
}

sph_status sph_forces_strength(sph_ctx *c) {
  ENTER(c);
  CK(launch_predict_pack(c, 0));
  CK(launch_eos_pack(c));
  CK(launch_forces(c));
  return SPH_OK;
}

sph_status sph_stress_update(sph_ctx *c, double dt) {
  ENTER(c);
  if (!(dt > 0.0)) return fail(c, SPH_E_ARG, "dt must be positive");
  sph_status s = set_dt(c, dt);
  if (s != SPH_OK) return s;
  CK(launch_kick(c, 1));
  return SPH_OK;
}

sph_status sph_prime(sph_ctx *c, sph_step_info *info) {
  ENTER(c);
  sph_status s = run_neighbours(c, 0);
  if (s != SPH_OK) return s;
  s = run_derivatives(c, 0);
  if (s != SPH_OK) return s;
  CK(launch_kick(c, 0));
  s = sync_status(c, info, 0.0);
  if (s == SPH_OK || s == SPH_E_NOCONV) c->primed = 1;
  return s;
}

sph_status sph_step(sph_ctx *c, double dt, sph_step_info *info) {
  ENTER(c);
  if (!(dt > 0.0)) {
    if (!c->primed || !(c->dt_next > 0.0))
      return fail(c, SPH_E_STATE, "dt <= 0 needs a dt_next from sph_prime or an earlier step");
    dt = c->dt_next;
  }
  sph_status s = set_dt(c, dt);
  if (s != SPH_OK) return s;
  s = run_neighbours(c, 1);
  if (s != SPH_OK) return s;
  s = run_derivatives(c, 1);
  if (s != SPH_OK) return s;
  CK(launch_kick(c, 1));
  CK(mark(c, 6));
  s = sync_status(c, info, dt);
  const sph_status t = collect_times(c);
  return s != SPH_OK ? s : t;
}

sph_status sph_step_host(sph_ctx *c, const sph_state *host, double dt, sph_step_info *info,
                         int64_t *bytes_in, int64_t *bytes_out) {
  ENTER(c);
  if (!host || !state_complete(host)) return fail(c, SPH_E_ARG, "incomplete host state");
  const sph_state &d = c->st;
  const int64_t n = c->n;
  double *const hd[28] = {host->x,    host->y,    host->z,     host->vx,    host->vy,   host->vz,
                          host->u,    host->m,    host->h,     host->sxx,   host->syy,  host->sxy,
                          host->sxz,  host->syz,  host->rho,   host->omega, host->pres, host->cs,
                          host->ax,   host->ay,   host->az,    host->dudt,  host->dsxx, host->dsyy,
                          host->dsxy, host->dsxz, host->dsyz,  host->eps_ii};
  double *const dd[28] = {d.x,    d.y,    d.z,     d.vx,    d.vy,   d.vz,   d.u,    d.m,
                          d.h,    d.sxx,  d.syy,   d.sxy,   d.sxz,  d.syz,  d.rho,  d.omega,
                          d.pres, d.cs,   d.ax,    d.ay,    d.az,   d.dudt, d.dsxx, d.dsyy,
                          d.dsxy, d.dsxz, d.dsyz,  d.eps_ii};
  int32_t *const hi[3] = {host->nngb, host->mat, host->flags};
  int32_t *const di[3] = {d.nngb, d.mat, d.flags};
  const size_t b8 = sizeof(double) * (size_t)n, b4 = sizeof(int32_t) * (size_t)n;
  for (int k = 0; k < 28; ++k) CK(cudaMemcpyAsync(dd[k], hd[k], b8, cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(di[k], hi[k], b4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.id, host->id, b8, cudaMemcpyHostToDevice, c->stream));
  const sph_status s = sph_step(c, dt, info);
  for (int k = 0; k < 28; ++k) CK(cudaMemcpyAsync(hd[k], dd[k], b8, cudaMemcpyDeviceToHost, c->stream));
  for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(hi[k], di[k], b4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(host->id, d.id, b8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const int64_t bytes = 29 * (int64_t)b8 + 3 * (int64_t)b4;
  if (bytes_in) *bytes_in = bytes;
  if (bytes_out) *bytes_out = bytes;
  return s;
}

}  // extern "C"
