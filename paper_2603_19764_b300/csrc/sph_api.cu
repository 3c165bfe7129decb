// sph_api.cu -- the extern "C" entry points of include/sph.h: context
// set-up, validation, scratch ownership, the call sequences of one step
// (§2.4), batches of independent systems, CUDA-graph replay of the step and
// status reporting.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph_kick.cuh"

using namespace sphk;

namespace {

// Host-side trace ranges (NVTX, header-only): inert unless a profiler or
// tracer attaches. They mark where each call and phase is enqueued -- with
// direct launches, the kernels that follow; under stream capture, the
// capture itself.
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

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

// A checked CUDA runtime call. An injected failure (sph_inject_cuda_failure)
// turns the chosen successful call into cudaErrorUnknown.
inline cudaError_t injected(sph_ctx *c, cudaError_t e) {
  if (e == cudaSuccess && c && c->fail_after > 0 && --c->fail_after == 0) return cudaErrorUnknown;
  return e;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = injected(c, (call));                 \
    if (e_ != cudaSuccess) return fail_cuda(c, e_, #call); \
  } while (0)

// Entry of a context call. An error that earlier, unrelated work left
// pending (not sticky) is cleared, so that the launch checks of this call
// report its own launches.
#define ENTER(c)                                                                 \
  do {                                                                           \
    if (!(c)) return SPH_E_ARG;                                                  \
    if ((c)->broken) return fail(c, SPH_E_STATE, "context unusable after a CUDA error"); \
    (c)->nlaunch = 0;                                                            \
    (void)cudaGetLastError();                                                    \
  } while (0)

template <typename T> cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

// A material's parameters and derived constants in the type of a form.
template <typename T> MatT<T> mat_copy(const sph_material &m) {
  MatT<T> o;
  memset(&o, 0, sizeof(o));
  o.eos = m.eos;
  o.strength = m.strength;
  o.thermal_softening = m.thermal_softening;
  o.rho0_d = m.rho0;
  o.Eiv_d = m.Eiv;
  o.Ecv_d = m.Ecv;
  o.c0sq_d = m.c0 * m.c0;
  o.p_min_d = m.p_min;
  o.rho0 = (T)m.rho0;
  o.inv_rho0 = (T)(1.0 / m.rho0);
  o.c0 = (T)m.c0;
  o.c0sq = (T)(m.c0 * m.c0);
  o.A = (T)m.A;
  o.B = (T)m.B;
  o.E0 = (T)m.E0;
  o.a = (T)m.a;
  o.b = (T)m.b;
  o.alpha = (T)m.alpha;
  o.beta = (T)m.beta;
  o.inv_dE = m.Ecv > m.Eiv ? (T)(1.0 / (m.Ecv - m.Eiv)) : (T)0;
  o.floor2 = (T)(0.01 * m.A / m.rho0);
  o.shear_G = (T)m.shear_G;
  o.Y0 = (T)m.Y0;
  o.mu_i = (T)m.mu_i;
  o.Ym = (T)m.Ym;
  o.mu_d = (T)m.mu_d;
  o.xi = (T)m.xi;
  o.Tm = (T)m.Tm;
  o.T0 = (T)m.T0;
  o.inv_cv = (T)(1.0 / m.cv);
  o.p_min = (T)m.p_min;
  return o;
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
// positive mass and H, finite positions; in a batch, ids in 0..n-1.
// In a periodic box every position must lie in [box_lo, box_hi).
__global__ void k_validate(sph_state s, int64_t n, int nmat, int check_id, KParams P,
                           unsigned *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool ok = s.mat[i] >= 0 && s.mat[i] < nmat && s.m[i] > 0.0 && s.h[i] > 0.0 &&
              isfinite(s.x[i]) && isfinite(s.y[i]) && isfinite(s.z[i]) && isfinite(s.h[i]);
    if (check_id) ok = ok && s.id[i] >= 0 && s.id[i] < n;
    if (P.periodic) {
      const double c[3] = {s.x[i], s.y[i], s.z[i]};
      for (int a = 0; a < 3; ++a) ok = ok && c[a] >= P.box_lo[a] && c[a] < P.box_hi[a];
    }
    if (!ok) atomicOr(bad, 1u);
  }
}

void free_all(sph_ctx *c) {
  void *dev[] = {c->d_mats, c->d_matf, c->d_matd, c->d_gtab, c->d_phitab, c->d_radii,
                 c->d_gtab_f, c->w.vsig, c->w.edot2, c->w.yld, c->w.cc, c->w.pos32, c->w.pos64,
                 c->w.fj32, c->w.fj64, c->w.posh32, c->w.posh64,
                 c->w.fs32[0], c->w.fs32[1], c->w.fs32[2], c->w.fs64[0], c->w.fs64[1],
                 c->w.fs64[2], c->keys, c->keys_alt, c->vals, c->vals_alt, c->hist, c->scan_tot,
                 c->cell_start, c->cell_end, c->tmp, c->d_dt, c->d_status,
                 c->d_sys, c->d_sys_begin, c->d_sys_bucket, c->d_red_tile, c->w.tcrit,
                 c->w.terms[0], c->w.terms[1], c->w.terms[2], c->w.terms[3], c->w.terms[4],
                 c->w.terms[5], c->w.terms[6], c->w.terms[7], c->w.terms[8],
                 c->tile_partials, c->d_chunk_ctr, c->w.divv,
                 c->learn.hprev, c->learn.hprop, c->learn.feat[0], c->learn.feat[1],
                 c->learn.feat[2], c->learn.x_out, c->learn.y_out, c->dens_spill, c->w.rung,
                 c->w.act, c->w.act_tiles};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_sys) cudaFreeHost(c->h_sys);
  if (c->h_dt) cudaFreeHost(c->h_dt);
  free(c->sys_first);
  free(c->dt_next);
}

sph_status status_from_flags(sph_ctx *c, unsigned flags) {
  if (flags & ERR_BOUNDS)
    return fail(c, SPH_E_INTERNAL, "an index check of the checked build failed");
  if (flags & ERR_NONFINITE) return fail(c, SPH_E_NONFINITE, "non-finite density or derivative");
  if (flags & ERR_TIMEOUT) return fail(c, SPH_E_TIMEOUT, "device wait timed out");
  if (flags & ERR_CAPACITY)
    return fail(c, SPH_E_CAPACITY, "periodic box not wider than twice a search radius");
  if (flags & ERR_NOCONV) return fail(c, SPH_E_NOCONV, "smoothing-length solve did not converge");
  return SPH_OK;
}

// Enqueue the copies of the device records to their pinned mirrors and the
// clearing of the latched error word.
sph_status enqueue_status_readback(sph_ctx *c) {
  CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(Status), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(c->h_sys, c->d_sys, sizeof(SysRec) * c->nsys, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemsetAsync(&c->d_status->err, 0, sizeof(unsigned), c->stream));
  return SPH_OK;
}

// Report of system `sys` (sys < 0: totals over the batch).
void fill_info(const sph_ctx *c, int sys, sph_step_info *info) {
  const Status &h = *c->h_status;
  memset(info, 0, sizeof(*info));
  const int k0 = sys < 0 ? 0 : sys, k1 = sys < 0 ? c->nsys : sys + 1;
  info->dt = c->h_dt[k0];
  info->dt_next = INFINITY;
  for (int k = k0; k < k1; ++k) {
    const SysRec &r = c->h_sys[k];
    info->e_kin += r.sums[0];
    info->e_int += r.sums[1];
    info->e_pot += r.sums[2];
    for (int a = 0; a < 3; ++a) {
      info->p[a] += r.sums[3 + a];
      info->L[a] += r.sums[6 + a];
    }
    if (c->dt_next[k] < info->dt_next) info->dt_next = c->dt_next[k];
  }
  // counters are kept for the whole batch only
  info->sweeps = h.max_sweeps;
  info->n_unconverged = h.n_unconv;
  info->n_capped = h.n_capped;
  info->n_cfallback = h.n_cfallback;
  info->pairs_density = (int64_t)h.pairs_density;
  info->pairs_force = (int64_t)h.pairs_force;
  info->device_flags = h.err;
  info->cand_density = (int64_t)h.cand_density;
  info->cand_force = (int64_t)h.cand_force;
  info->groups_density = (int64_t)h.groups_density;
  info->groups_force = (int64_t)h.groups_force;
  info->kernel_launches = c->nlaunch;
  info->sweeps_total = (int64_t)h.sweeps_total;
  info->n_expanded = h.n_expanded;
  info->particle_updates = (int64_t)h.updates;
  for (int r = 0; r < 16; ++r) info->rung_counts[r] = h.rung_hist[r];
  if (c->rungs == 0) info->rung_counts[0] = (int32_t)h.updates;   // one global step
}

// After a synchronisation: per-system dt_next from the mirrors, the report,
// the status.
sph_status finish_sync(sph_ctx *c, sph_step_info *info) {
  for (int k = 0; k < c->nsys; ++k) {
    const unsigned long long e = c->h_sys[k].dtmin_enc;
    const double dtn = dec_d(e);
    if (e != ~0ull && dtn > 0.0) c->dt_next[k] = dtn;
  }
  if (info) fill_info(c, -1, info);
  return status_from_flags(c, c->h_status->err);
}

sph_status sync_status(sph_ctx *c, sph_step_info *info) {
  sph_status s = enqueue_status_readback(c);
  if (s != SPH_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  return finish_sync(c, info);
}

sph_status upload_dt(sph_ctx *c) {
  CK(cudaMemcpyAsync(c->d_dt, c->h_dt, sizeof(double) * c->nsys, cudaMemcpyHostToDevice,
                     c->stream));
  return SPH_OK;
}

// Phase marker k (0..SPH_NUM_PHASES) when timing is on. Steps replayed
// from a graph are not phase-timed (events recorded by graph nodes give no
// elapsed times), so nothing is recorded while capturing.
cudaError_t mark(sph_ctx *c, int k) {
  return c->timing && !c->capturing ? cudaEventRecord(c->ev[k], c->stream) : cudaSuccess;
}

// Copy-out of sph_step_host, overlapped with the rest of the step: group g
// of the state is final once the phase before this call has run (0: after
// the sort -- positions, masses, ids, materials, flags; 1: after the
// density solve -- H, rho, Omega; 2: after the EOS -- P, c_s; 3: after the
// force pass -- derivatives and counts; 4: after the kicks -- v, u, S and
// the strain invariant).
sph_status copy_out(sph_ctx *c, int g) {
  if (!c->host_out || c->capturing) return SPH_OK;
  const sph_state &d = c->st, &h = *c->host_out;
  const size_t b8 = sizeof(double) * (size_t)c->n, b4 = sizeof(int32_t) * (size_t)c->n;
  CK(cudaEventRecord(c->out_ev[g], c->stream));
  CK(cudaStreamWaitEvent(c->cstream, c->out_ev[g], 0));
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->cstream);
  };
  switch (g) {
    case 0:
      CK(cp(h.x, d.x, b8)); CK(cp(h.y, d.y, b8)); CK(cp(h.z, d.z, b8)); CK(cp(h.m, d.m, b8));
      CK(cp(h.id, d.id, b8)); CK(cp(h.mat, d.mat, b4)); CK(cp(h.flags, d.flags, b4));
      break;
    case 1:
      CK(cp(h.h, d.h, b8)); CK(cp(h.rho, d.rho, b8)); CK(cp(h.omega, d.omega, b8));
      break;
    case 2:
      CK(cp(h.pres, d.pres, b8)); CK(cp(h.cs, d.cs, b8));
      break;
    case 3:
      CK(cp(h.ax, d.ax, b8)); CK(cp(h.ay, d.ay, b8)); CK(cp(h.az, d.az, b8));
      CK(cp(h.dudt, d.dudt, b8)); CK(cp(h.dsxx, d.dsxx, b8)); CK(cp(h.dsyy, d.dsyy, b8));
      CK(cp(h.dsxy, d.dsxy, b8)); CK(cp(h.dsxz, d.dsxz, b8)); CK(cp(h.dsyz, d.dsyz, b8));
      CK(cp(h.nngb, d.nngb, b4));
      break;
    default:
      CK(cp(h.vx, d.vx, b8)); CK(cp(h.vy, d.vy, b8)); CK(cp(h.vz, d.vz, b8)); CK(cp(h.u, d.u, b8));
      CK(cp(h.sxx, d.sxx, b8)); CK(cp(h.syy, d.syy, b8)); CK(cp(h.sxy, d.sxy, b8));
      CK(cp(h.sxz, d.sxz, b8)); CK(cp(h.syz, d.syz, b8)); CK(cp(h.eps_ii, d.eps_ii, b8));
      break;
  }
  return SPH_OK;
}

// First sorted position of bucket b (the bucket count: n). Buckets are 32
// consecutive positions of one system, the systems' buckets in order.
int64_t bucket_first(const sph_ctx *c, int b) {
  int64_t off = 0;
  for (int k = 0; k < c->nsys; ++k) {
    const int64_t nb = (c->sys_first[k + 1] - c->sys_first[k] + 31) / 32;
    if (b < off + nb) return c->sys_first[k] + 32 * (b - off);
    off += nb;
  }
  return c->n;
}

// Force pass of a global step of sph_step_host in copy_chunks launches over
// consecutive bucket ranges (the force pass kicks, so a range's state is
// final when its launch completes), alternating between two streams so
// that one launch's last buckets overlap the next launch's first; each
// range's derivatives, counts, v, u, S and strain invariant are copied back
// on the copy stream as soon as its launch completes.
sph_status forces_chunked(sph_ctx *c) {
  const int K = c->copy_chunks;
  const int nb = c->kp.nbuckets;
  const sph_state &d = c->st, &h = *c->host_out;
  CK(cudaMemsetAsync(c->d_chunk_ctr, 0, sizeof(unsigned) * K, c->stream));
  CK(cudaEventRecord(c->ev_pre, c->stream));
  CK(cudaStreamWaitEvent(c->fstream[0], c->ev_pre, 0));
  CK(cudaStreamWaitEvent(c->fstream[1], c->ev_pre, 0));
  double *const hd[19] = {h.ax,  h.ay,  h.az,  h.dudt, h.dsxx, h.dsyy, h.dsxy, h.dsxz, h.dsyz, h.vx,
                          h.vy,  h.vz,  h.u,   h.sxx,  h.syy,  h.sxy,  h.sxz,  h.syz,  h.eps_ii};
  double *const dd[19] = {d.ax,  d.ay,  d.az,  d.dudt, d.dsxx, d.dsyy, d.dsxy, d.dsxz, d.dsyz, d.vx,
                          d.vy,  d.vz,  d.u,   d.sxx,  d.syy,  d.sxy,  d.sxz,  d.syz,  d.eps_ii};
  for (int k = 0; k < K; ++k) {
    const int b0 = (int)((int64_t)nb * k / K), b1 = (int)((int64_t)nb * (k + 1) / K);
    cudaStream_t fs = c->fstream[k & 1];
    CK(launch_forces_range(c, b0, b1, c->d_chunk_ctr + k, fs));
    CK(cudaEventRecord(c->chunk_ev[k], fs));
    CK(cudaStreamWaitEvent(c->cstream, c->chunk_ev[k], 0));
    const int64_t p0 = bucket_first(c, b0), p1 = bucket_first(c, b1);
    if (p1 <= p0) continue;
    const size_t n8 = sizeof(double) * (size_t)(p1 - p0);
    for (int q = 0; q < 19; ++q)
      CK(cudaMemcpyAsync(hd[q] + p0, dd[q] + p0, n8, cudaMemcpyDeviceToHost, c->cstream));
    CK(cudaMemcpyAsync(h.nngb + p0, d.nngb + p0, sizeof(int32_t) * (size_t)(p1 - p0),
                       cudaMemcpyDeviceToHost, c->cstream));
  }
  // the rest of the step follows the last launch of each stream
  CK(cudaStreamWaitEvent(c->stream, c->chunk_ev[K - 1], 0));
  if (K > 1) CK(cudaStreamWaitEvent(c->stream, c->chunk_ev[K - 2], 0));
  return SPH_OK;
}

// all = 1 permutes every array of the state (sph_neighbours on its own);
// steps pass 0 and recompute rho, Omega, P, c_s and the counts in the new
// order (with hierarchical steps rho, Omega and the counts still follow the
// sort: particles between their steps keep them).
// sort = 0 (hierarchical substeps right after a sorted one): drift only;
// the order, the grid and the cells stay, and the pair kernels search the
// cells within their radius plus this drift's largest coordinate change.
sph_status run_neighbours(sph_ctx *c, int drift, int all, int sort = 1) {
  const TraceRange tr("sph neighbours");
  CK(mark(c, 0));
  CK(launch_reset_status(c, 0));
  CK(launch_drift_bbox(c, drift));
  CK(launch_grid_setup(c, sort ? 0 : 1));
  if (sort) CK(launch_sort_permute(c, all, c->split_in ? 1 : 0));
  else c->src = c->st;
  CK(mark(c, 1));
  return copy_out(c, 0);
}

// Tuner marker k (density start / end, forces start / end) on tuning steps.
cudaError_t tmark(sph_ctx *c, int k) {
  return c->tune_now ? cudaEventRecord(c->tev[k], c->stream) : cudaSuccess;
}

sph_status run_derivatives(sph_ctx *c, int predict) {
  const TraceRange tr("sph derivatives");
  // split copy-in: the density solve needs only the positions; the
  // predictor (in the EOS pass) waits for the rest of the state
  CK(launch_pack(c));
  CK(mark(c, 2));
  CK(tmark(c, 0));
  CK(launch_density(c, 1));   // the force pass that follows counts the neighbours
  CK(tmark(c, 1));
  CK(mark(c, 3));
  sph_status s = copy_out(c, 1);
  if (s != SPH_OK) return s;
  if (c->split_in) {
    CK(cudaStreamWaitEvent(c->stream, c->in_ev, 0));
    CK(launch_permute_rest(c));
  }
  CK(launch_eos_pack(c, predict));
  CK(mark(c, 4));
  s = copy_out(c, 2);
  if (s != SPH_OK) return s;
  CK(tmark(c, 2));
  // sph_step_host, global step: the pass in ranges, each copied back as it
  // completes; otherwise one launch, and with the kicks in it the whole
  // final state is copied back after it
  const bool chunked = c->host_out && c->fuse_kick && c->copy_chunks > 1;
  if (chunked) {
    s = forces_chunked(c);
    if (s != SPH_OK) return s;
  } else {
    CK(launch_forces(c));
  }
  CK(tmark(c, 3));
  CK(launch_learn(c));
  CK(mark(c, 5));
  if (chunked || !c->host_out) {
    c->out_done = c->host_out != nullptr;
    return SPH_OK;
  }
  s = copy_out(c, 3);
  if (s == SPH_OK && c->fuse_kick) {
    s = copy_out(c, 4);
    c->out_done = 1;
  }
  return s;
}

// Everything one step enqueues, from the dt upload to the status readback.
// With hierarchical steps: the rungs from the last derivatives, then every
// substep's drift, sort, solve, force pass and kicks (kernel parameters
// carry the substep index; the copy-out of sph_step_host follows the last
// substep).
sph_status enqueue_step(sph_ctx *c) {
  sph_status s = upload_dt(c);
  if (s != SPH_OK) return s;
  const int L = 1 << c->rungs;
  c->kp.max_rung = c->rungs;
  c->kp.sub_scale = ldexp(1.0, -c->rungs);
  if (L > 1) {
    const cudaError_t e = launch_rung_init(c);
    if (e != cudaSuccess) s = fail_cuda(c, e, "launch_rung_init");
  }
  const sph_state *out = c->host_out;
  // one system: the pair kernels take buckets of active particles only
  c->kp.act = L > 1 ? c->w.act : nullptr;
  // global steps: the arrays the step rewrites are read from the
  // permutation's scratch instead of being copied back
  c->lazy = L == 1;
  for (int sub = 0; sub < L && s == SPH_OK; ++sub) {
    c->kp.substep = sub;
    c->host_out = sub == L - 1 ? out : nullptr;
    // a substep whose steps end only on the finest rung (sub even: no
    // coarser rung ends there) follows a sorted substep of this call and
    // keeps its order: the particles moved by one drift since (not the
    // call's first substep: the caller may have moved particles between
    // calls; not a periodic box, whose wrap moves a particle by a box length)
    const int sort = sub == 0 || (sub & 1) || c->kp.periodic;
    s = run_neighbours(c, 1, 0, sort);
    if (s == SPH_OK && c->kp.act) {
      const cudaError_t e = launch_compact_active(c);
      if (e != cudaSuccess) s = fail_cuda(c, e, "launch_compact_active");
    }
    // global steps of sph_step_host: the force pass kicks each particle as
    // soon as its derivatives are formed (its outputs are then copied back
    // range by range), leaving the sums to two small kernels; device steps
    // keep the kick kernel (same bits, same time on the device)
    c->fuse_kick = L == 1 && c->host_out != nullptr;
    if (s == SPH_OK) s = run_derivatives(c, 1);
    if (s == SPH_OK) {
      const cudaError_t e = c->fuse_kick ? launch_reduce_buckets(c) : launch_kick(c, 1);
      if (e != cudaSuccess) s = fail_cuda(c, e, "launch_kick");
    }
    c->fuse_kick = 0;
  }
  c->kp.substep = 0;
  c->kp.max_rung = 0;
  c->kp.sub_scale = 1.0;
  c->kp.act = nullptr;
  c->lazy = 0;
  c->src = c->st;
  c->host_out = out;
  if (s != SPH_OK) return s;
  CK(mark(c, 6));
  s = c->out_done ? SPH_OK : copy_out(c, 4);
  c->out_done = 0;
  if (s != SPH_OK) return s;
  return enqueue_status_readback(c);
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

void drop_graph(sph_ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
}

// Start of a step: while tuning, the candidate this step runs with (phase
// 0: a group span for both kernels; phase 1: a staging depth for both, at
// the spans phase 0 chose).
void tune_begin(sph_ctx *c) {
  c->tune_now = c->tune_left > 0;
  if (!c->tune_now) return;
  if (c->tune_phase == 0) {
    const int span = kSpans[c->tune_idx % kNumSpans];
    c->kp.span_d = span;
    c->kp.span_f = span;
  } else {
    const int depth = kDepths[c->tune_idx % kNumDepths];
    c->depth_d = depth;
    c->depth_f = depth;
  }
}

// End of a synchronised tuning step: book its kernel times; after the last
// one of a phase, keep each kernel's fastest candidate. The FP32 form then
// tunes the staging depth (the FP64 form has one compiled depth).
sph_status tune_end(sph_ctx *c) {
  if (!c->tune_now) return SPH_OK;
  c->tune_now = 0;
  float md = 0.f, mf = 0.f;
  CK(cudaEventElapsedTime(&md, c->tev[0], c->tev[1]));
  CK(cudaEventElapsedTime(&mf, c->tev[2], c->tev[3]));
  if (c->tune_phase == 0) {
    const int k = c->tune_idx % kNumSpans;
    c->tune_ms_d[k] += md;
    c->tune_ms_f[k] += mf;
    c->tune_n[k] += 1;
  } else {
    const int k = c->tune_idx % kNumDepths;
    c->tune_dms_d[k] += md;
    c->tune_dms_f[k] += mf;
    c->tune_dn[k] += 1;
  }
  c->tune_idx += 1;
  c->tune_left -= 1;
  if (c->tune_left > 0) return SPH_OK;
  int bd = 0, bf = 0;
  if (c->tune_phase == 0) {
    for (int q = 1; q < kNumSpans; ++q) {
      if (c->tune_ms_d[q] / c->tune_n[q] < c->tune_ms_d[bd] / c->tune_n[bd]) bd = q;
      if (c->tune_ms_f[q] / c->tune_n[q] < c->tune_ms_f[bf] / c->tune_n[bf]) bf = q;
    }
    c->kp.span_d = kSpans[bd];
    c->kp.span_f = kSpans[bf];
    if (c->kp.precision == SPH_FP32K) {
      c->tune_phase = 1;
      c->tune_idx = 0;
      c->tune_left = c->tune_rounds * kNumDepths;
    }
  } else {
    for (int q = 1; q < kNumDepths; ++q) {
      if (c->tune_dms_d[q] / c->tune_dn[q] < c->tune_dms_d[bd] / c->tune_dn[bd]) bd = q;
      if (c->tune_dms_f[q] / c->tune_dn[q] < c->tune_dms_f[bf] / c->tune_dn[bf]) bf = q;
    }
    c->depth_d = kDepths[bd];
    c->depth_f = kDepths[bf];
  }
  drop_graph(c);
  return SPH_OK;
}

// One step, enqueued directly or replayed from a CUDA graph captured on the
// library's own stream (the caller's stream may be the legacy default
// stream, which cannot be captured). Tuning steps are always direct.
// Synchronises.
sph_status run_step(sph_ctx *c, sph_step_info *info) {
  tune_begin(c);
  const bool via_graph = c->use_graph && !c->tune_now;
  if (!via_graph) {
    sph_status s = enqueue_step(c);
    if (s != SPH_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
  } else {
    cudaStream_t caller = c->stream;
    CK(cudaEventRecord(c->fence, caller));
    CK(cudaStreamWaitEvent(c->gstream, c->fence, 0));
    if (!c->graph_exec) {
      c->stream = c->gstream;
      c->capturing = 1;
      const cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
      sph_status s = e == cudaSuccess ? enqueue_step(c) : fail_cuda(c, e, "cudaStreamBeginCapture");
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
      c->stream = caller;
      c->capturing = 0;
      if (s != SPH_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e2 != cudaSuccess) return fail_cuda(c, e2, "cudaStreamEndCapture");
      const cudaError_t e3 = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (e3 != cudaSuccess) return fail_cuda(c, e3, "cudaGraphInstantiate");
      c->graph_nlaunch = c->nlaunch;
    }
    c->nlaunch = c->graph_nlaunch;
    CK(cudaGraphLaunch(c->graph_exec, c->gstream));
    CK(cudaStreamSynchronize(c->gstream));
  }
  const sph_status s = finish_sync(c, info);
  sph_status t = via_graph ? SPH_OK : collect_times(c);
  if (t == SPH_OK) t = tune_end(c);
  return s != SPH_OK ? s : t;
}

// Stage the dt of every system: dt[k] > 0 as given, otherwise that
// system's dt_next.
sph_status stage_dt(sph_ctx *c, const double *dt, double all) {
  for (int k = 0; k < c->nsys; ++k) {
    double d = dt ? dt[k] : all;
    if (!(d > 0.0)) {
      if (!c->primed || !(c->dt_next[k] > 0.0))
        return fail(c, SPH_E_STATE, "dt <= 0 needs a dt_next from sph_prime or an earlier step");
      d = c->dt_next[k];
    }
    c->h_dt[k] = d;
  }
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
    case SPH_E_CAPACITY: return "periodic box too narrow for the search radius";
    case SPH_E_NONFINITE: return "non-finite result";
    case SPH_E_TIMEOUT: return "device wait timed out";
    case SPH_E_STATE: return "context unusable";
    case SPH_E_INTERNAL: return "internal index check failed";
  }
  return "unknown status";
}

const char *sph_last_error(const sph_ctx *c) { return c ? c->err : "no context"; }

sph_status sph_inject_cuda_failure(sph_ctx *c, int32_t after) {
  if (!c || after < 0) return SPH_E_ARG;
  c->fail_after = after;
  return SPH_OK;
}

sph_status sph_init_batch(sph_ctx **out, const sph_params *p, const sph_material *mats,
                          int32_t n_mat, const sph_state *st, int64_t n, int32_t n_sys,
                          const int64_t *sys_first, void *cuda_stream) {
  if (!out) return SPH_E_ARG;
  *out = nullptr;
  if (!p || !mats || !st || n < 1 || n > (int64_t)1 << 30) return SPH_E_ARG;
  if (n_mat < 1 || n_mat > SPH_MAX_MATERIALS || !state_complete(st)) return SPH_E_ARG;
  if (n_sys < 1 || n_sys > SPH_MAX_SYSTEMS || !sys_first) return SPH_E_ARG;
  if (sys_first[0] != 0 || sys_first[n_sys] != n) return SPH_E_ARG;
  for (int k = 0; k < n_sys; ++k)
    if (sys_first[k + 1] <= sys_first[k]) return SPH_E_ARG;
  if (p->precision != SPH_FP64 && p->precision != SPH_FP32K) return SPH_E_ARG;
  if (p->jaumann != SPH_JAUMANN_OBJECTIVE && p->jaumann != SPH_JAUMANN_PRINTED) return SPH_E_ARG;
  if (p->yield_norm != SPH_YIELD_SQRT_J2 && p->yield_norm != SPH_YIELD_SQRT_3J2) return SPH_E_ARG;
  if (p->gradient_form != SPH_GRADIENT_SYMMETRIC && p->gradient_form != SPH_GRADIENT_ONE_SIDED)
    return SPH_E_ARG;
  if (p->max_rung < 0 || p->max_rung > 15) return SPH_E_ARG;
  if (p->gravity < SPH_GRAVITY_NONE || p->gravity > SPH_GRAVITY_RADIAL) return SPH_E_ARG;
  if (p->gravity == SPH_GRAVITY_RADIAL && n_sys > 1) return SPH_E_ARG;
  if (p->periodic != 0 && p->periodic != 1) return SPH_E_ARG;
  if (p->periodic) {
    // one system, one global step, no radial field
    if (n_sys != 1 || p->max_rung != 0 || p->gravity == SPH_GRAVITY_RADIAL) return SPH_E_ARG;
    for (int a = 0; a < 3; ++a)
      if (!(p->box_hi[a] > p->box_lo[a]) || !isfinite(p->box_lo[a]) || !isfinite(p->box_hi[a]))
        return SPH_E_ARG;
  }
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
  c->src = *st;
  c->n = n;
  c->stream = (cudaStream_t)cuda_stream;
  c->nsys = n_sys;
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

  // Systems: particle ranges and 32-particle buckets that never straddle
  // two systems, a cell budget of twice the particle count (at least 4096,
  // at most 2^24) each.
  c->sys_first = (int64_t *)malloc(sizeof(int64_t) * (n_sys + 1));
  c->dt_next = (double *)calloc(n_sys, sizeof(double));
  SysRec *rec = (SysRec *)calloc(n_sys, sizeof(SysRec));
  int *bnd = (int *)malloc(sizeof(int) * 2 * (n_sys + 1));
  if (!c->sys_first || !c->dt_next || !rec || !bnd) {
    free(rec);
    free(bnd);
    free_all(c);
    free(c);
    return SPH_E_ARG;
  }
  int *bb = bnd, *bk = bnd + (n_sys + 1);
  int64_t buckets = 0, cells = 0;
  for (int k = 0; k <= n_sys; ++k) {
    c->sys_first[k] = sys_first[k];
    bb[k] = (int)sys_first[k];
    bk[k] = (int)buckets;
    if (k == n_sys) break;
    const int64_t cnt = sys_first[k + 1] - sys_first[k];
    rec[k].begin = (int)sys_first[k];
    rec[k].end = (int)sys_first[k + 1];
    rec[k].bucket_off = (int)buckets;
    int64_t cap = 2 * cnt;
    if (cap < 4096) cap = 4096;
    if (cap > (1 << 24)) cap = 1 << 24;
    rec[k].cell_cap = (int)cap;
    buckets += (cnt + 31) / 32;
    cells += cap;
  }
  // 32-bit sort keys: the system index above a Morton code of 3 * axis_bits
  int sys_bits = 0;
  while ((1 << sys_bits) < n_sys) ++sys_bits;
  int axis_bits = (32 - sys_bits) / 3;
  if (axis_bits > 10) axis_bits = 10;
  c->max_cells = (int)cells;
  KParams &kp = c->kp;
  kp.nsys = n_sys;
  kp.axis_bits = axis_bits;
  kp.nbuckets = (int)buckets;
  kp.span_d = 2;
  kp.span_f = 2;
  c->depth_d = kDepthDensity;
  c->depth_f = kDepthForces;
  cudaError_t es = dalloc(&c->d_sys, n_sys);
  if (es == cudaSuccess) es = cudaMemcpy(c->d_sys, rec, sizeof(SysRec) * n_sys, cudaMemcpyHostToDevice);
  if (es == cudaSuccess) es = dalloc(&c->d_sys_begin, n_sys + 1);
  if (es == cudaSuccess) es = dalloc(&c->d_sys_bucket, n_sys + 1);
  if (es == cudaSuccess)
    es = cudaMemcpy(c->d_sys_begin, bb, sizeof(int) * (n_sys + 1), cudaMemcpyHostToDevice);
  if (es == cudaSuccess)
    es = cudaMemcpy(c->d_sys_bucket, bk, sizeof(int) * (n_sys + 1), cudaMemcpyHostToDevice);
  free(rec);
  free(bnd);
  CKI(es);
  kp.sys = c->d_sys;
  kp.sys_begin = c->d_sys_begin;
  kp.sys_bucket = c->d_sys_bucket;
  {
    // reduction tiles of kRedTile buckets within each system
    std::vector<int> t0, t1, st;
    int b1 = 0;
    for (int k = 0; k < n_sys; ++k) {
      st.push_back((int)t0.size());
      const int b0 = b1;
      b1 = b0 + (int)((c->sys_first[k + 1] - c->sys_first[k] + 31) / 32);
      for (int b = b0; b < b1; b += kRedTile) {
        t0.push_back(b);
        t1.push_back(b + kRedTile < b1 ? b + kRedTile : b1);
      }
    }
    st.push_back((int)t0.size());
    const int nt = (int)t0.size();
    std::vector<int> all(t0);
    all.insert(all.end(), t1.begin(), t1.end());
    all.insert(all.end(), st.begin(), st.end());
    CKI(dalloc(&c->d_red_tile, all.size()));
    CKI(cudaMemcpy(c->d_red_tile, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
    CKI(dalloc(&c->tile_partials, (size_t)nt * kNSlot));
    kp.red_tile = c->d_red_tile;
    kp.red_tile_end = c->d_red_tile + nt;
    kp.sys_tile = c->d_red_tile + 2 * nt;
    kp.nred_tiles = nt;
  }

  CKI(dalloc(&c->d_mats, SPH_MAX_MATERIALS));
  CKI(cudaMemcpy(c->d_mats, c->mats, sizeof(c->mats), cudaMemcpyHostToDevice));
  {
    MatT<float> mf[SPH_MAX_MATERIALS];
    MatT<double> md[SPH_MAX_MATERIALS];
    for (int k = 0; k < SPH_MAX_MATERIALS; ++k) {
      mf[k] = mat_copy<float>(c->mats[k]);
      md[k] = mat_copy<double>(c->mats[k]);
      const double hk = c->mats[k].rho0 > 0.0
                            ? 3.0 * p->n_ngb / (4.0 * kPi * c->mats[k].rho0)
                            : 0.0;
      mf[k].hcap_k = (float)hk;
      md[k].hcap_k = hk;
      mf[k].hcap_f = (float)p->h_cap_factor;
      md[k].hcap_f = p->h_cap_factor;
    }
    CKI(dalloc(&c->d_matf, SPH_MAX_MATERIALS));
    CKI(dalloc(&c->d_matd, SPH_MAX_MATERIALS));
    CKI(cudaMemcpy(c->d_matf, mf, sizeof(mf), cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(c->d_matd, md, sizeof(md), cudaMemcpyHostToDevice));
  }
  kp.n_ngb = p->n_ngb;
  kp.av_alpha = p->av_alpha;
  kp.av_beta = p->av_beta;
  kp.av_eps = p->av_eps;
  kp.eta_c = p->eta_c;
  kp.eta_a = p->eta_a;
  kp.h_tol = p->h_tol;
  kp.av_alpha_f = (float)p->av_alpha;
  kp.lattice_k_f = (float)(3.0 * p->n_ngb / (4.0 * kPi));
  kp.av_beta_f = (float)p->av_beta;
  kp.av_eps_f = (float)p->av_eps;
  kp.h_tol_f = (float)p->h_tol;
  kp.max_sweeps = p->max_sweeps;
  kp.h_cap_factor = p->h_cap_factor;
  kp.precision = p->precision;
  kp.jaumann = p->jaumann;
  kp.yield_norm = p->yield_norm;
  kp.correction = p->correction_tensor;
  kp.grad_wi = p->gradient_form == SPH_GRADIENT_ONE_SIDED ? -1.0 : -0.5;
  kp.grad_wj = p->gradient_form == SPH_GRADIENT_ONE_SIDED ? 0.0 : -0.5;
  kp.grad_wi_f = (float)kp.grad_wi;
  kp.grad_wj_f = (float)kp.grad_wj;
  // hierarchical steps are switched on only while a step is enqueued: every
  // other call (sph_prime, sph_density, ...) treats all particles alike
  c->rungs = p->max_rung;
  c->copy_chunks = 8;
  kp.max_rung = 0;
  kp.substep = 0;
  kp.sub_scale = 1.0;
  kp.periodic = p->periodic;
  for (int a = 0; a < 3; ++a) {
    kp.box_lo[a] = p->box_lo[a];
    kp.box_hi[a] = p->box_hi[a];
    kp.box_len[a] = p->box_hi[a] - p->box_lo[a];
  }
  kp.gravity = p->gravity;
  for (int a = 0; a < 3; ++a) {
    kp.g_uniform[a] = p->g_uniform[a];
    kp.g_uniform_f[a] = (float)p->g_uniform[a];
    kp.g_center[a] = p->g_center[a];
  }
  kp.mats = c->d_mats;
  kp.matf = c->d_matf;
  kp.matd = c->d_matd;
  if (p->gravity == SPH_GRAVITY_RADIAL) {
    const int gn = p->g_n;
    std::vector<double> radii(gn);
    for (int k = 0; k < gn; ++k)
      radii[k] = p->g_rmin * pow(p->g_rmax / p->g_rmin, (double)k / (double)(gn - 1));
    CKI(dalloc(&c->d_gtab, gn));
    CKI(dalloc(&c->d_phitab, gn));
    CKI(dalloc(&c->d_radii, gn));
    CKI(cudaMemcpy(c->d_gtab, p->g_table, sizeof(double) * gn, cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(c->d_phitab, p->phi_table, sizeof(double) * gn, cudaMemcpyHostToDevice));
    CKI(cudaMemcpy(c->d_radii, radii.data(), sizeof(double) * gn, cudaMemcpyHostToDevice));
    {
      std::vector<float> tf(3 * (size_t)gn);
      for (int k = 0; k < gn; ++k) {
        tf[k] = (float)p->g_table[k];
        tf[gn + k] = (float)p->phi_table[k];
        tf[2 * gn + k] = (float)radii[k];
      }
      CKI(dalloc(&c->d_gtab_f, 3 * (size_t)gn));
      CKI(cudaMemcpy(c->d_gtab_f, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice));
    }
    kp.g_table = c->d_gtab;
    kp.phi_table = c->d_phitab;
    kp.g_radii = c->d_radii;
    kp.g_n = gn;
    kp.g_rmin = p->g_rmin;
    kp.g_rmax = p->g_rmax;
    kp.g_gm = p->g_gm;
    kp.g_inv_log_ratio = (double)(gn - 1) / log2(p->g_rmax / p->g_rmin);
    kp.g_table_f = c->d_gtab_f;
    kp.phi_table_f = c->d_gtab_f + gn;
    kp.g_radii_f = c->d_gtab_f + 2 * gn;
    kp.g_rmin_f = (float)kp.g_rmin;
    kp.g_rmax_f = (float)kp.g_rmax;
    kp.g_gm_f = (float)kp.g_gm;
    kp.g_inv_log_ratio_f = (float)kp.g_inv_log_ratio;
  }
  c->params.g_table = c->d_gtab;
  c->params.phi_table = c->d_phitab;

  Work &w = c->w;
  CKI(dalloc(&w.vsig, n));
  CKI(dalloc(&w.edot2, n));
  CKI(dalloc(&w.yld, n));
  CKI(dalloc(&w.cc, n));
  if (p->max_rung > 0) {
    CKI(dalloc(&w.rung, n));
    CKI(cudaMemset(w.rung, 0, sizeof(int) * (size_t)n));
    if (n_sys == 1) {   // active-particle list of every substep
      CKI(dalloc(&w.act, n));
      CKI(dalloc(&w.act_tiles, (n + 2047) / 2048));
    }
  }
  kp.rung = w.rung;
  if (fp32) {
    CKI(dalloc(&w.pos32, n));
    CKI(dalloc(&w.posh32, n));
    CKI(dalloc(&w.fj32, (size_t)4 * n));
    for (int k = 0; k < 3; ++k) CKI(dalloc(&w.fs32[k], n));
  } else {
    CKI(dalloc(&w.pos64, n));
    CKI(dalloc(&w.posh64, n));
    CKI(dalloc(&w.fj64, (size_t)4 * n));
    for (int k = 0; k < 3; ++k) CKI(dalloc(&w.fs64[k], n));
  }
  CKI(dalloc(&c->keys, n));
  CKI(dalloc(&c->keys_alt, n));
  CKI(dalloc(&c->vals, n));
  CKI(dalloc(&c->vals_alt, n));
  c->ntiles = (int)((n + 2047) / 2048);
  CKI(dalloc(&c->hist, (size_t)256 * c->ntiles));
  CKI(dalloc(&c->scan_tot, (size_t)(256 * c->ntiles + 1023) / 1024 + 1));
  CKI(dalloc(&c->cell_start, c->max_cells));
  CKI(dalloc(&c->cell_end, c->max_cells));
  c->tmp_words = 32;
  CKI(cudaMalloc(&c->tmp, (size_t)n * c->tmp_words * 8));
  CKI(alloc_density_spill(c));
  for (int k = 0; k < kNSum; ++k) CKI(dalloc(&w.terms[k], n));
  CKI(dalloc(&w.tcrit, n));
  CKI(dalloc(&c->d_dt, n_sys));
  CKI(cudaMemset(c->d_dt, 0, sizeof(double) * n_sys));
  kp.dt = c->d_dt;
  CKI(dalloc(&c->d_status, 1));
  CKI(cudaMemset(c->d_status, 0, sizeof(Status)));
  CKI(cudaMallocHost((void **)&c->h_status, sizeof(Status)));
  CKI(cudaMallocHost((void **)&c->h_sys, sizeof(SysRec) * n_sys));
  CKI(cudaMallocHost((void **)&c->h_dt, sizeof(double) * n_sys));
  memset(c->h_status, 0, sizeof(Status));
  memset(c->h_sys, 0, sizeof(SysRec) * n_sys);
  memset(c->h_dt, 0, sizeof(double) * n_sys);
  // validate the caller's state once
  unsigned *bad = nullptr;
  CKI(dalloc(&bad, 1));
  CKI(cudaMemset(bad, 0, sizeof(unsigned)));
  k_validate<<<148 * 4, kBlock, 0, c->stream>>>(c->st, n, n_mat, n_sys > 1, c->kp, bad);
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

sph_status sph_init(sph_ctx **out, const sph_params *p, const sph_material *mats, int32_t n_mat,
                    const sph_state *st, int64_t n, void *cuda_stream) {
  const int64_t first[2] = {0, n};
  return sph_init_batch(out, p, mats, n_mat, st, n, 1, first, cuda_stream);
}

sph_status sph_set_timing(sph_ctx *c, int32_t on) {
  ENTER(c);
  CK(cudaStreamSynchronize(c->stream));

  if (on && !c->timing) {
    for (int k = 0; k <= SPH_NUM_PHASES; ++k) CK(cudaEventCreate(&c->ev[k]));
  }
  if (!on && c->timing) {
    for (int k = 0; k <= SPH_NUM_PHASES; ++k) {
      cudaEventDestroy(c->ev[k]);
      c->ev[k] = nullptr;
    }
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

sph_status sph_set_graph(sph_ctx *c, int32_t on) {
  ENTER(c);
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  if (on && !c->gstream) {
    CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->fence, cudaEventDisableTiming));
  }
  c->use_graph = on ? 1 : 0;
  return SPH_OK;
}

sph_status sph_destroy(sph_ctx *c) {
  if (!c) return SPH_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->gstream) cudaStreamSynchronize(c->gstream);
  drop_graph(c);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->fence) cudaEventDestroy(c->fence);
  if (c->cstream) {
    cudaStreamSynchronize(c->cstream);
    cudaStreamDestroy(c->cstream);
  }
  if (c->istream) {
    cudaStreamSynchronize(c->istream);
    cudaStreamDestroy(c->istream);
  }
  for (int k = 0; k < 2; ++k)
    if (c->fstream[k]) {
      cudaStreamSynchronize(c->fstream[k]);
      cudaStreamDestroy(c->fstream[k]);
    }
  if (c->ev_pre) cudaEventDestroy(c->ev_pre);
  for (int k = 0; k < SPH_MAX_COPY_CHUNKS; ++k)
    if (c->chunk_ev[k]) cudaEventDestroy(c->chunk_ev[k]);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->in_ev) cudaEventDestroy(c->in_ev);
  // handles that a failed set-up never created stay null and are skipped
  for (int k = 0; k < 5; ++k)
    if (c->out_ev[k]) cudaEventDestroy(c->out_ev[k]);
  for (int k = 0; k <= SPH_NUM_PHASES; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  for (int k = 0; k < 4; ++k)
    if (c->tev[k]) cudaEventDestroy(c->tev[k]);
  free_all(c);
  free(c);
  // teardown reports nothing to the caller; leave no error pending
  (void)cudaGetLastError();
  return SPH_OK;
}

sph_status sph_autotune(sph_ctx *c, int32_t rounds) {
  ENTER(c);
  if (rounds < 0 || rounds > 64) return fail(c, SPH_E_ARG, "rounds must be in 0..64");
  if (rounds > 0 && !c->tev[0])
    for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&c->tev[k]));
  c->tune_left = rounds * kNumSpans;
  c->tune_rounds = rounds;
  c->tune_phase = 0;
  c->tune_idx = 0;
  for (int k = 0; k < kNumSpans; ++k) {
    c->tune_ms_d[k] = c->tune_ms_f[k] = 0.0;
    c->tune_n[k] = 0;
  }
  for (int k = 0; k < kNumDepths; ++k) {
    c->tune_dms_d[k] = c->tune_dms_f[k] = 0.0;
    c->tune_dn[k] = 0;
  }
  return SPH_OK;
}

sph_status sph_set_copy_chunks(sph_ctx *c, int32_t chunks) {
  ENTER(c);
  if (chunks < 1 || chunks > SPH_MAX_COPY_CHUNKS)
    return fail(c, SPH_E_ARG, "chunks must be in 1..SPH_MAX_COPY_CHUNKS");
  c->copy_chunks = chunks;
  return SPH_OK;
}

sph_status sph_set_spans(sph_ctx *c, int32_t span_density, int32_t span_forces) {
  ENTER(c);
  if (span_density < kSpans[0] || span_density > kSpans[kNumSpans - 1] ||
      span_forces < kSpans[0] || span_forces > kSpans[kNumSpans - 1])
    return fail(c, SPH_E_ARG, "span out of range");
  c->tune_left = 0;
  c->kp.span_d = span_density;
  c->kp.span_f = span_forces;
  drop_graph(c);
  return SPH_OK;
}

sph_status sph_set_stage_depths(sph_ctx *c, int32_t depth_density, int32_t depth_forces) {
  ENTER(c);
  bool okd = false, okf = false;
  for (int k = 0; k < kNumDepths; ++k) {
    okd = okd || depth_density == kDepths[k];
    okf = okf || depth_forces == kDepths[k];
  }
  if (!okd || !okf) return fail(c, SPH_E_ARG, "staging depth must be 3 or 4");
  c->tune_left = 0;
  c->depth_d = depth_density;
  c->depth_f = depth_forces;
  drop_graph(c);
  return SPH_OK;
}

sph_status sph_tune_info(const sph_ctx *c, sph_tune_report *out) {
  if (!c || !out) return SPH_E_ARG;
  memset(out, 0, sizeof(*out));
  const bool fp32 = c->kp.precision == SPH_FP32K;
  out->span_density = c->kp.span_d;
  out->span_forces = c->kp.span_f;
  // the depth phase still to come after the spans (FP32 form)
  out->steps_left = c->tune_left +
                    (c->tune_left > 0 && c->tune_phase == 0 && fp32 ? c->tune_rounds * kNumDepths
                                                                    : 0);
  out->n_cand = kNumSpans;
  for (int k = 0; k < kNumSpans; ++k) {
    out->cand[k] = kSpans[k];
    out->timed[k] = c->tune_n[k];
    out->ms_density[k] = c->tune_ms_d[k];
    out->ms_forces[k] = c->tune_ms_f[k];
  }
  out->depth_density = fp32 ? c->depth_d : kDepthDensity;
  out->depth_forces = fp32 ? c->depth_f : kDepthForces;
  out->n_depth = fp32 ? kNumDepths : 1;
  for (int k = 0; k < out->n_depth; ++k) {
    out->depth_cand[k] = fp32 ? kDepths[k] : kDepthDensity;
    out->depth_timed[k] = fp32 ? c->tune_dn[k] : 0;
    out->ms_depth_density[k] = fp32 ? c->tune_dms_d[k] : 0.0;
    out->ms_depth_forces[k] = fp32 ? c->tune_dms_f[k] : 0.0;
  }
  return SPH_OK;
}

sph_status sph_neighbours(sph_ctx *c) {
  ENTER(c);
  return run_neighbours(c, 0, 1);
}

sph_status sph_density(sph_ctx *c, int32_t *sweeps) {
  ENTER(c);
  CK(launch_pack(c));
  CK(launch_density(c, 0));   // standalone: every solve ends on an evaluation
  sph_step_info info;
  const sph_status s = sync_status(c, &info);
  if (sweeps) *sweeps = info.sweeps;
  return s;
}

sph_status sph_forces_strength(sph_ctx *c) {
  ENTER(c);
  CK(launch_pack(c));
  CK(launch_eos_pack(c, 0));
  CK(launch_forces(c));
  return SPH_OK;
}

sph_status sph_stress_update(sph_ctx *c, double dt) {
  ENTER(c);
  if (!(dt > 0.0)) return fail(c, SPH_E_ARG, "dt must be positive");
  for (int k = 0; k < c->nsys; ++k) c->h_dt[k] = dt;
  sph_status s = upload_dt(c);
  if (s != SPH_OK) return s;
  CK(launch_kick(c, 1));
  CK(cudaStreamSynchronize(c->stream));  // the staging buffer is reused by the next call
  return SPH_OK;
}

sph_status sph_prime(sph_ctx *c, sph_step_info *info) {
  const TraceRange tr("sph_prime");
  ENTER(c);
  for (int k = 0; k < c->nsys; ++k) c->h_dt[k] = 0.0;
  sph_status s = upload_dt(c);
  if (s == SPH_OK) s = run_neighbours(c, 0, 0);
  if (s != SPH_OK) return s;
  s = run_derivatives(c, 0);
  if (s != SPH_OK) return s;
  CK(launch_kick(c, 0));
  s = sync_status(c, info);
  if (s == SPH_OK || s == SPH_E_NOCONV) c->primed = 1;
  return s;
}

sph_status sph_step(sph_ctx *c, double dt, sph_step_info *info) {
  const TraceRange tr("sph_step");
  ENTER(c);
  const sph_status s = stage_dt(c, nullptr, dt);
  return s != SPH_OK ? s : run_step(c, info);
}

sph_status sph_step_batch(sph_ctx *c, const double *dt, sph_step_info *info) {
  const TraceRange tr("sph_step_batch");
  ENTER(c);
  if (!dt) return fail(c, SPH_E_ARG, "dt array is NULL");
  const sph_status s = stage_dt(c, dt, 0.0);
  return s != SPH_OK ? s : run_step(c, info);
}

sph_status sph_set_learned_h(sph_ctx *c, int32_t guess, int32_t record, const sph_mlp *net) {
  ENTER(c);
  if (guess < SPH_GUESS_PREVIOUS || guess > SPH_GUESS_NETWORK || (record != 0 && record != 1))
    return fail(c, SPH_E_ARG, "unknown guess mode");
  if (guess == SPH_GUESS_NETWORK && !net) return fail(c, SPH_E_ARG, "network guess needs a network");
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  LearnArgs &L = c->learn;
  const int64_t n = c->n;
  if (!record) {   // recording buffers
    void *p[] = {L.feat[0], L.feat[1], L.feat[2], L.x_out, L.y_out};
    for (void *q : p)
      if (q) cudaFree(q);
    L.feat[0] = L.feat[1] = L.feat[2] = nullptr;
    L.x_out = L.y_out = nullptr;
  }
  if (guess == SPH_GUESS_PREVIOUS && !record) {
    void *p[] = {c->w.divv, L.hprev, L.hprop};
    for (void *q : p)
      if (q) cudaFree(q);
    memset(&L, 0, sizeof(L));
    c->w.divv = nullptr;
    c->kp.h_guess = nullptr;
    c->net = nullptr;
    return SPH_OK;
  }
  if (!L.hprev) {
    // samples are written by particle id
    unsigned *bad = nullptr;
    CK(dalloc(&bad, 1));
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), c->stream));
    k_validate<<<148 * 4, kBlock, 0, c->stream>>>(c->st, n, c->nmat, 1, c->kp, bad);
    unsigned hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(bad);
    if (hbad) return fail(c, SPH_E_ARG, "the learned form needs ids 0..n-1");
    CK(dalloc(&c->w.divv, n));
    CK(dalloc(&L.hprev, n));
    CK(dalloc(&L.hprop, n));
  }
  if (record && !L.x_out) {
    for (int k = 0; k < 3; ++k) CK(dalloc(&L.feat[k], n));
    CK(dalloc(&L.x_out, (size_t)n * 6));
    CK(dalloc(&L.y_out, n));
    CK(cudaMemsetAsync(L.x_out, 0xff, sizeof(float) * 6 * n, c->stream));   // NaN
    CK(cudaMemsetAsync(L.y_out, 0xff, sizeof(float) * n, c->stream));
  }
  // the sort carries the learned arrays with their particles
  const int words = 29 + 2 + (record ? 3 : 0) + 2;
  if (c->tmp_words < words) {
    CK(cudaFree(c->tmp));
    c->tmp = nullptr;
    CK(cudaMalloc(&c->tmp, (size_t)n * words * 8));
    c->tmp_words = words;
  }
  L.guess = guess;
  L.record = record;
  L.divv = c->w.divv;
  c->net = guess == SPH_GUESS_NETWORK ? net : nullptr;
  // the history restarts: the first step after the call records no sample
  // and the solve starts from the previous radius until a proposal exists
  CK(cudaMemsetAsync(L.hprev, 0, sizeof(double) * n, c->stream));
  CK(cudaMemsetAsync(L.hprop, 0, sizeof(double) * n, c->stream));
  c->kp.h_guess = guess == SPH_GUESS_PREVIOUS ? nullptr : L.hprop;
  CK(cudaStreamSynchronize(c->stream));
  return SPH_OK;
}

sph_status sph_learn_samples(sph_ctx *c, float *X, float *y) {
  ENTER(c);
  if (!X || !y) return fail(c, SPH_E_ARG, "NULL sample buffer");
  if (!c->learn.record || !c->learn.x_out) return fail(c, SPH_E_STATE, "not recording");
  CK(cudaMemcpyAsync(X, c->learn.x_out, sizeof(float) * 6 * c->n, cudaMemcpyDeviceToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(y, c->learn.y_out, sizeof(float) * c->n, cudaMemcpyDeviceToDevice,
                     c->stream));
  return SPH_OK;
}

sph_status sph_learn_proposal(sph_ctx *c, double *h_next) {
  ENTER(c);
  if (!h_next) return fail(c, SPH_E_ARG, "NULL output");
  if (!c->learn.hprop || c->learn.guess == SPH_GUESS_PREVIOUS)
    return fail(c, SPH_E_STATE, "no proposal mode");
  CK(cudaMemcpyAsync(h_next, c->learn.hprop, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                     c->stream));
  return SPH_OK;
}

sph_status sph_batch_info(const sph_ctx *c, sph_step_info *info, int32_t n) {
  if (!c || !info || n < 1 || n > c->nsys) return SPH_E_ARG;
  for (int k = 0; k < n; ++k) fill_info(c, k, &info[k]);
  return SPH_OK;
}

sph_status sph_step_host(sph_ctx *c, const sph_state *host, double dt, sph_step_info *info,
                         int64_t *bytes_in, int64_t *bytes_out) {
  const TraceRange tr("sph_step_host");
  ENTER(c);
  if (!host || !state_complete(host)) return fail(c, SPH_E_ARG, "incomplete host state");
  if (!c->cstream) {
    CK(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) CK(cudaEventCreateWithFlags(&c->out_ev[k], cudaEventDisableTiming));
  }
  if (!c->istream) {
    CK(cudaStreamCreateWithFlags(&c->istream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->in_ev, cudaEventDisableTiming));
  }
  if (!c->fstream[0]) {
    for (int k = 0; k < 2; ++k) CK(cudaStreamCreateWithFlags(&c->fstream[k], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_pre, cudaEventDisableTiming));
    for (int k = 0; k < SPH_MAX_COPY_CHUNKS; ++k)
      CK(cudaEventCreateWithFlags(&c->chunk_ev[k], cudaEventDisableTiming));
    CK(cudaMalloc(&c->d_chunk_ctr, sizeof(unsigned) * SPH_MAX_COPY_CHUNKS));
  }
  const sph_state &d = c->st;
  const int64_t n = c->n;
  const size_t b8 = sizeof(double) * (size_t)n, b4 = sizeof(int32_t) * (size_t)n;
  // in: everything the step reads before writing it (rho, Omega, P, c_s and
  // the counts are recomputed in the step, so they stay on the host). First,
  // on the context's stream, what the drift, the sort and the density solve
  // read; then, on the input stream once those copies are done, the rest,
  // which arrives while the sort and the density solve run (with
  // hierarchical steps every substep needs the whole state: one stream)
  double *const ha[8] = {host->x, host->y, host->z, host->vx, host->vy, host->vz, host->m, host->h};
  double *const da[8] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.m, d.h};
  double *const hb[16] = {host->u,    host->sxx,  host->syy,  host->sxy,  host->sxz,  host->syz,
                          host->ax,   host->ay,   host->az,   host->dudt, host->dsxx, host->dsyy,
                          host->dsxy, host->dsxz, host->dsyz, host->eps_ii};
  double *const db[16] = {d.u,    d.sxx,  d.syy,  d.sxy,  d.sxz,  d.syz,  d.ax,   d.ay,
                          d.az,   d.dudt, d.dsxx, d.dsyy, d.dsxy, d.dsxz, d.dsyz, d.eps_ii};
  const int split = c->rungs == 0;
  for (int k = 0; k < 8; ++k) CK(cudaMemcpyAsync(da[k], ha[k], b8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.id, host->id, b8, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.mat, host->mat, b4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.flags, host->flags, b4, cudaMemcpyHostToDevice, c->stream));
  cudaStream_t bs = c->stream;
  if (split) {
    CK(cudaEventRecord(c->ev_a, c->stream));
    CK(cudaStreamWaitEvent(c->istream, c->ev_a, 0));
    bs = c->istream;
  }
  for (int k = 0; k < 16; ++k) CK(cudaMemcpyAsync(db[k], hb[k], b8, cudaMemcpyHostToDevice, bs));
  if (split) CK(cudaEventRecord(c->in_ev, c->istream));
  int64_t in = 25 * (int64_t)b8 + 2 * (int64_t)b4;
  if (c->rungs > 0) {   // particles between their steps keep H, rho, Omega and their count
    CK(cudaMemcpyAsync(d.rho, host->rho, b8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.omega, host->omega, b8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.nngb, host->nngb, b4, cudaMemcpyHostToDevice, c->stream));
    in += 2 * (int64_t)b8 + (int64_t)b4;
  }
  // out: each array group as soon as the step has finished it, on the copy
  // stream (direct launches: the captured graph has no copy-out)
  c->host_out = host;
  c->split_in = split;
  const int graph = c->use_graph;
  c->use_graph = 0;
  const sph_status s = sph_step(c, dt, info);
  c->use_graph = graph;
  c->host_out = nullptr;
  c->split_in = 0;
  // the input stream is idle once the step has waited for it; if the step
  // stopped early it may still be copying
  const cudaError_t ei = cudaStreamSynchronize(c->istream);
  if (ei != cudaSuccess) return fail_cuda(c, ei, "copy-in");
  const cudaError_t e = cudaStreamSynchronize(c->cstream);
  if (e != cudaSuccess) return fail_cuda(c, e, "copy-out");
  if (bytes_in) *bytes_in = in;
  if (bytes_out) *bytes_out = 29 * (int64_t)b8 + 3 * (int64_t)b4;
  return s;
}

}  // extern "C"
