// sph_update.cu -- closing and opening kicks with radial return (§2.4,
// Eq. 41-43), FP64 global sums (energies, momentum, angular momentum Eq. 46)
// and the time-step minimum of Eq. 38-39.
#include "sph_internal.cuh"

namespace sphk {

constexpr int kNSum = 9;

// kick = 1: close to i (v, u, S alike), rescale S with Y at (rho_i, u_i),
// accumulate 1/2 edot:edot dt, sum diagnostics at i, open to i+1/2.
// kick = 0: diagnostics and time step of the state as it stands. The
// integration and the sums are FP64; the EOS, yield and time-step criteria
// are evaluated in T.
// One block per chunk of kChunk consecutive particles of one system, so
// that every system's sums are formed in a fixed order of its own.
// src: where v, u, S and the strain invariant are read (the step's read
// view: their permuted copies when the permutation did not copy them
// back); s: where they are written, for every particle then.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_kick(sph_state s, sph_state src, Work w, int kick,
                                                KParams P, double *partials, Status *st) {
  const bool copy = src.vx != s.vx;   // lazy step: write every particle
  __shared__ double red[kNSum][kBlock];
  __shared__ double redt[kBlock / 32];
  __shared__ int hist[16];
  if (threadIdx.x < 16) hist[threadIdx.x] = 0;
  __syncthreads();
  const int b = blockIdx.x;
  const int sy = P.nsys > 1 ? sys_lookup(P.sys_chunk, P.nsys, b) : 0;
  SysRec &R = P.sys[sy];
  const int64_t c0 = R.begin + (int64_t)(b - R.chunk_off) * kChunk;
  const int64_t c1 = c0 + kChunk < R.end ? c0 + kChunk : R.end;
  // the substep; without rungs the step (sub_scale = 1)
  const double sub = kick ? P.dt[sy] * P.sub_scale : 0.0;
  const bool last = P.substep + 1 == (1 << P.max_rung);   // every particle's step ends
  int updates = 0;
  double acc[kNSum] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  T tmin = T(INFINITY);
  const T eta_a = to_t<T>(P.eta_a), eta_c = to_t<T>(P.eta_c);
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    // hierarchical steps: before the last substep only the kicked particles
    // matter (the sums and the time step are those of the big step's end)
    if (!last && !rung_active(P, i)) continue;
    const bool fixed = s.flags[i] & SPH_FLAG_FIXED;
    const double m = s.m[i];
    const double a[3] = {s.ax[i], s.ay[i], s.az[i]};
    double v[3] = {src.vx[i], src.vy[i], src.vz[i]};
    double u = src.u[i];
    // kicked: moving particles whose own step ends with this substep
    if (kick && !fixed && rung_active(P, i)) {
      const double dt = sub * (double)rung_len(P, i), hdt = 0.5 * dt;
      const MatT<T> &M = mat_t<T>(P, s.mat[i]);
      const double dS[5] = {s.dsxx[i], s.dsyy[i], s.dsxy[i], s.dsxz[i], s.dsyz[i]};
      double S[5] = {src.sxx[i], src.syy[i], src.sxy[i], src.sxz[i], src.syz[i]};
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] += hdt * a[k];
      u += hdt * s.dudt[i];
#pragma unroll
      for (int k = 0; k < 5; ++k) S[k] += hdt * dS[k];
      if (M.strength) {
        const EosT<T> e = eos_t<T>(M, s.rho[i], u);
        const T St[5] = {to_t<T>(S[0]), to_t<T>(S[1]), to_t<T>(S[2]), to_t<T>(S[3]), to_t<T>(S[4])};
        const double f = from_t(radial_factor_t<T>(St, yield_t<T>(M, e.P, to_t<T>(u)), P.yield_norm));
        if (f < 1.0) {   // below the yield surface f is exactly 1
#pragma unroll
          for (int k = 0; k < 5; ++k) S[k] *= f;
        }
      } else {
        S[0] = S[1] = S[2] = S[3] = S[4] = 0.0;
      }
      s.eps_ii[i] = src.eps_ii[i] + dt * w.edot2[i];
      // opening kick from the state at i; with rungs over the next step of
      // the rung the criteria ask for, no coarser than the coarsest rung
      // whose steps start at the next substep
      double ho = hdt;
      if (P.max_rung) {
        const double am = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        const double h = s.h[i];
        const double ta = am > 0.0 ? P.eta_a * sqrt(h / am) : INFINITY;
        const double tc = P.eta_c * h / w.vsig[i];
        int r = rung_want(P, sub, ta < tc ? ta : tc);
        int r_al = P.max_rung;
        for (int m = P.substep + 1; r_al > 0 && (m & 1) == 0; m >>= 1) --r_al;
        r = r > r_al ? r : r_al;
        w.rung[i] = r;
        ho = 0.5 * sub * (double)(1 << (P.max_rung - r));
        if (last) atomicAdd(&hist[r], 1);
      }
      ++updates;
      s.vx[i] = v[0] + ho * a[0];
      s.vy[i] = v[1] + ho * a[1];
      s.vz[i] = v[2] + ho * a[2];
      s.u[i] = u + ho * s.dudt[i];
      s.sxx[i] = S[0] + ho * dS[0];
      s.syy[i] = S[1] + ho * dS[1];
      s.sxy[i] = S[2] + ho * dS[2];
      s.sxz[i] = S[3] + ho * dS[3];
      s.syz[i] = S[4] + ho * dS[4];
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
    acc[0] += m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);   // halved below (exact)
    acc[1] += m * u;
    acc[2] += m * from_t(phi);
    acc[3] += m * v[0];
    acc[4] += m * v[1];
    acc[5] += m * v[2];
    acc[6] += m * (y * v[2] - z * v[1]);
    acc[7] += m * (z * v[0] - x * v[2]);
    acc[8] += m * (x * v[1] - y * v[0]);
    if (!fixed) {
      const T H = to_t<T>(s.h[i]);
      const T ax = to_t<T>(a[0]), ay = to_t<T>(a[1]), az = to_t<T>(a[2]);
      const T am = sqrt(ax * ax + ay * ay + az * az);
      const T ta = am > T(0) ? eta_a * sqrt(H / am) : T(INFINITY);   // Eq. 38, eps = H
      const T tc = eta_c * H / to_t<T>(w.vsig[i]);                    // Eq. 39
      tmin = tmin_(tmin, tmin_(ta, tc));
    }
  }
  // block sums in a fixed order: every thread parks its nine partial sums
  // in shared memory; warp q then reduces sum q (warp 0 also sum 8) over
  // the block, each lane adding kBlock / 32 values in sequence before a
  // shuffle tree. Nine shuffle trees per thread would cost three times the
  // FP64 additions, and this kernel is bound by the FP64 unit.
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNSum; ++k) red[k][threadIdx.x] = acc[k];
  const double tm = wmin(from_t(tmin));
  if (lane == 0) redt[wi] = tm;
  __syncthreads();
  static_assert(kNSum <= 2 * (kBlock / 32) && kNSum > kBlock / 32, "one or two sums per warp");
  for (int k = wi; k < kNSum; k += kBlock / 32) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kBlock / 32; ++q) t += red[k][32 * q + lane];
    t = wsum(t);
    if (lane == 0) partials[blockIdx.x * kNSum + k] = k == 0 ? 0.5 * t : t;
  }
  const int wu = wsum(updates);
  if (lane == 0 && wu) atomicAdd(&st->updates, (unsigned long long)wu);
  if (threadIdx.x < 16 && hist[threadIdx.x]) atomicAdd(&st->rung_hist[threadIdx.x], hist[threadIdx.x]);
  if (threadIdx.x == 0) {
    double t = INFINITY;
    for (int q = 0; q < kBlock / 32; ++q) t = fmin(t, redt[q]);
    atomicMin(&R.dtmin_enc, enc_d(t));
  }
}

// Per system (one block each): fixed-order sum of its chunks' partials,
// strided per thread, then a tree over the block.
__global__ void __launch_bounds__(kBlock) k_reduce_final(const double *partials, KParams P) {
  __shared__ double red[kBlock / 32];
  SysRec &R = P.sys[blockIdx.x];
  const int b0 = R.chunk_off, b1 = P.sys_chunk[blockIdx.x + 1];
  for (int k = 0; k < kNSum; ++k) {
    double t = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) t += partials[b * kNSum + k];
    t = wsum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < kBlock / 32; ++q) s += red[q];
      R.sums[k] = s;
    }
    __syncthreads();
  }
}

// Hierarchical steps: at the start of a big step every moving particle
// takes the rung its criteria ask for (from the last derivatives; every
// particle is at the same time, so any rung is aligned).
__global__ void __launch_bounds__(kBlock) k_rung_init(sph_state s, Work w, int64_t n, KParams P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (s.flags[i] & SPH_FLAG_FIXED) {
      w.rung[i] = 0;
      continue;
    }
    const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, i) : 0;
    const double am = sqrt(s.ax[i] * s.ax[i] + s.ay[i] * s.ay[i] + s.az[i] * s.az[i]);
    const double h = s.h[i];
    const double ta = am > 0.0 ? P.eta_a * sqrt(h / am) : INFINITY;
    const double tc = P.eta_c * h / w.vsig[i];
    w.rung[i] = rung_want(P, P.dt[sy] * P.sub_scale, ta < tc ? ta : tc);
  }
}

cudaError_t launch_rung_init(sph_ctx *c) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  k_rung_init<<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->kp);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// ------------------------------------------------- active-particle list
// Hierarchical steps of one system: the sorted positions of the particles
// whose step ends with the current substep, in sorted (Morton) order, so
// that 32 consecutive entries are a spatially compact bucket of active
// particles. Three passes over tiles of kActTile particles: per-tile
// counts, one exclusive scan of the counts (which also gives n_active),
// and the stable scatter.
constexpr int kActTile = 2048;

__global__ void __launch_bounds__(kBlock) k_active_count(int64_t n, KParams P, int *tiles) {
  __shared__ int wc[kBlock / 32];
  const int64_t t0 = (int64_t)blockIdx.x * kActTile;
  int c = 0;
  for (int64_t i = t0 + threadIdx.x; i < n && i < t0 + kActTile; i += blockDim.x)
    c += rung_active(P, i) ? 1 : 0;
  c = wsum(c);
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < kBlock / 32; ++q) t += wc[q];
    tiles[blockIdx.x] = t;
  }
}

// One block: exclusive scan of the tile counts in place, in chunks of
// kBlock tiles, and the total into the status record.
__global__ void __launch_bounds__(kBlock) k_active_scan(int *tiles, int ntiles, Status *st) {
  __shared__ int wsums[kBlock / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b0 = 0; b0 < ntiles; b0 += kBlock) {
    const int k = b0 + threadIdx.x;
    const int v = k < ntiles ? tiles[k] : 0;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int u = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += u;
    }
    if (lane == 31) wsums[w] = inc;
    __syncthreads();
    int before = carry;
    for (int q = 0; q < w; ++q) before += wsums[q];
    if (k < ntiles) tiles[k] = before + inc - v;
    __syncthreads();
    if (threadIdx.x == kBlock - 1) carry = before + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) st->n_active = carry;
}

__global__ void __launch_bounds__(kBlock) k_active_scatter(int64_t n, KParams P, const int *tiles,
                                                          int *act, unsigned *err) {
  __shared__ int wc[kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * kActTile;
  int base = tiles[blockIdx.x];
  // the tile in rounds of kBlock particles, each round in order
  for (int64_t r0 = t0; r0 < n && r0 < t0 + kActTile; r0 += blockDim.x) {
    const int64_t i = r0 + threadIdx.x;
    const bool a = i < n && i < t0 + kActTile && rung_active(P, i);
    const unsigned bal = __ballot_sync(kFull, a);
    if (lane == 0) wc[w] = __popc(bal);
    __syncthreads();
    int before = base;
    for (int q = 0; q < w; ++q) before += wc[q];
    if (a) act[checked(before + __popc(bal & ((1u << lane) - 1u)), n, err)] = (int)i;
    int total = 0;
    for (int q = 0; q < kBlock / 32; ++q) total += wc[q];
    __syncthreads();
    base += total;
  }
}

cudaError_t launch_compact_active(sph_ctx *c) {
  const int nt = (int)((c->n + kActTile - 1) / kActTile);
  k_active_count<<<nt, kBlock, 0, c->stream>>>(c->n, c->kp, c->w.act_tiles);
  k_active_scan<<<1, kBlock, 0, c->stream>>>(c->w.act_tiles, nt, c->d_status);
  k_active_scatter<<<nt, kBlock, 0, c->stream>>>(c->n, c->kp, c->w.act_tiles, c->w.act,
                                                 &c->d_status->err);
  c->nlaunch += 3;
  return cudaGetLastError();
}

cudaError_t launch_kick(sph_ctx *c, int kick) {
  if (c->kp.precision == SPH_FP32K)
    k_kick<float><<<c->nchunks, kBlock, 0, c->stream>>>(c->st, c->src, c->w, kick, c->kp,
                                                         c->partials, c->d_status);
  else
    k_kick<double><<<c->nchunks, kBlock, 0, c->stream>>>(c->st, c->src, c->w, kick, c->kp,
                                                          c->partials, c->d_status);
  k_reduce_final<<<c->nsys, kBlock, 0, c->stream>>>(c->partials, c->kp);
  c->nlaunch += 2;
  return cudaGetLastError();
}

}  // namespace sphk
