// sph_update.cu -- closing and opening kicks with radial return (§2.4,
// Eq. 41-43), FP64 global sums (energies, momentum, angular momentum Eq. 46)
// and the time-step minimum of Eq. 38-39.
#include "sph_kick.cuh"

namespace sphk {

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
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    // hierarchical steps: before the last substep only the kicked particles
    // matter (the sums and the time step are those of the big step's end)
    if (!last && !rung_active(P, i)) continue;
    const KickIn d = {{s.ax[i], s.ay[i], s.az[i]},
                      s.dudt[i],
                      {s.dsxx[i], s.dsyy[i], s.dsxy[i], s.dsxz[i], s.dsyz[i]},
                      w.edot2[i],
                      w.vsig[i]};
    kick_particle<T>(s, src, w, P, i, kick != 0, sub, last, copy, d, acc, tmin, updates, hist);
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

// Fixed-order sums of partial sums over units [b0, b1): each thread sums a
// strided subset, all nine sums at once and four units per round so that
// the loads overlap, then a tree over the block, one warp per sum. The
// result goes to out[0..kNSum).
constexpr int kReduceThreads = 1024;
__device__ __forceinline__ void reduce_units(const double *partials, int b0, int b1,
                                             double *out) {
  __shared__ double red[kNSum][kReduceThreads / 32];
  double t[kNSum] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  constexpr int kU = 4;
  int b = b0 + threadIdx.x;
  for (; b + (kU - 1) * kReduceThreads < b1; b += kU * kReduceThreads) {
    double v[kU][kNSum];
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int k = 0; k < kNSum; ++k) v[u][k] = partials[(int64_t)(b + u * kReduceThreads) * kNSum + k];
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int k = 0; k < kNSum; ++k) t[k] += v[u][k];
  }
  for (; b < b1; b += kReduceThreads)
#pragma unroll
    for (int k = 0; k < kNSum; ++k) t[k] += partials[(int64_t)b * kNSum + k];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNSum; ++k) {
    const double s = wsum(t[k]);
    if (lane == 0) red[k][w] = s;
  }
  __syncthreads();
  if (w < kNSum) {
    const double s = wsum(red[w][lane]);   // kReduceThreads / 32 = 32 warp sums
    if (lane == 0) out[w] = s;
  }
}

// Per system (one block each): its sums from the partials of its reduction
// chunks (k_kick) or from those of its reduction tiles (the force pass's
// kick, after k_reduce_tiles).
__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *partials, KParams P,
                                                                int per_tile) {
  SysRec &R = P.sys[blockIdx.x];
  const int b0 = per_tile ? P.sys_tile[blockIdx.x] : R.chunk_off;
  const int b1 = per_tile ? P.sys_tile[blockIdx.x + 1] : P.sys_chunk[blockIdx.x + 1];
  reduce_units(partials, b0, b1, R.sums);
}

// One block per reduction tile: the fixed-order sum of the partials of its
// kRedTile buckets.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_tiles(const double *partials, KParams P,
                                                                double *tile_partials) {
  const int t = blockIdx.x;
  reduce_units(partials, P.red_tile[t], P.red_tile_end[t], tile_partials + (int64_t)t * kNSum);
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
  k_reduce_final<<<c->nsys, kReduceThreads, 0, c->stream>>>(c->partials, c->kp, 0);
  c->nlaunch += 2;
  return cudaGetLastError();
}

// The sums of a step whose force pass kicked every particle (per-bucket
// partials): per tile of kRedTile buckets, then per system.
cudaError_t launch_reduce_buckets(sph_ctx *c) {
  k_reduce_tiles<<<c->kp.nred_tiles, kReduceThreads, 0, c->stream>>>(c->partials, c->kp,
                                                                     c->tile_partials);
  k_reduce_final<<<c->nsys, kReduceThreads, 0, c->stream>>>(c->tile_partials, c->kp, 1);
  c->nlaunch += 2;
  return cudaGetLastError();
}

}  // namespace sphk
