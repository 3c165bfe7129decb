// sph_update.cu -- closing and opening kicks with radial return (§2.4,
// Eq. 41-43), FP64 global sums (energies, momentum, angular momentum Eq. 46)
// and the time-step minimum of Eq. 38-39.
#include "sph_kick.cuh"

namespace sphk {

// The step's reductions in a fixed order. Per reduction tile (64 buckets,
// 2048 sorted positions of one system; one block): every thread adds the
// terms of 8 particles in sequence, then the block's sums are formed
// through shared memory, warp q adding sum q (warp 0 also sum 8) over the
// block, each lane 8 values in sequence before a shuffle tree. A shuffle
// tree per sum and thread would cost five FP64 additions per value, and
// FP64 instructions are the expensive ones here. Per system (one block):
// the tiles' slots in the same way.
constexpr int kReduceThreads = 256;
static_assert(kRedTile * 32 == 8 * kReduceThreads, "8 particles per thread and tile");
static_assert(kNSum <= 2 * (kReduceThreads / 32) && kNSum > kReduceThreads / 32,
              "one or two sums per warp");

// Block-wide fixed-order reduction of per-thread values acc[0..kNSum) (sums)
// and tm (minimum); thread 0 holds nothing special, out[0..kNSlot) gets the
// result (written by several warps; read after a __syncthreads).
__device__ __forceinline__ void block_slots(const double acc[kNSum], double tm, double *out) {
  __shared__ double red[kNSum][kReduceThreads];
  __shared__ double redt[kReduceThreads / 32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNSum; ++k) red[k][threadIdx.x] = acc[k];
  tm = __longlong_as_double(wmin(__double_as_longlong(tm)));
  if (lane == 0) redt[wi] = tm;
  __syncthreads();
  for (int k = wi; k < kNSum; k += kReduceThreads / 32) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kReduceThreads / 32; ++q) t += red[k][32 * q + lane];
    t = wsum(t);
    if (lane == 0) out[k] = t;
  }
  if (threadIdx.x == 0) {
    double t = INFINITY;
    for (int q = 0; q < kReduceThreads / 32; ++q) t = min_crit(t, redt[q]);
    out[kSlotDt] = t;
  }
}

// Sorted positions [p0, p1) of reduction tile t and its system.
__device__ __forceinline__ int tile_range(const KParams &P, int t, int64_t &p0, int64_t &p1) {
  const int b0 = P.red_tile[t], b1 = P.red_tile_end[t];
  const int sy = P.nsys > 1 ? sys_lookup(P.sys_bucket, P.nsys, b0) : 0;
  const SysRec &R = P.sys[sy];
  p0 = R.begin + (int64_t)(b0 - R.bucket_off) * 32;
  p1 = R.begin + (int64_t)(b1 - R.bucket_off) * 32;
  if (p1 > R.end) p1 = R.end;
  return sy;
}

// kick = 1: close to i (v, u, S alike), rescale S with Y at (rho_i, u_i),
// accumulate 1/2 edot:edot dt, sum diagnostics at i, open to i+1/2.
// kick = 0: diagnostics and time step of the state as it stands. The
// integration and the sums are FP64; the EOS, yield and time-step criteria
// are evaluated in T. One block per reduction tile; each thread kicks 8
// particles of it and adds their terms in sequence (without contraction),
// then the tile's slots are formed (block_slots): the order of
// k_reduce_tiles over the terms that the force pass leaves when it kicks,
// so both ways give the same bits.
// src: where v, u, S and the strain invariant are read (the step's read
// view: their permuted copies when the permutation did not copy them
// back); s: where they are written, for every particle then.
// Four blocks per SM (64 registers, some spilled): the kernel is bound by
// its FP64 unit, and 32 resident warps keep it busier than 16 (two blocks at
// 99 registers: 15 % slower) or 24 (three: 8 % slower); five and six blocks
// spill more than they gain.
template <typename T>
__global__ void __launch_bounds__(kReduceThreads, 4) k_kick(sph_state s, sph_state src, Work w,
                                                           int kick, KParams P,
                                                           double *tile_partials, Status *st) {
  const bool copy = src.vx != s.vx;   // lazy step: write every particle
  __shared__ int hist[16];
  if (threadIdx.x < 16) hist[threadIdx.x] = 0;
  __syncthreads();
  int64_t p0, p1;
  const int sy = tile_range(P, blockIdx.x, p0, p1);
  // the substep; without rungs the step (sub_scale = 1)
  const double sub = kick ? P.dt[sy] * P.sub_scale : 0.0;
  const bool last = P.substep + 1 == (1 << P.max_rung);   // every particle's step ends
  int updates = 0;
  double acc[kNSum] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double tm = INFINITY;
  for (int64_t i = p0 + threadIdx.x; i < p1; i += kReduceThreads) {
    // hierarchical steps: before the last substep only the kicked particles
    // matter (the sums and the time step are those of the big step's end)
    if (!last && !rung_active(P, i)) continue;
    const KickIn d = {{s.ax[i], s.ay[i], s.az[i]},
                      s.dudt[i],
                      {s.dsxx[i], s.dsyy[i], s.dsxy[i], s.dsxz[i], s.dsyz[i]},
                      w.edot2[i],
                      w.vsig[i]};
    double term[kNSum], tcr;
    kick_particle<T>(s, src, w, P, i, kick != 0, sub, last, copy, d, term, &tcr, updates, hist);
#pragma unroll
    for (int k = 0; k < kNSum; ++k) acc[k] = __dadd_rn(acc[k], term[k]);
    tm = min_crit(tm, tcr);
  }
  block_slots(acc, tm, tile_partials + (int64_t)blockIdx.x * kNSlot);
  const int wu = wsum(updates);
  if ((threadIdx.x & 31) == 0 && wu) atomicAdd(&st->updates, (unsigned long long)wu);
  __syncthreads();
  if (threadIdx.x < 16 && hist[threadIdx.x]) atomicAdd(&st->rung_hist[threadIdx.x], hist[threadIdx.x]);
}

// The terms the force pass left when it kicked, in k_kick's order.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_tiles(Work w, KParams P,
                                                                double *tile_partials) {
  int64_t p0, p1;
  tile_range(P, blockIdx.x, p0, p1);
  double acc[kNSum] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double tm = INFINITY;
  for (int64_t i = p0 + threadIdx.x; i < p1; i += kReduceThreads) {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) acc[k] = __dadd_rn(acc[k], w.terms[k][i]);
    tm = min_crit(tm, w.tcrit[i]);
  }
  block_slots(acc, tm, tile_partials + (int64_t)blockIdx.x * kNSlot);
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *tile_partials,
                                                                KParams P) {
  __shared__ double out[kNSlot];
  SysRec &R = P.sys[blockIdx.x];
  double acc[kNSum] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double tm = INFINITY;
  for (int t = P.sys_tile[blockIdx.x] + threadIdx.x; t < P.sys_tile[blockIdx.x + 1];
       t += kReduceThreads) {
#pragma unroll
    for (int k = 0; k < kNSum; ++k) acc[k] += tile_partials[(int64_t)t * kNSlot + k];
    tm = min_crit(tm, tile_partials[(int64_t)t * kNSlot + kSlotDt]);
  }
  block_slots(acc, tm, out);
  __syncthreads();
  if (threadIdx.x < kNSum) R.sums[threadIdx.x] = threadIdx.x == 0 ? 0.5 * out[0] : out[threadIdx.x];
  if (threadIdx.x == 0) atomicMin(&R.dtmin_enc, enc_d(out[kSlotDt]));
}

// Hierarchical steps: at the start of a big step every moving particle
// takes the rung its criteria ask for (from the last derivatives; every
// particle is at the same time, so any rung is aligned).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_rung_init(sph_state s, Work w, int64_t n, KParams P) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (s.flags[i] & SPH_FLAG_FIXED) {
      w.rung[i] = 0;
      continue;
    }
    const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, i) : 0;
    const double a[3] = {s.ax[i], s.ay[i], s.az[i]};
    w.rung[i] = rung_want(P, P.dt[sy] * P.sub_scale, from_t(crit_t<T>(P, a, s.h[i], w.vsig[i])));
  }
}

cudaError_t launch_rung_init(sph_ctx *c) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  if (c->kp.precision == SPH_FP32K)
    k_rung_init<float><<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->kp);
  else
    k_rung_init<double><<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->kp);
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

// The step's sums from the per-particle terms: per tile of kRedTile
// buckets, then per system.
cudaError_t launch_reduce_buckets(sph_ctx *c) {
  k_reduce_tiles<<<c->kp.nred_tiles, kReduceThreads, 0, c->stream>>>(c->w, c->kp,
                                                                     c->tile_partials);
  k_reduce_final<<<c->nsys, kReduceThreads, 0, c->stream>>>(c->tile_partials, c->kp);
  c->nlaunch += 2;
  return cudaGetLastError();
}

cudaError_t launch_kick(sph_ctx *c, int kick) {
  const int nt = c->kp.nred_tiles;
  if (c->kp.precision == SPH_FP32K)
    k_kick<float><<<nt, kReduceThreads, 0, c->stream>>>(c->st, c->src, c->w, kick, c->kp,
                                                        c->tile_partials, c->d_status);
  else
    k_kick<double><<<nt, kReduceThreads, 0, c->stream>>>(c->st, c->src, c->w, kick, c->kp,
                                                         c->tile_partials, c->d_status);
  k_reduce_final<<<c->nsys, kReduceThreads, 0, c->stream>>>(c->tile_partials, c->kp);
  c->nlaunch += 2;
  return cudaGetLastError();
}

}  // namespace sphk
