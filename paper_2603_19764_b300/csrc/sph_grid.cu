// sph_grid.cu -- drift, bounding box, uniform cell grid, Morton keys, stable
// LSD radix sort and the in-place permutation of the particle arrays.
//
// The paper finds neighbours with pkdgrav3's tree (§2.1, §4). Here a uniform
// grid of cell edge L_c = max H over Morton-ordered cells takes its place:
// particles are sorted by the Morton key of their cell so that every cell is
// a contiguous index range and consecutive particles are close in space.
#include "sph_internal.cuh"

namespace sphk {

// ---------------------------------------------------------------- status
// counters = 0 (substeps after the first of a big step): the work counters
// keep adding up; the per-system boxes and extrema always restart.
__global__ void k_reset_status(Status *st, SysRec *sys, int nsys, int full, int counters) {
  if (threadIdx.x < 16 && counters) st->rung_hist[threadIdx.x] = 0;
  if (threadIdx.x == 0 && counters) {
    st->updates = 0;
    st->max_sweeps = 0;
    st->n_unconv = 0;
    st->n_capped = 0;
    st->n_cfallback = 0;
    st->pairs_density = 0;
    st->pairs_force = 0;
    st->cand_density = 0;
    st->cand_force = 0;
    st->groups_density = 0;
    st->groups_force = 0;
    st->sweeps_total = 0;
    st->n_expanded = 0;
  }
  if (threadIdx.x == 0 && full) st->err = 0;
  for (int k = threadIdx.x; k < nsys; k += blockDim.x) {
    SysRec &r = sys[k];
    for (int a = 0; a < 3; ++a) {
      r.lo_enc[a] = ~0ull;
      r.hi_enc[a] = 0ull;
    }
    r.hmax_enc = 0ull;
    r.hmax2_enc = 0ull;
    r.dtmin_enc = ~0ull;
    r.disp_enc = 0ull;
  }
}

cudaError_t launch_reset_status(sph_ctx *c, int full) {
  k_reset_status<<<1, 256, 0, c->stream>>>(c->d_status, c->d_sys, c->nsys, full,
                                           c->kp.substep == 0);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------ drift + bounding box
// x_i = x_{i-1} + dt v_{i-1/2} for moving particles (§2.4), then the box of
// every system's positions and its largest H. Runs before the sort, so a
// particle's system comes from its id. A block covers kDriftChunk
// consecutive particles, which belong to one system except near system
// boundaries (systems stay contiguous through every sort). Each thread
// keeps running extrema for the system of its current particle and flushes
// them with atomics only when the system changes; at the end the block
// combines the threads that share one system (the common case) before a
// single set of atomics.
// Running extrema are kept as order-preserving 64-bit encodings (enc_d), so
// that the per-particle min / max run on the integer pipe: FP64 min / max
// instructions share the FP64 unit, which runs at 1/64 of the FP32 rate.
__device__ __forceinline__ void flush_box(SysRec &r, const unsigned long long (&lo)[3],
                                          const unsigned long long (&hi)[3],
                                          unsigned long long hm, unsigned long long dm) {
  for (int a = 0; a < 3; ++a) {
    atomicMin(&r.lo_enc[a], lo[a]);
    atomicMax(&r.hi_enc[a], hi[a]);
  }
  atomicMax(&r.hmax_enc, hm);
  if (dm) atomicMax(&r.disp_enc, dm);
}

// finite by the exponent field alone (no FP64 instruction)
__device__ __forceinline__ bool finite_bits(double d) {
  return ((__double_as_longlong(d) >> 52) & 0x7ff) != 0x7ff;
}

constexpr int kDriftChunk = 8 * kBlock;
constexpr unsigned long long kEncMax = ~0ull, kEncMin = 0ull;

// PER: a periodic box (a template parameter, so that closed boxes run no
// FP64 compare or wrap: the compiler evaluates a run-time branch's cheap
// sides unconditionally)
// TRACK: also record each system's largest coordinate change (hierarchical
// steps, whose next substep may keep this order and search a skin that
// wide)
template <bool PER, bool TRACK>
__global__ void __launch_bounds__(kBlock) k_drift_bbox(sph_state s, int64_t n, KParams P,
                                                      int do_drift) {
  __shared__ unsigned long long red[8][kBlock / 32];
  __shared__ int wsys[kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long lo[3] = {kEncMax, kEncMax, kEncMax}, hi[3] = {kEncMin, kEncMin, kEncMin};
  unsigned long long hm = kEncMin, dm = kEncMin;   // largest H; largest coordinate change
  int cur = -1;   // system of the running extrema (-1: none)
  const int64_t c0 = (int64_t)blockIdx.x * kDriftChunk;
  const int64_t c1 = c0 + kDriftChunk < n ? c0 + kDriftChunk : n;
  for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, s.id[i]) : 0;
    double p[3] = {s.x[i], s.y[i], s.z[i]};
    if (do_drift && !(s.flags[i] & SPH_FLAG_FIXED)) {
      const double dt = P.dt[sy] * P.sub_scale;   // the substep (the step without rungs)
      const double p0[3] = {p[0], p[1], p[2]};
      p[0] += dt * s.vx[i];
      p[1] += dt * s.vy[i];
      p[2] += dt * s.vz[i];
      if (TRACK) {   // the coordinate change, as the order-preserving encoding
        for (int a = 0; a < 3; ++a) {
          const double d = p[a] - p0[a];
          const unsigned long long e = enc_d(fabs(d));
          dm = finite_bits(d) && e > dm ? e : dm;
        }
      }
      if (PER) {   // back into [box_lo, box_hi): one box length at most
        for (int a = 0; a < 3; ++a) {
          if (p[a] >= P.box_hi[a]) p[a] -= P.box_len[a];
          else if (p[a] < P.box_lo[a]) p[a] += P.box_len[a];
        }
      }
      s.x[i] = p[0];
      s.y[i] = p[1];
      s.z[i] = p[2];
    }
    if (sy != cur) {
      if (cur >= 0) flush_box(P.sys[cur], lo, hi, hm, dm);
      cur = sy;
      for (int a = 0; a < 3; ++a) {
        lo[a] = kEncMax;
        hi[a] = kEncMin;
      }
      hm = kEncMin;
      dm = kEncMin;
    }
    // a non-finite position is left out of the box (the step's checks
    // report it), as the FP64 min / max would
    for (int a = 0; a < 3; ++a) {
      if (!finite_bits(p[a])) continue;
      const unsigned long long e = enc_d(p[a]);
      lo[a] = e < lo[a] ? e : lo[a];
      hi[a] = e > hi[a] ? e : hi[a];
    }
    const unsigned long long eh = enc_d(s.h[i]);
    hm = eh > hm ? eh : hm;
  }
  // threads of a warp with one common system reduce by shuffles, warps of
  // a block with one common system through shared memory
  int any = -1;   // a system held by some lane of the warp (lane 0 first)
  {
    const unsigned has = __ballot_sync(kFull, cur >= 0);
    if (has) any = __shfl_sync(kFull, cur, __ffs(has) - 1);
  }
  const bool warp_uniform = __all_sync(kFull, cur < 0 || cur == any);
  unsigned long long v[8] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], hm, dm};
  if (warp_uniform) {
    for (int k = 0; k < 3; ++k) v[k] = wmin(v[k]);
    for (int k = 3; k < 8; ++k) v[k] = wmax(v[k]);
  } else if (cur >= 0) {
    flush_box(P.sys[cur], lo, hi, hm, dm);   // mixed warp: every lane on its own
  }
  if (lane == 0) {
    wsys[w] = warp_uniform ? any : -2;   // -1: no particle, -2: flushed
    for (int k = 0; k < 8; ++k) red[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int sb = -1;
    bool one = true;
    for (int q = 0; q < kBlock / 32; ++q) {
      if (wsys[q] == -1) continue;
      if (wsys[q] == -2 || (sb >= 0 && wsys[q] != sb)) one = false;
      else sb = wsys[q];
    }
    if (one && sb >= 0) {
      unsigned long long b[8] = {kEncMax, kEncMax, kEncMax, kEncMin, kEncMin, kEncMin, kEncMin,
                                 kEncMin};
      for (int q = 0; q < kBlock / 32; ++q) {
        if (wsys[q] < 0) continue;
        for (int k = 0; k < 3; ++k) b[k] = red[k][q] < b[k] ? red[k][q] : b[k];
        for (int k = 3; k < 8; ++k) b[k] = red[k][q] > b[k] ? red[k][q] : b[k];
      }
      const unsigned long long bl[3] = {b[0], b[1], b[2]}, bh[3] = {b[3], b[4], b[5]};
      flush_box(P.sys[sb], bl, bh, b[6], b[7]);
    } else {
      for (int q = 0; q < kBlock / 32; ++q) {
        if (wsys[q] < 0) continue;
        const unsigned long long bl[3] = {red[0][q], red[1][q], red[2][q]};
        const unsigned long long bh[3] = {red[3][q], red[4][q], red[5][q]};
        flush_box(P.sys[wsys[q]], bl, bh, red[6][q], red[7][q]);
      }
    }
  }
}

cudaError_t launch_drift_bbox(sph_ctx *c, int do_drift) {
  const int blocks = (int)((c->n + kDriftChunk - 1) / kDriftChunk);
  if (c->kp.periodic)
    k_drift_bbox<true, false><<<blocks, kBlock, 0, c->stream>>>(c->st, c->n, c->kp, do_drift);
  else if (c->kp.max_rung > 0)
    k_drift_bbox<false, true><<<blocks, kBlock, 0, c->stream>>>(c->st, c->n, c->kp, do_drift);
  else
    k_drift_bbox<false, false><<<blocks, kBlock, 0, c->stream>>>(c->st, c->n, c->kp, do_drift);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------ grid setup
// Per system: cell edge L_c = max H; at most 2^axis_bits cells per axis and
// the system's cell capacity in all, growing L_c by 2^(1/3) until both hold.
// Then the systems' cell ranges are laid out one after the other. In a
// periodic box the grid starts at box_lo and its ceil(box / L_c) cells per
// axis cover [box_lo, box_hi) (the last one may reach past box_hi, where no
// particle lies).
// keep = 1: the grid, the cells and the order stay those of the last sort
// (hierarchical substeps that do not re-sort); only the staging skin (this
// drift's largest coordinate change, the only one since that sort) and the
// force pass's starting search radius are set.
__global__ void k_grid_setup(Status *st, SysRec *sys, int nsys, int axis_bits, KParams P,
                             int keep) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (keep) {
    for (int k = 0; k < nsys; ++k) {
      SysRec &r = sys[k];
      const double d = r.disp_enc ? dec_d(r.disp_enc) : 0.0;
      r.skin = d * (1.0 + 1e-6);
      r.skinf = __double2float_ru(r.skin);
      // the force pass's search bound (max H) widened by the skin
      if (P.act) r.hmax2_enc = enc_d(dec_d(r.hmax_enc) + r.skin);
    }
    return;
  }
  const double max_axis = (double)(1 << axis_bits);
  int off = 0, bits = 0;
  for (int k = 0; k < nsys; ++k) {
    SysRec &r = sys[k];
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = P.periodic ? P.box_lo[a] : dec_d(r.lo_enc[a]);
      hi[a] = P.periodic ? P.box_hi[a] : dec_d(r.hi_enc[a]);
    }
    double L = dec_d(r.hmax_enc);
    const double ext = fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    if (!(L > 1e-30 * ext) || !(L > 0.0)) L = fmax(ext, 1.0) * 1e-3;
    int d[3] = {1, 1, 1};
    bool ok = false;
    for (int it = 0; it < 200 && !ok; ++it) {
      long long tot = 1;
      ok = true;
      for (int a = 0; a < 3; ++a) {
        const double kk = P.periodic ? fmax(ceil((hi[a] - lo[a]) / L), 1.0)
                                     : floor((hi[a] - lo[a]) / L) + 1.0;
        if (!(kk <= max_axis)) ok = false;
        d[a] = (int)fmin(fmax(kk, 1.0), 2.0 * max_axis);
        tot *= d[a];
      }
      if (tot > r.cell_cap) ok = false;
      if (!ok) L *= 1.2599210498948732;
    }
    if (!ok) {  // non-finite box: one cell holding the whole system
      d[0] = d[1] = d[2] = 1;
      L = INFINITY;
      atomicOr(&st->err, ERR_NONFINITE);
    }
    // the force pass's search radius covers the largest H: the density
    // solve raises it for the particles it solves; when it solves only the
    // active list, everyone else's H must be in it from the start
    if (P.act) r.hmax2_enc = r.hmax_enc;
    Grid &g = r.grid;
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = lo[a];
      g.dims[a] = d[a];
    }
    g.L = L;
    g.invL = 1.0 / L;
    g.Lf = (float)L;
    g.invLf = (float)(1.0 / L);
    g.ncells = d[0] * d[1] * d[2];
    g.cell_off = off;
    r.skin = 0.0;
    r.skinf = 0.f;
    off += g.ncells;
    for (int a = 0; a < 3; ++a)
      if (d[a] > 1) bits = max(bits, 32 - __clz(d[a] - 1));
  }
  // the sort keys hold the system index right above the Morton bits the
  // grids use, so that a single system or a batch of small ones needs
  // fewer radix passes (the order of the keys is the same)
  st->key_shift = 3 * bits;
  st->key_or = 0u;
  st->total_cells = off;
}

cudaError_t launch_grid_setup(sph_ctx *c, int keep) {
  k_grid_setup<<<1, 32, 0, c->stream>>>(c->d_status, c->d_sys, c->nsys, c->kp.axis_bits, c->kp,
                                        keep);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// Cell index floor((x - lo) / L) clamped to [0, dim): the scaled offset in
// FP64, its floor from the IEEE 754 layout in integer arithmetic (no
// conversion instruction, which would run on the FP64 unit).
__device__ __forceinline__ int cell_coord(double x, double lo, double invL, int dim) {
  const long long b = __double_as_longlong((x - lo) * invL);
  if (b < 0x3ff0000000000000LL) return 0;   // below 1 (negative included)
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e >= 31) return dim - 1;              // 2^31 and beyond, infinity, NaN
  const long long m = (b & 0xfffffffffffffLL) | (1LL << 52);
  const int k = (int)(m >> (52 - e));
  return k >= dim ? dim - 1 : k;
}

// Key = system << key_shift | Morton code of the cell within the system
// (key_shift: three times the Morton bits per axis the grids need); values
// start as the identity. The OR of all keys tells the sort which passes
// it can leave out.
__global__ void __launch_bounds__(kBlock) k_keys(sph_state s, int64_t n, KParams P, unsigned *keys,
                                                int *vals, Status *st) {
  const int shift = st->key_shift;
  unsigned o = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, s.id[i]) : 0;
    const Grid &g = P.sys[sy].grid;
    const double invL = g.invL;
    const int cx = cell_coord(s.x[i], g.lo[0], invL, g.dims[0]);
    const int cy = cell_coord(s.y[i], g.lo[1], invL, g.dims[1]);
    const int cz = cell_coord(s.z[i], g.lo[2], invL, g.dims[2]);
    const unsigned k = ((unsigned)sy << shift) | morton3(cx, cy, cz);
    keys[i] = k;
    vals[i] = (int)i;
    o |= k;
  }
  o = __reduce_or_sync(kFull, o);
  if ((threadIdx.x & 31) == 0 && o) atomicOr(&st->key_or, o);
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) pairs, 8-bit digits, up to four
// passes. Per pass: tile histograms (digit-major), one exclusive scan, and a
// stable scatter in which each key's rank inside its tile comes from warp
// match masks plus per-warp digit counts. The kernels of a pass whose digit
// and every higher one are zero in all keys return at once (sort_passes);
// the sorted pairs are then in the buffers of the last pass that ran.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned *keys, int n, int shift,
                                                             unsigned *hist, int ntiles,
                                                             const Status *st) {
  if ((st->key_or >> shift) == 0u) return;
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kTile;
  for (int k = 0; k < kSortItems; ++k) {
    const int i = base + k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of the m = 256 * ntiles tile counts (digit-major) in three
// kernels: per-segment totals, a scan of the totals, per-segment scans.
constexpr int kScanSeg = 1024;

__device__ __forceinline__ unsigned block_scan_incl(unsigned v, unsigned *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(kFull, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;
  }
  __syncthreads();
  const unsigned add = w > 0 ? sh[w - 1] : 0u;
  __syncthreads();
  return v + add;
}

__global__ void __launch_bounds__(kScanSeg) k_scan_totals(const unsigned *hist, int m,
                                                          unsigned *tot, int shift,
                                                          const Status *st) {
  if ((st->key_or >> shift) == 0u) return;
  __shared__ unsigned sh[32];
  const int i = blockIdx.x * kScanSeg + threadIdx.x;
  unsigned v = i < m ? hist[i] : 0u;
  v = block_scan_incl(v, sh);
  if (threadIdx.x == kScanSeg - 1) tot[blockIdx.x] = v;
}

// One block, chunks of kScanSeg totals with a running carry.
__global__ void __launch_bounds__(kScanSeg) k_scan_of_totals(unsigned *tot, int nseg, int shift,
                                                             const Status *st) {
  if ((st->key_or >> shift) == 0u) return;
  __shared__ unsigned sh[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int b = 0; b < nseg; b += kScanSeg) {
    const int i = b + threadIdx.x;
    const unsigned v = i < nseg ? tot[i] : 0u;
    const unsigned inc = block_scan_incl(v, sh);
    const unsigned c0 = carry;
    if (i < nseg) tot[i] = c0 + inc - v;   // exclusive
    __syncthreads();
    if (threadIdx.x == kScanSeg - 1) carry = c0 + inc;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanSeg) k_scan_apply(unsigned *hist, int m,
                                                         const unsigned *tot, int shift,
                                                         const Status *st) {
  if ((st->key_or >> shift) == 0u) return;
  __shared__ unsigned sh[32];
  const int i = blockIdx.x * kScanSeg + threadIdx.x;
  const unsigned v = i < m ? hist[i] : 0u;
  const unsigned inc = block_scan_incl(v, sh);
  if (i < m) hist[i] = tot[blockIdx.x] + inc - v;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned *kin, const int *vin,
                                                                unsigned *kout, int *vout, int n,
                                                                int shift, const unsigned *hist,
                                                                int ntiles, Status *st) {
  if ((st->key_or >> shift) == 0u) return;
  unsigned *const err = &st->err;
  constexpr int NW = kSortThreads / 32;
  __shared__ unsigned base[256];
  __shared__ unsigned wcnt[NW][256];
  const int w = threadIdx.x >> 5;
  base[threadIdx.x] = hist[threadIdx.x * ntiles + blockIdx.x];
  for (int k = 0; k < NW; ++k) wcnt[k][threadIdx.x] = 0;
  __syncthreads();
  const int tile0 = blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int i = tile0 + r * kSortThreads + threadIdx.x;
    const bool ok = i < n;
    const unsigned key = ok ? kin[i] : 0u;
    const unsigned d = ok ? ((key >> shift) & 255u) : 256u;   // 256 never matches a real digit
    const unsigned peers = __match_any_sync(kFull, d);
    const unsigned rank_w = __popc(peers & lanemask_lt());
    if (ok && rank_w == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (ok) {
      unsigned pos = base[d] + rank_w;
      for (int k = 0; k < w; ++k) pos += wcnt[k][d];
      pos = (unsigned)checked(pos, n, err);
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    unsigned add = 0;
    for (int k = 0; k < NW; ++k) {
      add += wcnt[k][threadIdx.x];
      wcnt[k][threadIdx.x] = 0;
    }
    base[threadIdx.x] += add;
    __syncthreads();
  }
}

// ------------------------------------------------------------ permutation
// Every array of sph_state is gathered through the sort permutation into a
// scratch block and copied back, so the caller's arrays end up in cell order.
// Within a step the arrays that the step itself recomputes before reading
// them are left out: their values are overwritten in the new order.
constexpr int kNF64 = 29;   // 28 double arrays + id
constexpr int kNI32 = 4;   // mat, flags, count; the rungs of hierarchical steps
constexpr int kNLearn = 5;  // learned form: H_prev, H proposal, three feature pairs

struct PermTable {
  unsigned long long *f64[kNF64 + kNLearn];
  unsigned *i32[kNI32];
  int nf64;    // 8-byte fields in use
  int nback;   // the first nback of them are copied back to the caller's arrays
  int ni32;    // 4-byte fields in use (always copied back)
};

// part 0: every array a step permutes; part 1 (the copy-in of
// sph_step_host is split in two): what the drift, the sort and the density
// solve read -- positions, velocities, H, masses, ids, materials, flags and
// the library's per-particle arrays; part 2: the rest -- u, S, the
// derivatives at i-1 and the strain invariant, which only the predictor and
// the kicks read. lazy: the arrays that a later kernel of the step rewrites
// for every particle (v, H, u, S, the derivatives, the strain invariant) are
// gathered but not copied back (sph_ctx::src reads them from the scratch).
static PermTable perm_table(const sph_state &s, const Work &w, const LearnArgs &L, bool all,
                            bool rungs, int part = 0, bool lazy = false) {
  PermTable t;
  t.nf64 = 0;
  t.ni32 = 0;
  unsigned long long *later[24];   // candidates for the lazy part
  int nl = 0;
  auto add = [&](double *p, bool rewritten) {
    if (lazy && rewritten) later[nl++] = (unsigned long long *)p;
    else t.f64[t.nf64++] = (unsigned long long *)p;
  };
  if (part != 2) {
    add(s.x, false);
    add(s.y, false);
    add(s.z, false);
    add(s.m, false);
    t.f64[t.nf64++] = (unsigned long long *)s.id;
    t.i32[t.ni32++] = (unsigned *)s.mat;
    t.i32[t.ni32++] = (unsigned *)s.flags;
    // rho, Omega and the counts are recomputed in a step only for the
    // particles that are solved: with hierarchical steps they must follow
    // the sort (solved or not), P and c_s are always recomputed
    if (all || rungs) {
      t.f64[t.nf64++] = (unsigned long long *)s.rho;
      t.f64[t.nf64++] = (unsigned long long *)s.omega;
      t.i32[t.ni32++] = (unsigned *)s.nngb;
    }
    if (all) {
      t.f64[t.nf64++] = (unsigned long long *)s.pres;
      t.f64[t.nf64++] = (unsigned long long *)s.cs;
    }
    if (w.rung) t.i32[t.ni32++] = (unsigned *)w.rung;   // hierarchical steps
    // the learned form's per-particle arrays follow their particles
    if (L.hprev) {
      t.f64[t.nf64++] = (unsigned long long *)L.hprev;
      t.f64[t.nf64++] = (unsigned long long *)L.hprop;
      if (L.feat[0])
        for (int k = 0; k < 3; ++k) t.f64[t.nf64++] = (unsigned long long *)L.feat[k];
    }
    add(s.vx, true);
    add(s.vy, true);
    add(s.vz, true);
    add(s.h, true);
  }
  if (part != 1) {
    double *b[16] = {s.u,    s.sxx,  s.syy,  s.sxy,  s.sxz,  s.syz,  s.ax,   s.ay,
                     s.az,   s.dudt, s.dsxx, s.dsyy, s.dsxy, s.dsxz, s.dsyz, s.eps_ii};
    for (int k = 0; k < 16; ++k) add(b[k], true);
  }
  t.nback = t.nf64;
  for (int k = 0; k < nl; ++k) t.f64[t.nf64++] = later[k];
  return t;
}

__global__ void __launch_bounds__(kBlock) k_gather(PermTable t, const int *perm0,
                                                  const int *perm1, int64_t n,
                                                  unsigned long long *tmp, Status *st) {
  // the sort's permutation: in perm1 after an odd number of passes
  const int *perm = (sort_passes(st->key_or) & 1) ? perm1 : perm0;
  unsigned *const err = &st->err;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = checked(perm[i], n, err);
#pragma unroll 8
    for (int f = 0; f < t.nf64; ++f) tmp[f * n + i] = t.f64[f][j];
    unsigned *t32 = (unsigned *)(tmp + t.nf64 * n);
    for (int f = 0; f < t.ni32; ++f) t32[f * n + i] = t.i32[f][j];
  }
}

__global__ void __launch_bounds__(kBlock) k_scatter_back(PermTable t, int64_t n,
                                                        const unsigned long long *tmp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll 8
    for (int f = 0; f < t.nback; ++f) t.f64[f][i] = tmp[f * n + i];
    const unsigned *t32 = (const unsigned *)(tmp + t.nf64 * n);
    for (int f = 0; f < t.ni32; ++f) t.i32[f][i] = t32[f * n + i];
  }
}

// Cell start / end over the sorted keys, and the packed cell coordinates.
__global__ void __launch_bounds__(kBlock) k_clear_cells(int *start, const Status *st) {
  const int nc = st->total_cells;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    start[i] = -1;
}

__global__ void __launch_bounds__(kBlock) k_cells(const unsigned *keys0, const unsigned *keys1,
                                                 int64_t n, KParams P, int *start, int *end,
                                                 int *cc, int max_cells, Status *st) {
  // the sorted keys: in keys1 after an odd number of passes
  const unsigned *keys = (sort_passes(st->key_or) & 1) ? keys1 : keys0;
  unsigned *const err = &st->err;
  const int sh = st->key_shift;
  const unsigned mask = sh >= 32 ? ~0u : ((1u << sh) - 1u);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned k = keys[i];
    const int sy = sh >= 32 ? 0 : (int)(k >> sh);
    const unsigned mc = k & mask;
    const Grid &g = P.sys[sy].grid;
    const int cx = compact1by2(mc), cy = compact1by2(mc >> 1), cz = compact1by2(mc >> 2);
    const int lin = (int)checked(g.cell_off + (cz * g.dims[1] + cy) * g.dims[0] + cx, max_cells,
                                 err);
    cc[i] = cx | (cy << 10) | (cz << 20);
    if (i == 0 || keys[i - 1] != k) start[lin] = (int)i;
    if (i == n - 1 || keys[i + 1] != k) end[lin] = (int)(i + 1);
  }
}

static int grid_for(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  if (b > 148 * 16) b = 148 * 16;
  return (int)(b < 1 ? 1 : b);
}

// Gather and copy back the arrays of one part of the permutation table
// through the last sort's permutation (c->vals), into the scratch block from
// word `base` on. The lazy fields (not copied back) become the read view
// c->src.
static void enqueue_permute(sph_ctx *c, const PermTable &t, int64_t base) {
  const int64_t n = c->n;
  const int gb = grid_for(n, kBlock);
  unsigned long long *tmp = (unsigned long long *)c->tmp + base * n;
  k_gather<<<gb, kBlock, 0, c->stream>>>(t, c->vals, c->vals_alt, n, tmp, c->d_status);
  k_scatter_back<<<gb, kBlock, 0, c->stream>>>(t, n, tmp);
  c->nlaunch += 2;
  for (int f = t.nback; f < t.nf64; ++f) {
    double *permuted = (double *)(tmp + (int64_t)f * n);
    const sph_state &s = c->st;
    sph_state &r = c->src;
    double *const caller[20] = {s.vx,   s.vy,   s.vz,   s.h,    s.u,    s.sxx,  s.syy,
                                s.sxy,  s.sxz,  s.syz,  s.ax,   s.ay,   s.az,   s.dudt,
                                s.dsxx, s.dsyy, s.dsxy, s.dsxz, s.dsyz, s.eps_ii};
    double **view[20] = {&r.vx,   &r.vy,   &r.vz,   &r.h,    &r.u,    &r.sxx,  &r.syy,
                         &r.sxy,  &r.sxz,  &r.syz,  &r.ax,   &r.ay,   &r.az,   &r.dudt,
                         &r.dsxx, &r.dsyy, &r.dsxy, &r.dsxz, &r.dsyz, &r.eps_ii};
    for (int k = 0; k < 20; ++k)
      if ((unsigned long long *)caller[k] == t.f64[f]) *view[k] = permuted;
  }
}

// Words of the scratch block a table's fields take (8-byte fields, then
// the 4-byte ones two to a word).
static int64_t table_words(const PermTable &t) { return t.nf64 + (t.ni32 + 1) / 2; }

cudaError_t launch_permute_rest(sph_ctx *c) {
  // after the first part's fields in the scratch block
  const PermTable first = perm_table(c->st, c->w, c->learn, false, false, 1, c->lazy != 0);
  enqueue_permute(c, perm_table(c->st, c->w, c->learn, false, false, 2, c->lazy != 0),
                  table_words(first));
  return cudaGetLastError();
}

cudaError_t launch_sort_permute(sph_ctx *c, int all, int part) {
  const int64_t n = c->n;
  const int gb = grid_for(n, kBlock);
  Status *const st = c->d_status;
  k_keys<<<gb, kBlock, 0, c->stream>>>(c->st, n, c->kp, c->keys, c->vals, st);
  unsigned *ka = c->keys, *kb = c->keys_alt;
  int *va = c->vals, *vb = c->vals_alt;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 8 * pass;
    k_radix_hist<<<c->ntiles, kSortThreads, 0, c->stream>>>(ka, (int)n, shift, c->hist, c->ntiles,
                                                            st);
    const int m = 256 * c->ntiles, nseg = (m + kScanSeg - 1) / kScanSeg;
    k_scan_totals<<<nseg, kScanSeg, 0, c->stream>>>(c->hist, m, c->scan_tot, shift, st);
    k_scan_of_totals<<<1, kScanSeg, 0, c->stream>>>(c->scan_tot, nseg, shift, st);
    k_scan_apply<<<nseg, kScanSeg, 0, c->stream>>>(c->hist, m, c->scan_tot, shift, st);
    k_radix_scatter<<<c->ntiles, kSortThreads, 0, c->stream>>>(ka, va, kb, vb, (int)n, shift,
                                                               c->hist, c->ntiles, st);
    unsigned *tk = ka;
    ka = kb;
    kb = tk;
    int *tv = va;
    va = vb;
    vb = tv;
  }
  // the sorted pairs are in keys / vals after an even number of passes that
  // ran, in keys_alt / vals_alt after an odd one (the kernels that read
  // them choose on the device)
  c->src = c->st;
  enqueue_permute(c, perm_table(c->st, c->w, c->learn, all != 0, c->kp.max_rung > 0, part,
                                c->lazy != 0 && all == 0),
                  0);
  k_clear_cells<<<grid_for(c->max_cells, kBlock), kBlock, 0, c->stream>>>(c->cell_start,
                                                                          c->d_status);
  k_cells<<<gb, kBlock, 0, c->stream>>>(c->keys, c->keys_alt, n, c->kp, c->cell_start,
                                        c->cell_end, c->w.cc, c->max_cells, st);
  c->nlaunch += 1 + 4 * 5 + 2;   // keys, four radix passes, cells (permutation counted above)
  return cudaGetLastError();
}

}  // namespace sphk
