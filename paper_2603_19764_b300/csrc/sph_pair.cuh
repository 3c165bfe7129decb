// sph_pair.cuh -- warp-per-bucket machinery shared by the two pair kernels
// (density solve and force loop).
//
// A bucket is 32 consecutive cell-sorted particles, one per lane. Lanes whose
// cells lie within two cells of the first unfinished lane form a group; a
// group stages its candidate neighbours, particles of the cells that overlap
// the group's bounding box grown by a search radius, into a per-warp
// shared-memory list after a bounding-box distance filter. The staging is
// resumable so that a list longer than the buffer is processed in segments.
#pragma once

#include <type_traits>

#include "sph_internal.cuh"

namespace sphk {

template <typename T> struct V4T;
template <> struct V4T<float> {
  using type = float4;
  static __device__ __forceinline__ float4 ld(const float4 *p, int64_t i) { return __ldg(p + i); }
  // two consecutive vectors p[0], p[1] in one 32-byte read-only load (p
  // 32-byte aligned)
  static __device__ __forceinline__ void ld2(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
  }
  static __device__ __forceinline__ float4 make(float x, float y, float z, float w) {
    return make_float4(x, y, z, w);
  }
};
template <> struct V4T<double> {
  using type = double4_32a;
  static __device__ __forceinline__ double4_32a ld(const double4_32a *p, int64_t i) { return p[i]; }
  static __device__ __forceinline__ void ld2(const double4_32a *p, double4_32a &a,
                                             double4_32a &b) {
    a = p[0];
    b = p[1];
  }
  static __device__ __forceinline__ double4_32a make(double x, double y, double z, double w) {
    return make_double4_32a(x, y, z, w);
  }
};

// Two FP32 values in one 64-bit register, and the sm_100-family arithmetic
// on such pairs: one instruction applies the same IEEE operation (round to
// nearest, no flush) to both halves, so a packed result equals the two
// scalar results bit for bit.
namespace px {
using u64 = unsigned long long;
__device__ __forceinline__ u64 dup(float a) {
  u64 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ void split(u64 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 sub(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
}  // namespace px

// Larger / smaller of two values: one min / max instruction (a compare and
// a select otherwise). The operands are finite wherever these are used; for
// a NaN operand the other one is returned.
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }

// Products and sums that the compiler may not fuse into one rounding.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
// A coordinate relative to the group's reference cell: c (relative to the
// particle's own cell) plus k cells of side L, rounded once for the product
// and once for the sum. The lane's own particle and the same particle staged
// as a candidate are formed this way from the same inputs, so their bits
// agree whatever the compiler contracts elsewhere, and the pair of a particle
// with itself sits at r = 0 exactly (the counts exclude it there).
template <typename T> __device__ __forceinline__ T rel_coord(T c, int k, T L) {
  return add_rn(c, mul_rn((T)k, L));
}
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

// Canonical FP64 squared distance (no contraction): the neighbour predicate
// r < H of every count compares this against H * H.
__device__ __forceinline__ double r2_canon(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Half-width of the band around H^2 inside which an FP32 r^2 cannot decide
// r < H. Coordinates relative to a reference cell of side L lie within six
// cells of it (a group spans at most three cells, its candidates one search
// radius more), so each is rounded by at most 7 L 2^-24 and a difference by
// twice that; for r close to H the squared distance then errs by at most
// 2 sqrt(3) H 8.4e-7 L plus the roundings of the squares, the sums and H^2
// (under 3e-7 H^2): below 3.2e-6 H max(H, L). The band is three times that;
// pairs inside it are decided with the FP64 predicate, and every mask or
// list test that must not lose a pair with r < H widens its radius^2 by it.
template <typename T>
__device__ __forceinline__ T guard_band(T H, T L) {
  return T(1e-5) * H * tmax(H, L);
}

// Squared distance in the fixed order ((dx dx) + dy dy) + dz dz, with the
// two fused multiply-adds written out, so that a packed mask test and a
// scalar walk round identically.
__device__ __forceinline__ float dist2(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
__device__ __forceinline__ double dist2(double dx, double dy, double dz) {
  return __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
}

// Staged candidates: x, y, z relative to the group's reference cell and one
// more value w, one 4-vector per candidate (the FP64 form's layout).
template <typename V4> struct CandAoS {
  template <typename T>
  static __device__ __forceinline__ void get(const V4 *L, int k, T &x, T &y, T &z, T &w) {
    const V4 q = L[k];
    x = q.x;
    y = q.y;
    z = q.z;
    w = q.w;
  }
};

// List views with the staging and walking interface of the density kernel
// (put / get of candidate k), over a buffer of S candidates:
// * ViewAoS: one 4-vector per candidate (the FP64 form).
// * ViewPlanes (FP32): x, y, z and w of candidate k in four planes of S
//   floats, so that a lane reading one candidate hits bank k mod 32 of
//   each plane (32 banks across the lanes of a walk, where the paired
//   layout reached 8), staging writes are consecutive, and the packed mask
//   test reads the x (y, z) of four candidates with one 16-byte load.
template <typename V4> struct ViewAoS {
  V4 *p;
  template <typename T>
  __device__ __forceinline__ void put(int k, T x, T y, T z, T w) const {
    p[k] = V4T<T>::make(x, y, z, w);
  }
  template <typename T>
  __device__ __forceinline__ void get(int k, T &x, T &y, T &z, T &w) const {
    const V4 q = p[k];
    x = q.x;
    y = q.y;
    z = q.z;
    w = q.w;
  }
};
template <int S> struct ViewPlanes {
  float *p;
  __device__ __forceinline__ void put(int k, float x, float y, float z, float w) const {
    p[k] = x;
    p[S + k] = y;
    p[2 * S + k] = z;
    p[3 * S + k] = w;
  }
  __device__ __forceinline__ void get(int k, float &x, float &y, float &z, float &w) const {
    x = p[k];
    y = p[S + k];
    z = p[2 * S + k];
    w = p[3 * S + k];
  }
};

// Membership words. A word covers staged candidates kb .. kb+31 (kb a
// multiple of 32) and holds candidate kb + b at bit 31 - b, so that the
// walk finds the next marked candidate in list order with one count of
// leading zeros. The test r^2 < thr of two non-negative values is decided
// on their bit patterns (which order like the values): the sign of the
// integer difference, shifted into the word.
__device__ __forceinline__ unsigned below(float a, float t) {
  return (unsigned)(__float_as_int(a) - __float_as_int(t));
}
__device__ __forceinline__ unsigned below(double a, double t) {
  return (unsigned)((unsigned long long)(__double_as_longlong(a) - __double_as_longlong(t)) >> 32);
}
// word = word << 1 | sign bit of d
__device__ __forceinline__ unsigned push_bit(unsigned word, unsigned d) {
  return __funnelshift_l(d, word, 1);
}
// The next marked candidate of a nonzero word (its offset b in the word),
// cleared from the word. For a zero word b is 0 and the word stays zero.
__device__ __forceinline__ int take_next(unsigned &mk) {
  const int b = __clz(mk) & 31;
  mk &= ~(0x80000000u >> b);
  return b;
}
// Keep the bits of the first `count` candidates of a word (1 <= count <= 32).
__device__ __forceinline__ unsigned first_bits(unsigned mk, int count) {
  return count < 32 ? mk & (0xffffffffu << (32 - count)) : mk;
}

// One lane's membership word: bit 31 - b set when r^2 < thr(w) for candidate
// kb + b, for b < count only.
template <typename V4, typename T, typename Thr>
__device__ __forceinline__ unsigned mask_word(const V4 *L, int kb, int count, T xi, T yi, T zi,
                                              Thr thr) {
  unsigned mk = 0;
  for (int b = 0; b < 32; ++b) {
    T x = T(0), y = T(0), z = T(0), w = T(0);
    if (b < count) CandAoS<V4>::get(L, kb + b, x, y, z, w);
    const T dx = xi - x, dy = yi - y, dz = zi - z;
    mk = push_bit(mk, below(dist2(dx, dy, dz), thr(w)));
  }
  return first_bits(mk, count);
}

template <typename V4, typename T, typename Thr>
__device__ __forceinline__ unsigned mask_word(const ViewAoS<V4> &L, int kb, int count, T xi, T yi,
                                              T zi, Thr thr) {
  return mask_word(static_cast<const V4 *>(L.p), kb, count, xi, yi, zi, thr);
}
// Planes: reads whole 32-candidate words (S a multiple of 32), clearing the
// bits past the list's end; two candidates per packed operation.
template <int S, typename Thr>
__device__ __forceinline__ unsigned mask_word(const ViewPlanes<S> &L, int kb, int count,
                                              float xi, float yi, float zi, Thr thr) {
  using namespace px;
  const u64 X = dup(xi), Y = dup(yi), Z = dup(zi);
  const ulonglong2 *PX = reinterpret_cast<const ulonglong2 *>(L.p + kb);
  const ulonglong2 *PY = reinterpret_cast<const ulonglong2 *>(L.p + S + kb);
  const ulonglong2 *PZ = reinterpret_cast<const ulonglong2 *>(L.p + 2 * S + kb);
  const ulonglong2 *PW = reinterpret_cast<const ulonglong2 *>(L.p + 3 * S + kb);
  unsigned mk = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const ulonglong2 a = PX[q], b = PY[q], c = PZ[q], w = PW[q];   // candidates 4q .. 4q+3
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const u64 dx = sub(X, h ? a.y : a.x), dy = sub(Y, h ? b.y : b.x), dz = sub(Z, h ? c.y : c.x);
      const u64 r2 = fma(dz, dz, fma(dy, dy, mul(dx, dx)));
      float r0, r1, w0, w1;
      split(r2, r0, r1);
      split(h ? w.y : w.x, w0, w1);
      mk = push_bit(mk, below(r0, thr(w0)));
      mk = push_bit(mk, below(r1, thr(w1)));
    }
  }
  return first_bits(mk, count);
}

// Squared distance of a point to an axis-aligned box (0 inside).
template <typename T>
__device__ __forceinline__ T box_d2(T x, T y, T z, T x0, T x1, T y0, T y1, T z0, T z1) {
  const T ex = tmax(x0 - x, tmax(T(0), x - x1));
  const T ey = tmax(y0 - y, tmax(T(0), y - y1));
  const T ez = tmax(z0 - z, tmax(T(0), z - z1));
  return ex * ex + ey * ey + ez * ez;
}

// Group of lanes around the first lane still in `todo`: the lanes whose
// cells lie within `span` cells of that lane's cell on every axis. A wider
// span stages fewer, longer candidate lists per bucket. Each lane's
// neighbours are visited in the same order whatever the span (cells in
// z, y, x order, particles in sorted order), so the span changes only the
// FP32 form's cell-relative frame, never the FP64 form's bits.
struct Group {
  int rx, ry, rz;   // reference cell
  bool member;
};
__device__ __forceinline__ Group next_group(unsigned &todo, int cx, int cy, int cz, int span) {
  const int lane = threadIdx.x & 31;
  Group g;
  const int ref = __ffs(todo) - 1;
  g.rx = __shfl_sync(kFull, cx, ref);
  g.ry = __shfl_sync(kFull, cy, ref);
  g.rz = __shfl_sync(kFull, cz, ref);
  g.member = ((todo >> lane) & 1u) && abs(cx - g.rx) <= span && abs(cy - g.ry) <= span &&
             abs(cz - g.rz) <= span;
  todo &= ~__ballot_sync(kFull, g.member);
  return g;
}

// Bounding box of the active lanes (warp-uniform result).
template <typename T> struct Box {
  T x0, x1, y0, y1, z0, z1;
};
template <typename T>
__device__ __forceinline__ Box<T> group_box(bool act, T x, T y, T z) {
  Box<T> b;
  b.x0 = wmin(act ? x : T(1e30));
  b.x1 = wmax(act ? x : T(-1e30));
  b.y0 = wmin(act ? y : T(1e30));
  b.y1 = wmax(act ? y : T(-1e30));
  b.z0 = wmin(act ? z : T(1e30));
  b.z1 = wmax(act ? z : T(-1e30));
  return b;
}

// Resumable stream of the particles of the cells overlapping box +- R, in
// cell order (z, then y, then x) and sorted order within a cell. The cell
// ranges are read 32 cells at a time, one cell per lane, so their loads
// overlap instead of forming a chain, and one batch ahead: the ranges of
// the next 32 cells are requested when a batch is taken up, so that taking
// up the next one waits for no load; a prefix sum over the lanes then maps
// stream positions to (cell, particle), and every chunk of 32 positions
// fills all lanes whatever the cell sizes. Coordinates are relative to the
// origin of the reference cell (FP32 form) or absolute (FP64 form): a
// particle's offset is (its cell - reference cell) * L, formed from exact
// integer-valued floats.
struct Stager {
  int kx0, ky0, kz0;       // first cell of the range
  int nx, ny, ncell;       // range extents in x and y, cells in the range
  int c0;                  // first cell of the next batch
  int s0, pre, off;        // this lane's cell of the batch: start, exclusive
                           // prefix of the counts, packed offset to the
                           // reference cell (10 bits per axis, biased 512)
  int total, pos;          // particles in the batch, next stream position
  int nst, nen, noff;      // the next batch's cell of this lane: start, end,
                           // packed offset (nst < 0: empty or past the range)
};

// All staged: no cell left and the batch consumed.
__device__ __forceinline__ bool stager_finished(const Stager &s) {
  return s.c0 >= s.ncell && s.pos >= s.total;
}

// Set up a stager for box +- R. REL: box in coordinates relative to cell
// (rx, ry, rz).
template <typename T, bool REL>
__device__ __forceinline__ Stager make_stager(const Box<T> &b, T R, const Grid &g, T invL,
                                              int rx, int ry, int rz) {
  int kx0, kx1, ky0, ky1, kz0, kz1;
  if (REL) {
    kx0 = rx + (int)floorf((float)((b.x0 - R) * invL));
    kx1 = rx + (int)floorf((float)((b.x1 + R) * invL));
    ky0 = ry + (int)floorf((float)((b.y0 - R) * invL));
    ky1 = ry + (int)floorf((float)((b.y1 + R) * invL));
    kz0 = rz + (int)floorf((float)((b.z0 - R) * invL));
    kz1 = rz + (int)floorf((float)((b.z1 + R) * invL));
  } else {
    kx0 = (int)floor(((double)b.x0 - (double)R - g.lo[0]) * (double)invL);
    kx1 = (int)floor(((double)b.x1 + (double)R - g.lo[0]) * (double)invL);
    ky0 = (int)floor(((double)b.y0 - (double)R - g.lo[1]) * (double)invL);
    ky1 = (int)floor(((double)b.y1 + (double)R - g.lo[1]) * (double)invL);
    kz0 = (int)floor(((double)b.z0 - (double)R - g.lo[2]) * (double)invL);
    kz1 = (int)floor(((double)b.z1 + (double)R - g.lo[2]) * (double)invL);
  }
  Stager s;
  s.kx0 = max(kx0, 0);
  s.ky0 = max(ky0, 0);
  s.kz0 = max(kz0, 0);
  s.nx = min(kx1, g.dims[0] - 1) - s.kx0 + 1;
  s.ny = min(ky1, g.dims[1] - 1) - s.ky0 + 1;
  const int nz = min(kz1, g.dims[2] - 1) - s.kz0 + 1;
  s.ncell = (s.nx > 0 && s.ny > 0 && nz > 0) ? s.nx * s.ny * nz : 0;
  s.c0 = 0;
  s.s0 = 0;
  s.pre = 0;
  s.off = 0;
  s.total = 0;
  s.pos = 0;
  s.nst = -1;
  s.nen = 0;
  s.noff = 0;
  (void)rx;
  (void)ry;
  (void)rz;
  return s;
}

// Request the cell range of this lane's cell in the batch from range cell
// c0 on (start, end and packed offset; start -1 past the range). Both loads
// are issued together; an empty cell's end is read but not used.
__device__ __forceinline__ void stager_fetch(const Stager &s, int c0, const Grid &g,
                                             const int *cstart, const int *cend, int rx, int ry,
                                             int rz, unsigned *err, int &st, int &en, int &off) {
  const int c = c0 + (int)(threadIdx.x & 31);
  st = -1;
  en = 0;
  off = 0;
  if (c < s.ncell) {
    const int x = c % s.nx, t = c / s.nx;
    const int y = t % s.ny, z = t / s.ny;
    const int gx = s.kx0 + x, gy = s.ky0 + y, gz = s.kz0 + z;
    const int cell = g.cell_off + (int)checked((gz * g.dims[1] + gy) * g.dims[0] + gx,
                                               g.ncells, err);
    st = cstart[cell];
    en = cend[cell];
    off = (gx - rx + 512) | ((gy - ry + 512) << 10) | ((gz - rz + 512) << 20);
  }
}

// Make the current batch of cells hold unconsumed stream positions,
// reading the next 32 cells of the range (one per lane) as often as needed.
// false when the stream is exhausted (warp-uniform). AHEAD: the ranges of
// the batch after are requested as a batch is taken up (three registers a
// lane held while the list is walked; the force pass, at its register
// limit, fetches each batch when it takes it up instead).
template <bool AHEAD>
__device__ __forceinline__ bool stager_refill(Stager &s, const Grid &g, const int *cstart,
                                              const int *cend, int rx, int ry, int rz,
                                              unsigned *err) {
  const int lane = threadIdx.x & 31;
  while (s.pos >= s.total) {
    if (s.c0 >= s.ncell) return false;
    int st, en, off;
    if (AHEAD) {
      // the first batch is fetched here, every later one a batch ahead
      if (s.c0 == 0)
        stager_fetch(s, 0, g, cstart, cend, rx, ry, rz, err, s.nst, s.nen, s.noff);
      st = s.nst;
      en = s.nen;
      off = s.noff;
      stager_fetch(s, s.c0 + 32, g, cstart, cend, rx, ry, rz, err, s.nst, s.nen, s.noff);
    } else {
      stager_fetch(s, s.c0, g, cstart, cend, rx, ry, rz, err, st, en, off);
    }
    const int cnt = st >= 0 ? en - st : 0;
    int inc = cnt;   // inclusive prefix over the lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += v;
    }
    s.s0 = st;
    s.pre = inc - cnt;
    s.off = off;
    s.total = __shfl_sync(kFull, inc, 31);
    s.pos = 0;
    s.c0 += 32;
  }
  return true;
}

// Stream position k of the current batch (every lane calls it, each with
// its own k): particle index j (valid when ok) and its coordinate offset.
template <typename T, bool REL>
__device__ __forceinline__ void stager_at(const Stager &s, int k, T Lt, int &j, bool &ok, T &ox,
                                          T &oy, T &oz) {
  ok = k < s.total;
  // the lane whose cell holds stream position k: the last one with pre <= k
  int own = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = own + step;
    const int pc = __shfl_sync(kFull, s.pre, cand & 31);
    if (cand < 32 && pc <= k) own = cand;
  }
  const int p0 = __shfl_sync(kFull, s.pre, own);
  j = __shfl_sync(kFull, s.s0, own) + (k - p0);
  const int off = __shfl_sync(kFull, s.off, own);
  if (REL) {
    // the candidate's coordinate is add_rn(c, o), as rel_coord forms it
    ox = mul_rn((T)((off & 1023) - 512), Lt);
    oy = mul_rn((T)(((off >> 10) & 1023) - 512), Lt);
    oz = mul_rn((T)(((off >> 20) & 1023) - 512), Lt);
  } else {
    ox = oy = oz = T(0);
  }
}

// ------------------------------------------------------------ periodic box
// In a periodic box the range box +- R may cross the box's faces. The part
// past a face holds the images of the particles at the opposite side, one
// box length away, so per axis the range is up to three runs of cells:
// [lo0, dims) shifted by -len (the part below box_lo), [m0, m0 + nm)
// unshifted, and [0, nu) shifted by +len (the part at or past box_hi).
// Each run stages its cells' particles with that shift added to their
// coordinates. While the box is wider than twice every search radius
// (checked by the kernels), a lane finds at most one image of any particle
// within its radius, and it is the minimum image; the particle itself
// appears unshifted only.
template <typename T> struct StagerP {
  int lo0[3], nlo[3], m0[3], nm[3], nu[3];   // the three runs per axis
  int nx, ny, ncell;                         // run-concatenated extents
  int c0;                                    // first cell of the next batch
  int s0, pre;                               // this lane's cell: start, prefix
  T ox, oy, oz;                              // this lane's cell: offset to the frame
  int total, pos;
};

template <typename T> __device__ __forceinline__ bool stager_finished(const StagerP<T> &s) {
  return s.c0 >= s.ncell && s.pos >= s.total;
}

// Runs of axis a for the range [b0 - R, b1 + R] (in the frame: relative to
// the reference cell's origin for REL, absolute otherwise). Cell indices
// come from the same floor((x - lo) / L) as the particles' own cells, in
// FP64.
template <typename T, bool REL>
__device__ __forceinline__ void periodic_runs(StagerP<T> &s, int a, T b0, T b1, T R,
                                              const Grid &g, const KParams &P, int r) {
  const double o = REL ? g.lo[a] + (double)r * g.L : 0.0;
  const double A = o + (double)(b0 - R), B = o + (double)(b1 + R);
  const int dims = g.dims[a];
  const double len = P.box_len[a];
  const int k0 = (int)floor((A - g.lo[a]) * g.invL), k1 = (int)floor((B - g.lo[a]) * g.invL);
  s.m0[a] = max(k0, 0);
  s.nm[a] = max(0, min(k1, dims - 1) - s.m0[a] + 1);
  s.lo0[a] = 0;
  s.nlo[a] = 0;
  s.nu[a] = 0;
  if (A < P.box_lo[a]) {
    const int kl = min(max((int)floor((A + len - g.lo[a]) * g.invL), 0), dims - 1);
    s.lo0[a] = kl;
    s.nlo[a] = dims - kl;
  }
  if (B >= P.box_hi[a]) {
    const int ku = min(max((int)floor((B - len - g.lo[a]) * g.invL), 0), dims - 1);
    s.nu[a] = ku + 1;
  }
}

template <typename T, bool REL>
__device__ __forceinline__ StagerP<T> make_stager_periodic(const Box<T> &b, T R, const Grid &g,
                                                           const KParams &P, int rx, int ry,
                                                           int rz) {
  StagerP<T> s;
  periodic_runs<T, REL>(s, 0, b.x0, b.x1, R, g, P, rx);
  periodic_runs<T, REL>(s, 1, b.y0, b.y1, R, g, P, ry);
  periodic_runs<T, REL>(s, 2, b.z0, b.z1, R, g, P, rz);
  const long long n0 = s.nlo[0] + s.nm[0] + s.nu[0], n1 = s.nlo[1] + s.nm[1] + s.nu[1],
                  n2 = s.nlo[2] + s.nm[2] + s.nu[2];
  const long long nc = n0 * n1 * n2;
  s.nx = (int)n0;
  s.ny = (int)n1;
  s.ncell = nc > 0x7fffffffLL ? 0x7fffffff : (int)nc;
  s.c0 = 0;
  s.s0 = 0;
  s.pre = 0;
  s.ox = s.oy = s.oz = T(0);
  s.total = 0;
  s.pos = 0;
  return s;
}

// Position v of axis a's runs: the cell and its shift in box lengths.
template <typename T>
__device__ __forceinline__ int periodic_cell(const StagerP<T> &s, int a, int v, int &shift) {
  if (v < s.nlo[a]) {
    shift = -1;
    return s.lo0[a] + v;
  }
  v -= s.nlo[a];
  if (v < s.nm[a]) {
    shift = 0;
    return s.m0[a] + v;
  }
  shift = 1;
  return v - s.nm[a];
}

// The candidate's coordinate offset for cell k of axis a at `shift` box
// lengths. REL: the unshifted offset is mul_rn(k - r, L) as for a closed
// box (and as rel_coord forms the lane's own coordinate); a shifted one is
// formed in FP64 and rounded once, so that its error is that of a small
// offset, not of a box length. Absolute frame: the shift alone.
template <typename T, bool REL>
__device__ __forceinline__ T periodic_offset(int k, int r, int shift, T Lt, const Grid &g,
                                             double len) {
  if (REL) {
    if (shift == 0) return mul_rn((T)(k - r), Lt);
    return (T)((double)(k - r) * g.L + (double)shift * len);
  }
  return shift == 0 ? T(0) : (T)((double)shift * len);
}

// As stager_refill and stager_at for a closed box, over the periodic runs
// (each batch fetched when it is taken up, whatever AHEAD).
template <typename T, bool REL, bool AHEAD>
__device__ __forceinline__ bool stager_refill(StagerP<T> &s, const Grid &g, const int *cstart,
                                              const int *cend, T Lt, const KParams &P, int rx,
                                              int ry, int rz, unsigned *err) {
  const int lane = threadIdx.x & 31;
  while (s.pos >= s.total) {
    if (s.c0 >= s.ncell) return false;
    const int c = s.c0 + lane;
    int cnt = 0, st = 0;
    T cx = T(0), cy = T(0), cz = T(0);
    if (c < s.ncell) {
      const int vx = c % s.nx, t = c / s.nx;
      const int vy = t % s.ny, vz = t / s.ny;
      int shx, shy, shz;
      const int gx = periodic_cell(s, 0, vx, shx);
      const int gy = periodic_cell(s, 1, vy, shy);
      const int gz = periodic_cell(s, 2, vz, shz);
      const int cell = g.cell_off + (int)checked((gz * g.dims[1] + gy) * g.dims[0] + gx,
                                                 g.ncells, err);
      st = cstart[cell];
      if (st >= 0) cnt = cend[cell] - st;
      cx = periodic_offset<T, REL>(gx, rx, shx, Lt, g, P.box_len[0]);
      cy = periodic_offset<T, REL>(gy, ry, shy, Lt, g, P.box_len[1]);
      cz = periodic_offset<T, REL>(gz, rz, shz, Lt, g, P.box_len[2]);
    }
    int inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += v;
    }
    s.s0 = st;
    s.pre = inc - cnt;
    s.ox = cx;
    s.oy = cy;
    s.oz = cz;
    s.total = __shfl_sync(kFull, inc, 31);
    s.pos = 0;
    s.c0 += 32;
  }
  return true;
}
template <typename T, bool REL>
__device__ __forceinline__ void stager_at(const StagerP<T> &s, int k, T, int &j, bool &ok, T &ox,
                                          T &oy, T &oz) {
  ok = k < s.total;
  int own = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int cand = own + step;
    const int pc = __shfl_sync(kFull, s.pre, cand & 31);
    if (cand < 32 && pc <= k) own = cand;
  }
  const int p0 = __shfl_sync(kFull, s.pre, own);
  j = __shfl_sync(kFull, s.s0, own) + (k - p0);
  ox = __shfl_sync(kFull, s.ox, own);
  oy = __shfl_sync(kFull, s.oy, own);
  oz = __shfl_sync(kFull, s.oz, own);
}

// One stager type per box kind, so that the closed-box kernels are
// unchanged.
template <typename T, bool PER> struct StagerOf {
  using type = Stager;
};
template <typename T> struct StagerOf<T, true> {
  using type = StagerP<T>;
};
template <typename T, bool REL, bool PER>
__device__ __forceinline__ typename StagerOf<T, PER>::type make_stager_for(
    const Box<T> &b, T R, const Grid &g, T invL, const KParams &P, int rx, int ry, int rz) {
  if constexpr (PER)
    return make_stager_periodic<T, REL>(b, R, g, P, rx, ry, rz);
  else
    return make_stager<T, REL>(b, R, g, invL, rx, ry, rz);
}
template <typename T, bool REL, bool AHEAD>
__device__ __forceinline__ bool stager_refill(Stager &s, const Grid &g, const int *cstart,
                                              const int *cend, T, const KParams &, int rx, int ry,
                                              int rz, unsigned *err) {
  return stager_refill<AHEAD>(s, g, cstart, cend, rx, ry, rz, err);
}

// Stage the stream into a list from position nl on, while a further 32
// entries fit below cap: each candidate's record is loaded (load(ok, j)),
// tested (keep(ok, q, ox, oy, oz, x, y, z) forms its coordinates and
// decides), and the kept ones are appended in stream order (put(at, x, y,
// z, q, j)). U chunks of 32 stream positions are located and their records
// loaded before the first of them is tested, so that U loads are in flight
// at once; chunks are consumed in order and the stager stops at the first
// one that finds no room (its loads are dropped), so the list is the one a
// chunk-by-chunk loop would build. Returns the new list length.
template <int U, bool AHEAD, typename T, bool REL, typename St, typename Ld, typename Kp,
          typename Pt>
__device__ __forceinline__ int stage_list(St &sg, const Grid &g, const int *cstart,
                                          const int *cend, T Lt, const KParams &P, int rx, int ry,
                                          int rz, int nl, int cap, int64_t n, unsigned *err,
                                          Ld load, Kp keep, Pt put) {
  const int lane = threadIdx.x & 31;
  while (nl <= cap - 32) {
    if (!stager_refill<T, REL, AHEAD>(sg, g, cstart, cend, Lt, P, rx, ry, rz, err)) break;
    const int avail = (sg.total - sg.pos + 31) >> 5;   // chunks left in this batch
    int j[U];
    bool ok[U];
    T ox[U], oy[U], oz[U];
    decltype(load(false, 0)) q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      j[u] = 0;
      ok[u] = false;
      ox[u] = oy[u] = oz[u] = T(0);
      if (u < avail) stager_at<T, REL>(sg, sg.pos + 32 * u + lane, Lt, j[u], ok[u], ox[u], oy[u],
                                       oz[u]);
      if (ok[u]) j[u] = (int)checked(j[u], n, err);
      q[u] = load(ok[u], j[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u >= avail || nl > cap - 32) break;   // warp-uniform
      T x, y, z;
      const bool kp = keep(ok[u], q[u], ox[u], oy[u], oz[u], x, y, z);
      const unsigned bal = __ballot_sync(kFull, kp);
      if (kp) put((int)checked(nl + __popc(bal & lanemask_lt()), cap, err), x, y, z, q[u], j[u]);
      nl += __popc(bal);
      sg.pos += 32;
    }
  }
  return nl;
}

// FP64 squared distance of the neighbour predicate in a periodic box: the
// minimum image along every axis, then the canonical sum.
__device__ __forceinline__ double r2_canon_periodic(double dx, double dy, double dz,
                                                    const double *len) {
  return r2_canon(min_image(dx, len[0]), min_image(dy, len[1]), min_image(dz, len[2]));
}

// The FP64 predicate r < H of a pair inside the FP32 form's guard band
// (particle i at (xi, yi, zi), candidate j; H the FP32 radius, whose square
// is exact in FP64). Out of line for the density walk, whose accumulation
// has no branch: written inline there, the compiler evaluated it for every
// pair, outside the band too. (The force walk keeps it inline: the call
// made that kernel spill.)
template <bool PER>
static __device__ __noinline__ bool fp64_within(const double *sx, const double *sy,
                                                const double *sz, double xi, double yi,
                                                double zi, int j, const double *blen, double H) {
  const double c2 = PER ? r2_canon_periodic(xi - sx[j], yi - sy[j], zi - sz[j], blen)
                        : r2_canon(xi - sx[j], yi - sy[j], zi - sz[j]);
  return c2 < __dmul_rn(H, H);
}

}  // namespace sphk
