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
  static __device__ __forceinline__ float4 make(float x, float y, float z, float w) {
    return make_float4(x, y, z, w);
  }
};
template <> struct V4T<double> {
  using type = double4_32a;
  static __device__ __forceinline__ double4_32a ld(const double4_32a *p, int64_t i) { return p[i]; }
  static __device__ __forceinline__ double4_32a make(double x, double y, double z, double w) {
    return make_double4_32a(x, y, z, w);
  }
};

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// Square root of x >= 0 and a quotient: correctly rounded in FP64; in FP32
// through the hardware reciprocal square root and the fast divide (a few
// ulp), which the FP32 form's tolerances absorb.
template <typename T> __device__ __forceinline__ T root(T x);
template <> __device__ __forceinline__ float root<float>(float x) {
  return x > 0.f ? x * rsqrtf(x) : 0.f;
}
template <> __device__ __forceinline__ double root<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T quot(T a, T b);
template <> __device__ __forceinline__ float quot<float>(float a, float b) {
  return __fdividef(a, b);
}
template <> __device__ __forceinline__ double quot<double>(double a, double b) { return a / b; }

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

// Resumable walk over the particles of the cells overlapping box +- R.
// Coordinates are relative to the origin of the reference cell (FP32 form)
// or absolute (FP64 form); (ox, oy, oz) converts the staged cell's packed
// positions into that frame. The cell counters advance without integer
// division, and the FP32 offsets are kept as exact integer-valued floats.
template <typename T> struct Stager {
  int kx0, kx1, ky0, ky1, kz0, kz1;  // cell range
  int x, y, z;                       // next cell
  T fx0, fy0, fx, fy, fz;            // (cell - reference) as exact floats
  int jb, je;                        // current chunk start, cell end
  T ox, oy, oz;                      // coordinate offset of the current cell
  bool done;                         // no further cell to fetch
};

// All staged: no further cell and the current one consumed.
template <typename T> __device__ __forceinline__ bool stager_finished(const Stager<T> &s) {
  return s.done && s.jb >= s.je;
}

// Set up a stager for box +- R. REL: coordinates relative to cell (rx, ry, rz).
template <typename T, bool REL>
__device__ __forceinline__ Stager<T> make_stager(const Box<T> &b, T R, const Grid &g, T invL,
                                                 int rx, int ry, int rz) {
  Stager<T> s;
  if (REL) {
    s.kx0 = rx + (int)floorf((float)((b.x0 - R) * invL));
    s.kx1 = rx + (int)floorf((float)((b.x1 + R) * invL));
    s.ky0 = ry + (int)floorf((float)((b.y0 - R) * invL));
    s.ky1 = ry + (int)floorf((float)((b.y1 + R) * invL));
    s.kz0 = rz + (int)floorf((float)((b.z0 - R) * invL));
    s.kz1 = rz + (int)floorf((float)((b.z1 + R) * invL));
  } else {
    s.kx0 = (int)floor(((double)b.x0 - (double)R - g.lo[0]) * (double)invL);
    s.kx1 = (int)floor(((double)b.x1 + (double)R - g.lo[0]) * (double)invL);
    s.ky0 = (int)floor(((double)b.y0 - (double)R - g.lo[1]) * (double)invL);
    s.ky1 = (int)floor(((double)b.y1 + (double)R - g.lo[1]) * (double)invL);
    s.kz0 = (int)floor(((double)b.z0 - (double)R - g.lo[2]) * (double)invL);
    s.kz1 = (int)floor(((double)b.z1 + (double)R - g.lo[2]) * (double)invL);
  }
  s.kx0 = max(s.kx0, 0);
  s.ky0 = max(s.ky0, 0);
  s.kz0 = max(s.kz0, 0);
  s.kx1 = min(s.kx1, g.dims[0] - 1);
  s.ky1 = min(s.ky1, g.dims[1] - 1);
  s.kz1 = min(s.kz1, g.dims[2] - 1);
  s.x = s.kx0;
  s.y = s.ky0;
  s.z = s.kz0;
  s.fx0 = (T)(s.kx0 - rx);
  s.fx = s.fx0;
  s.fy0 = (T)(s.ky0 - ry);
  s.fy = s.fy0;
  s.fz = (T)(s.kz0 - rz);
  s.jb = 0;
  s.je = 0;
  s.ox = s.oy = s.oz = T(0);
  s.done = s.kx0 > s.kx1 || s.ky0 > s.ky1 || s.kz0 > s.kz1;
  return s;
}

// Advance to the next non-empty cell; false when the range is exhausted.
template <typename T, bool REL>
__device__ __forceinline__ bool stager_next_cell(Stager<T> &s, const Grid &g, const int *cstart,
                                                 const int *cend, T Lt) {
  while (!s.done) {
    const int c = g.cell_off + (s.z * g.dims[1] + s.y) * g.dims[0] + s.x;
    const T fx = s.fx, fy = s.fy, fz = s.fz;
    // step to the following cell of the range
    if (s.x < s.kx1) {
      ++s.x;
      s.fx += T(1);
    } else {
      s.x = s.kx0;
      s.fx = s.fx0;
      if (s.y < s.ky1) {
        ++s.y;
        s.fy += T(1);
      } else {
        s.y = s.ky0;
        s.fy = s.fy0;
        if (s.z < s.kz1) {
          ++s.z;
          s.fz += T(1);
        } else {
          s.done = true;
        }
      }
    }
    const int s0 = cstart[c];
    if (s0 < 0) continue;
    s.jb = s0;
    s.je = cend[c];
    s.ox = REL ? fx * Lt : T(0);
    s.oy = REL ? fy * Lt : T(0);
    s.oz = REL ? fz * Lt : T(0);
    return true;
  }
  return false;
}

}  // namespace sphk
