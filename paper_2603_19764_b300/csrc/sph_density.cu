// sph_density.cu -- prediction, position packing, and the density /
// smoothing-length solve (§2.1, Eq. 1-3).
//
// One warp owns a bucket of 32 consecutive (cell-sorted) particles, one
// particle per lane. Lanes whose cells lie within two cells of the first
// unfinished lane form a group; the group's candidate neighbours (particles
// of the cells within ceil(R / L_c) of the group's cells, R the largest H in
// the group) are staged through a per-warp shared-memory list after a
// bounding-box filter, and every lane evaluates the list against its own
// particle. Each particle's Newton iteration on its own H runs inside the
// kernel: the density of particle i depends only on H_i, so no global sweep
// synchronisation is needed.
//
// FP64 form: absolute positions, canonical predicate r^2 = (dx dx + dy dy) +
// dz dz without fused multiply-add. FP32 form: positions relative to the
// group's reference cell; pairs with |r^2 - H^2| < 1e-5 H^2 are re-decided
// with the FP64 predicate so that neighbour counts stay exact.
#include <type_traits>

#include "sph_internal.cuh"

namespace sphk {

// Evaluation state and position packing. predict = 1: v, u, S at i from
// the half-step values and the derivatives at i-1 (Eq. 40); predict = 0:
// the state as it stands.
__global__ void __launch_bounds__(kBlock) k_predict_pack(sph_state s, Work w, int64_t n,
                                                        const double *dtp, int predict,
                                                        const Status *st, int fp32) {
  const Grid g = st->grid;
  const double hdt = predict ? 0.5 * (*dtp) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed = s.flags[i] & SPH_FLAG_FIXED;
    const double k = fixed ? 0.0 : hdt;
    w.vp[0][i] = s.vx[i] + k * s.ax[i];
    w.vp[1][i] = s.vy[i] + k * s.ay[i];
    w.vp[2][i] = s.vz[i] + k * s.az[i];
    w.up[i] = s.u[i] + k * s.dudt[i];
    w.sp[0][i] = s.sxx[i] + k * s.dsxx[i];
    w.sp[1][i] = s.syy[i] + k * s.dsyy[i];
    w.sp[2][i] = s.sxy[i] + k * s.dsxy[i];
    w.sp[3][i] = s.sxz[i] + k * s.dsxz[i];
    w.sp[4][i] = s.syz[i] + k * s.dsyz[i];
    const double x = s.x[i], y = s.y[i], z = s.z[i], m = s.m[i];
    if (fp32) {
      const int c = w.cc[i];
      const double ox = g.lo[0] + (c & 1023) * g.L;
      const double oy = g.lo[1] + ((c >> 10) & 1023) * g.L;
      const double oz = g.lo[2] + ((c >> 20) & 1023) * g.L;
      w.pos32[i] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), (float)m);
    } else {
      w.pos64[i] = make_double4_32a(x, y, z, m);
    }
  }
}

cudaError_t launch_predict_pack(sph_ctx *c, int predict) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  k_predict_pack<<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->d_dt, predict,
                                                  c->d_status, c->kp.precision == SPH_FP32K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- density
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  using type = float4;
  static __device__ __forceinline__ float4 load(const Work &w, int64_t i) { return __ldg(w.pos32 + i); }
};
template <> struct Vec4<double> {
  using type = double4_32a;
  static __device__ __forceinline__ double4_32a load(const Work &w, int64_t i) { return w.pos64[i]; }
};

template <typename T, int CAP> struct DList {
  T x[CAP], y[CAP], z[CAP], m[CAP];
  int idx[CAP];
};

struct DensArgs {
  sph_state s;
  Work w;
  int64_t n;
  const int *cell_start, *cell_end;
  KParams p;
  Status *st;
};

// Canonical FP64 squared distance (no contraction).
__device__ __forceinline__ double r2_canon(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

template <typename T, int CAP>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_density(DensArgs A) {
  constexpr bool REL = std::is_same<T, float>::value;
  using V4 = typename Vec4<T>::type;
  __shared__ DList<T, CAP> lists[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  DList<T, CAP> &Ls = lists[wib];
  const int64_t base = ((int64_t)blockIdx.x * kWarpsPerBlock + wib) * 32;
  if (base >= A.n) return;
  const int64_t i = base + lane;
  const bool valid = i < A.n;
  const int64_t ic = valid ? i : base;

  const Grid g = A.st->grid;
  const T Lt = (T)g.L;
  const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
  const int cc = A.w.cc[ic];
  const int cx = cc & 1023, cy = (cc >> 10) & 1023, cz = (cc >> 20) & 1023;
  const V4 p = Vec4<T>::load(A.w, ic);
  const double mi = A.s.m[ic];
  const sph_material &M = A.p.mats[A.s.mat[ic] & (SPH_MAX_MATERIALS - 1)];
  const double target = A.p.n_ngb * mi;
  const double Hcap = A.p.h_cap_factor * lattice_radius(A.p.n_ngb, mi, M.rho0);
  double H = fmin(A.s.h[ic], Hcap);
  double xi64 = 0.0, yi64 = 0.0, zi64 = 0.0;
  if (REL) {
    xi64 = A.s.x[ic];
    yi64 = A.s.y[ic];
    zi64 = A.s.z[ic];
  }
  // Newton state: 0 running, 1 converged, 2 capped, 3 gave up, 4 idle lane
  int state = valid ? 0 : 4;
  double lo = 0.0, hi = INFINITY;
  double rho_o = 0.0, om_o = 1.0, H_o = H;
  int cnt_o = 0, sweeps_o = 0;
  long long pairs = 0;

  unsigned todo = __ballot_sync(kFull, valid);
  while (todo) {
    const int ref = __ffs(todo) - 1;
    const int rx = __shfl_sync(kFull, cx, ref), ry = __shfl_sync(kFull, cy, ref),
              rz = __shfl_sync(kFull, cz, ref);
    const bool member = ((todo >> lane) & 1u) && abs(cx - rx) <= 2 && abs(cy - ry) <= 2 &&
                        abs(cz - rz) <= 2;
    todo &= ~__ballot_sync(kFull, member);
    const T xi = REL ? p.x + (T)(cx - rx) * Lt : p.x;
    const T yi = REL ? p.y + (T)(cy - ry) * Lt : p.y;
    const T zi = REL ? p.z + (T)(cz - rz) * Lt : p.z;

    for (int sweep = 1; sweep <= A.p.max_sweeps; ++sweep) {
      const bool act = member && state == 0;
      if (!__any_sync(kFull, act)) break;
      const T Ht = (T)H;
      const double H2c = __dmul_rn(H, H);
      const T H2 = REL ? Ht * Ht : (T)H2c;
      const T invH = (T)(1.0 / H);
      const T R = wmax(act ? Ht : T(0));
      const T bx0 = wmin(act ? xi : T(1e30)), bx1 = wmax(act ? xi : T(-1e30));
      const T by0 = wmin(act ? yi : T(1e30)), by1 = wmax(act ? yi : T(-1e30));
      const T bz0 = wmin(act ? zi : T(1e30)), bz1 = wmax(act ? zi : T(-1e30));
      const int x0 = wmin(act ? cx : 1 << 20), x1 = wmax(act ? cx : -1);
      const int y0 = wmin(act ? cy : 1 << 20), y1 = wmax(act ? cy : -1);
      const int z0 = wmin(act ? cz : 1 << 20), z1 = wmax(act ? cz : -1);
      const int span = max(1, (int)ceil((double)R / g.L));
      T rs = 0, rhs = 0;
      int cnt = 0;
      int nl = 0;

      auto evaluate = [&](int nlist) {
        for (int k = 0; k < nlist; ++k) {
          const T dx = xi - Ls.x[k], dy = yi - Ls.y[k], dz = zi - Ls.z[k];
          T r2;
          bool in;
          if (REL) {
            r2 = dx * dx + dy * dy + dz * dz;
            in = r2 < H2;
            if (act && fabs(r2 - H2) < T(1e-5) * H2) {
              const int j = Ls.idx[k];
              in = r2_canon(xi64 - A.s.x[j], yi64 - A.s.y[j], zi64 - A.s.z[j]) < H2c;
            }
          } else {
            r2 = (T)r2_canon((double)dx, (double)dy, (double)dz);
            in = r2 < H2;
          }
          if (act && in) {
            const T r = r2 > T(0) ? sqrt(r2) : T(0);
            const T q = r * invH;
            const T t = q < T(1) ? T(1) - q : T(0);
            const T t3 = t * t * t;
            const T mW = Ls.m[k] * t3;
            rs += mW * t * (T(1) + T(4) * q);
            rhs += mW * (T(-3) + q * (T(-9) + T(32) * q));
            cnt += (Ls.idx[k] != (int)i);
          }
        }
      };

      for (int z = max(z0 - span, 0); z <= min(z1 + span, nz - 1); ++z)
        for (int y = max(y0 - span, 0); y <= min(y1 + span, ny - 1); ++y)
          for (int x = max(x0 - span, 0); x <= min(x1 + span, nx - 1); ++x) {
            const int c = (z * ny + y) * nx + x;
            const int s0 = A.cell_start[c];
            if (s0 < 0) continue;
            const int s1 = A.cell_end[c];
            const T ox = REL ? (T)(x - rx) * Lt : T(0);
            const T oy = REL ? (T)(y - ry) * Lt : T(0);
            const T oz = REL ? (T)(z - rz) * Lt : T(0);
            for (int jb = s0; jb < s1; jb += 32) {
              const int j = jb + lane;
              const bool ok = j < s1;
              V4 q;
              if (ok) q = Vec4<T>::load(A.w, j);
              else q.x = q.y = q.z = q.w = T(0);
              const T xj = q.x + ox, yj = q.y + oy, zj = q.z + oz;
              const T ex = fmax(bx0 - xj, fmax(T(0), xj - bx1));
              const T ey = fmax(by0 - yj, fmax(T(0), yj - by1));
              const T ez = fmax(bz0 - zj, fmax(T(0), zj - bz1));
              const bool keep = ok && (ex * ex + ey * ey + ez * ez < R * R * T(1.0001));
              const unsigned bal = __ballot_sync(kFull, keep);
              if (keep) {
                const int at = nl + __popc(bal & lanemask_lt());
                Ls.x[at] = xj;
                Ls.y[at] = yj;
                Ls.z[at] = zj;
                Ls.m[at] = q.w;
                Ls.idx[at] = j;
              }
              nl += __popc(bal);
              if (nl > CAP - 32) {
                __syncwarp();
                evaluate(nl);
                __syncwarp();
                nl = 0;
              }
            }
          }
      __syncwarp();
      evaluate(nl);
      __syncwarp();

      if (act) {
        // Eq. 1 and Eq. 3 with the kernel constants applied once
        const double ih = 1.0 / H;
        const double rho = cW * ih * ih * ih * (double)rs;
        const double rhoH = cW * ih * ih * ih * ih * (double)rhs;
        const double om = 1.0 + H / (3.0 * rho) * rhoH;
        const double gv = 4.0 * kPi / 3.0 * H * H * H * rho - target;
        rho_o = rho;
        om_o = om;
        cnt_o = cnt;
        H_o = H;
        sweeps_o = sweep;
        pairs += cnt;
        if (fabs(gv) <= A.p.h_tol * target) {
          state = 1;
        } else if (gv < 0.0 && H >= Hcap) {
          state = 2;
        } else {
          if (gv < 0.0) lo = H;
          else hi = H;
          const double gp = 4.0 * kPi * H * H * rho * om;
          double Hn = gp > 0.0 ? H - gv / gp : (gv < 0.0 ? 1.25 * H : 0.75 * H);
          if (!(Hn >= 0.75 * H)) Hn = 0.75 * H;
          if (!(Hn <= 1.25 * H)) Hn = 1.25 * H;
          if (hi < INFINITY && (Hn <= lo || Hn >= hi)) Hn = 0.5 * (lo + hi);
          if (Hn > Hcap) Hn = Hcap;
          H = Hn;
        }
      }
    }
    if (member && state == 0) state = 3;
  }

  if (valid) {
    A.s.h[i] = H_o;
    A.s.rho[i] = rho_o;
    A.s.omega[i] = om_o;
    A.s.nngb[i] = cnt_o;
  }
  // step record: one atomic of each kind per warp
  const int sw = wmax(valid ? sweeps_o : 0);
  const int nu = __popc(__ballot_sync(kFull, state == 3));
  const int ncap = __popc(__ballot_sync(kFull, state == 2));
  const bool bad = valid && !(isfinite(rho_o) && isfinite(om_o) && rho_o > 0.0);
  const unsigned nbad = __ballot_sync(kFull, bad);
  const double hm = wmax(valid ? H_o : 0.0);
  const long long pw = wsum(pairs);
  if (lane == 0) {
    atomicMax(&A.st->max_sweeps, sw);
    if (nu) {
      atomicAdd(&A.st->n_unconv, nu);
      atomicOr(&A.st->err, ERR_NOCONV);
    }
    if (ncap) atomicAdd(&A.st->n_capped, ncap);
    if (nbad) atomicOr(&A.st->err, ERR_NONFINITE);
    atomicMax(&A.st->hmax2_enc, enc_d(hm));
    atomicAdd(&A.st->pairs_density, (unsigned long long)pw);
  }
}

cudaError_t launch_density(sph_ctx *c) {
  DensArgs a;
  a.s = c->st;
  a.w = c->w;
  a.n = c->n;
  a.cell_start = c->cell_start;
  a.cell_end = c->cell_end;
  a.p = c->kp;
  a.st = c->d_status;
  const int64_t buckets = (c->n + 31) / 32;
  const int blocks = (int)((buckets + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (c->kp.precision == SPH_FP32K)
    k_density<float, 256><<<blocks, 32 * kWarpsPerBlock, 0, c->stream>>>(a);
  else
    k_density<double, 256><<<blocks, 32 * kWarpsPerBlock, 0, c->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sphk
