// sph_forces.cu -- equation of state, yield and radial return of the
// evaluation stress, and the full-stress pair loop with its per-particle
// finalize (§2.1-§2.3: Eq. 4-8, 13, 18-37).
//
// Pair loop layout: one warp per bucket of 32 cell-sorted particles (one per
// lane), grouped as in the density kernel. Candidates j (cells within
// ceil(max(H_bucket, H_max) / L_c), bounding-box filtered against
// max(H_bucket, H_j)) are staged in a per-warp shared-memory list. Each lane
// first tests the whole list against its particle (broadcast reads, one bit
// per candidate: r < max(H_i, H_j), j != i), then walks its own set bits
// independently, so the heavy pair body runs only for real neighbours. The
// neighbour data (velocity, mass, m sigma / (Omega rho^2), m / (Omega rho),
// c, rho, 1/H, kernel constant) come from packed 16-byte vectors.
//
// The per-pair sums use the algebraically equal contracted forms
//   a_i   += m_j W'_i/r sig~_i x_ij + W'_j/r (m sig~)_j x_ij      (Eq. 4, 18)
//   du_i  += -m_j W'_i/r v_ij . (sig~_i x_ij)                     (Eq. 19, du|_H)
//   F_i   += g_ij v_ij (x) x_ij,  C_i^-1 += g_ij x_ij (x) x_ij      (Eq. 20-21)
// with sig~ = (-P I + S) / (Omega rho^2), W'/r the radial kernel derivative
// over r and g_ij = -1/2 (m_j W'_i/r / (Omega_i rho_i) + W'_j/r m_j /
// (Omega_j rho_j)), since every kernel gradient points along x_ij. In the
// FP32 form the energy and the F, C^-1 sums are Kahan-compensated.
#include <type_traits>

#include "sph_internal.cuh"

namespace sphk {

// ------------------------------------------------------------ EOS + pack
__global__ void __launch_bounds__(kBlock) k_eos_pack(sph_state s, Work w, int64_t n, KParams P,
                                                    int fp32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const sph_material &M = P.mats[s.mat[i] & (SPH_MAX_MATERIALS - 1)];
    const double rho = s.rho[i], u = w.up[i], om = s.omega[i], m = s.m[i], H = s.h[i];
    const EosOut e = eos(M, rho, u);
    s.pres[i] = e.P;
    s.cs[i] = e.c;
    const double Y = yield(M, e.P, u);
    w.yld[i] = Y;
    double S[5] = {w.sp[0][i], w.sp[1][i], w.sp[2][i], w.sp[3][i], w.sp[4][i]};
    if (!M.strength) {
      S[0] = S[1] = S[2] = S[3] = S[4] = 0.0;
    } else {
      radial_return(S, Y, P.yield_norm);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) w.sp[k][i] = S[k];
    const double inv = m / (om * rho * rho);
    const double sxx = (S[0] - e.P) * inv, syy = (S[1] - e.P) * inv;
    const double szz = (-S[0] - S[1] - e.P) * inv;
    const double ih = 1.0 / H;
    const double K = cG * ih * ih * ih * ih * ih;
    if (fp32) {
      w.fj32[0][i] = make_float4((float)w.vp[0][i], (float)w.vp[1][i], (float)w.vp[2][i], (float)m);
      w.fj32[1][i] = make_float4((float)sxx, (float)syy, (float)szz, (float)(S[2] * inv));
      w.fj32[2][i] = make_float4((float)(S[3] * inv), (float)(S[4] * inv), (float)(m / (om * rho)),
                                 (float)e.c);
      w.fj32[3][i] = make_float4((float)rho, (float)ih, (float)K, (float)H);
    } else {
      w.fj64[0][i] = make_double4_32a(w.vp[0][i], w.vp[1][i], w.vp[2][i], m);
      w.fj64[1][i] = make_double4_32a(sxx, syy, szz, S[2] * inv);
      w.fj64[2][i] = make_double4_32a(S[3] * inv, S[4] * inv, m / (om * rho), e.c);
      w.fj64[3][i] = make_double4_32a(rho, ih, K, H);
    }
  }
}

cudaError_t launch_eos_pack(sph_ctx *c) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  k_eos_pack<<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->kp,
                                              c->kp.precision == SPH_FP32K);
  return cudaGetLastError();
}

// ------------------------------------------------------------- pair loop
template <typename T> struct FVec;
template <> struct FVec<float> {
  using type = float4;
  static __device__ __forceinline__ float4 pos(const Work &w, int64_t i) { return __ldg(w.pos32 + i); }
  static __device__ __forceinline__ float4 fj(const Work &w, int k, int64_t i) {
    return __ldg(w.fj32[k] + i);
  }
};
template <> struct FVec<double> {
  using type = double4_32a;
  static __device__ __forceinline__ double4_32a pos(const Work &w, int64_t i) { return w.pos64[i]; }
  static __device__ __forceinline__ double4_32a fj(const Work &w, int k, int64_t i) {
    return w.fj64[k][i];
  }
};

// Running sum: plain in FP64, Kahan-compensated in FP32.
template <typename T> struct Acc {
  T s = 0;
  __device__ __forceinline__ void add(T v) { s += v; }
  __device__ __forceinline__ double get() const { return (double)s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

template <typename T, int CAP> struct FList {
  T x[CAP], y[CAP], z[CAP], h[CAP];
  int idx[CAP];
  unsigned mask[CAP / 32][32];
};

struct ForceArgs {
  sph_state s;
  Work w;
  int64_t n;
  const int *cell_start, *cell_end;
  KParams p;
  Status *st;
};

template <typename T, int CAP>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_forces(ForceArgs A) {
  constexpr bool REL = std::is_same<T, float>::value;
  using V4 = typename FVec<T>::type;
  __shared__ FList<T, CAP> lists[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  FList<T, CAP> &Ls = lists[wib];
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
  const double hmax_all = dec_d(A.st->hmax2_enc);

  // particle i, evaluation state
  const V4 p = FVec<T>::pos(A.w, ic);
  const double Hd = A.s.h[ic], rhod = A.s.rho[ic], omd = A.s.omega[ic], Pd = A.s.pres[ic];
  const double cd = A.s.cs[ic];
  double Sd[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) Sd[k] = A.w.sp[k][ic];
  const double inv = 1.0 / (omd * rhod * rhod);
  const T sxx = (T)((Sd[0] - Pd) * inv), syy = (T)((Sd[1] - Pd) * inv);
  const T szz = (T)((-Sd[0] - Sd[1] - Pd) * inv);
  const T sxy = (T)(Sd[2] * inv), sxz = (T)(Sd[3] * inv), syz = (T)(Sd[4] * inv);
  const T iOr = (T)(1.0 / (omd * rhod));
  const T Hi = (T)Hd, invHi = (T)(1.0 / Hd);
  const T Ki = (T)(cG / (Hd * Hd * Hd * Hd * Hd));
  const T vix = (T)A.w.vp[0][ic], viy = (T)A.w.vp[1][ic], viz = (T)A.w.vp[2][ic];
  const T ci = (T)cd, rhoi = (T)rhod;
  const T al = (T)A.p.av_alpha, be = (T)A.p.av_beta, ep = (T)A.p.av_eps;

  T ax = 0, ay = 0, az = 0, mumax = 0;
  Acc<T> du, F[9], Ci[6];
  int npairs = 0;

  unsigned todo = __ballot_sync(kFull, valid);
  while (todo) {
    const int ref = __ffs(todo) - 1;
    const int rx = __shfl_sync(kFull, cx, ref), ry = __shfl_sync(kFull, cy, ref),
              rz = __shfl_sync(kFull, cz, ref);
    const bool act = ((todo >> lane) & 1u) && abs(cx - rx) <= 2 && abs(cy - ry) <= 2 &&
                     abs(cz - rz) <= 2;
    todo &= ~__ballot_sync(kFull, act);
    const T xi = REL ? p.x + (T)(cx - rx) * Lt : p.x;
    const T yi = REL ? p.y + (T)(cy - ry) * Lt : p.y;
    const T zi = REL ? p.z + (T)(cz - rz) * Lt : p.z;
    const T Rb = wmax(act ? Hi : T(0));
    const double Rf = fmax((double)Rb, hmax_all);
    const T bx0 = wmin(act ? xi : T(1e30)), bx1 = wmax(act ? xi : T(-1e30));
    const T by0 = wmin(act ? yi : T(1e30)), by1 = wmax(act ? yi : T(-1e30));
    const T bz0 = wmin(act ? zi : T(1e30)), bz1 = wmax(act ? zi : T(-1e30));
    const int x0 = wmin(act ? cx : 1 << 20), x1 = wmax(act ? cx : -1);
    const int y0 = wmin(act ? cy : 1 << 20), y1 = wmax(act ? cy : -1);
    const int z0 = wmin(act ? cz : 1 << 20), z1 = wmax(act ? cz : -1);
    const int span = max(1, (int)ceil(Rf / g.L));
    int nl = 0;

    auto process = [&](int nlist) {
      const int nw = (nlist + 31) >> 5;
      // 1) membership bits, broadcast reads of the list
      for (int wd = 0; wd < nw; ++wd) {
        unsigned mk = 0;
        const int kend = min(32, nlist - (wd << 5));
        for (int b = 0; b < kend; ++b) {
          const int k = (wd << 5) + b;
          const T dx = xi - Ls.x[k], dy = yi - Ls.y[k], dz = zi - Ls.z[k];
          const T r2 = dx * dx + dy * dy + dz * dz;
          const T Rk = Hi > Ls.h[k] ? Hi : Ls.h[k];
          const bool in = act && r2 < Rk * Rk && Ls.idx[k] != (int)i;
          mk |= (unsigned)in << b;
        }
        Ls.mask[wd][lane] = mk;
      }
      __syncwarp();
      // 2) each lane walks its own neighbours
      int wd = 0;
      unsigned mk = nw > 0 ? Ls.mask[0][lane] : 0u;
      for (;;) {
        while (mk == 0u && wd + 1 < nw) mk = Ls.mask[++wd][lane];
        if (mk == 0u) break;
        const int k = (wd << 5) + __ffs(mk) - 1;
        mk &= mk - 1u;
        const int j = Ls.idx[k];
        const T dx = xi - Ls.x[k], dy = yi - Ls.y[k], dz = zi - Ls.z[k];
        const T r2 = dx * dx + dy * dy + dz * dz;
        const T r = r2 > T(0) ? sqrt(r2) : T(0);
        const V4 f0 = FVec<T>::fj(A.w, 0, j);
        const V4 f1 = FVec<T>::fj(A.w, 1, j);
        const V4 f2 = FVec<T>::fj(A.w, 2, j);
        const V4 f3 = FVec<T>::fj(A.w, 3, j);
        T ti = T(1) - r * invHi;
        ti = ti > T(0) ? ti : T(0);
        T tj = T(1) - r * f3.y;
        tj = tj > T(0) ? tj : T(0);
        const T Wi = Ki * ti * ti * ti;          // W'(r, H_i) / r
        const T Wj = f3.z * tj * tj * tj;        // W'(r, H_j) / r
        const T mj = f0.w;
        const T vx = vix - f0.x, vy = viy - f0.y, vz = viz - f0.z;
        // sig~_i x_ij and (m sig~)_j x_ij
        const T yix = sxx * dx + sxy * dy + sxz * dz;
        const T yiy = sxy * dx + syy * dy + syz * dz;
        const T yiz = sxz * dx + syz * dy + szz * dz;
        const T yjx = f1.x * dx + f1.w * dy + f2.x * dz;
        const T yjy = f1.w * dx + f1.y * dy + f2.y * dz;
        const T yjz = f2.x * dx + f2.y * dy + f1.z * dz;
        const T mWi = mj * Wi;
        ax += mWi * yix + Wj * yjx;
        ay += mWi * yiy + Wj * yjy;
        az += mWi * yiz + Wj * yjz;
        T dsum = -mWi * (vx * yix + vy * yiy + vz * yiz);
        const T vr = vx * dx + vy * dy + vz * dz;
        if (vr < T(0)) {                        // Eq. 5-8
          const T hb = T(0.5) * (Hi + Ls.h[k]);
          const T mu = hb * vr / (r2 + ep * hb * hb);
          const T Pi = (-al * T(0.5) * (ci + f2.w) * mu + be * mu * mu) / (T(0.5) * (rhoi + f3.x));
          const T t = mj * Pi * T(0.5) * (Wi + Wj);
          ax -= t * dx;
          ay -= t * dy;
          az -= t * dz;
          dsum += T(0.5) * t * vr;
          mumax = -mu > mumax ? -mu : mumax;
        }
        du.add(dsum);
        const T gs = T(-0.5) * (mWi * iOr + Wj * f2.z);   // Eq. 20-21 weight
        const T gvx = gs * vx, gvy = gs * vy, gvz = gs * vz;
        F[0].add(gvx * dx); F[1].add(gvx * dy); F[2].add(gvx * dz);
        F[3].add(gvy * dx); F[4].add(gvy * dy); F[5].add(gvy * dz);
        F[6].add(gvz * dx); F[7].add(gvz * dy); F[8].add(gvz * dz);
        const T gx = gs * dx, gy = gs * dy;
        Ci[0].add(gx * dx); Ci[1].add(gx * dy); Ci[2].add(gx * dz);
        Ci[3].add(gy * dy); Ci[4].add(gy * dz); Ci[5].add(gs * dz * dz);
        ++npairs;
      }
      __syncwarp();
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
            V4 q, f3;
            if (ok) {
              q = FVec<T>::pos(A.w, j);
              f3 = FVec<T>::fj(A.w, 3, j);
            } else {
              q.x = q.y = q.z = q.w = T(0);
              f3.x = f3.y = f3.z = f3.w = T(0);
            }
            const T xj = q.x + ox, yj = q.y + oy, zj = q.z + oz;
            const T ex = fmax(bx0 - xj, fmax(T(0), xj - bx1));
            const T ey = fmax(by0 - yj, fmax(T(0), yj - by1));
            const T ez = fmax(bz0 - zj, fmax(T(0), zj - bz1));
            const T R = Rb > f3.w ? Rb : f3.w;
            const bool keep = ok && (ex * ex + ey * ey + ez * ez < R * R * T(1.0001));
            const unsigned bal = __ballot_sync(kFull, keep);
            if (keep) {
              const int at = nl + __popc(bal & lanemask_lt());
              Ls.x[at] = xj;
              Ls.y[at] = yj;
              Ls.z[at] = zj;
              Ls.h[at] = f3.w;
              Ls.idx[at] = j;
            }
            nl += __popc(bal);
            if (nl > CAP - 32) {
              __syncwarp();
              process(nl);
              nl = 0;
            }
          }
        }
    __syncwarp();
    process(nl);
  }

  // ------------------------------------------------ finalize (FP64)
  int fallback = 0;
  if (valid) {
    const sph_material &M = A.p.mats[A.s.mat[i] & (SPH_MAX_MATERIALS - 1)];
    const bool fixed = A.s.flags[i] & SPH_FLAG_FIXED;
    double Fm[9], Cm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
#pragma unroll
    for (int k = 0; k < 9; ++k) Fm[k] = F[k].get();
    const double c00 = Ci[0].get(), c01 = Ci[1].get(), c02 = Ci[2].get();
    const double c11 = Ci[3].get(), c12 = Ci[4].get(), c22 = Ci[5].get();
    if (A.p.correction) {
      // inverse of the symmetric C^-1 by cofactors (Eq. 21-22)
      const double k00 = c11 * c22 - c12 * c12, k01 = c02 * c12 - c01 * c22,
                   k02 = c01 * c12 - c02 * c11;
      const double det = c00 * k00 + c01 * k01 + c02 * k02;
      if (A.s.nngb[i] >= 8 && fabs(det) >= 1e-3) {
        const double id = 1.0 / det;
        Cm[0] = k00 * id;
        Cm[1] = Cm[3] = k01 * id;
        Cm[2] = Cm[6] = k02 * id;
        Cm[4] = (c00 * c22 - c02 * c02) * id;
        Cm[5] = Cm[7] = (c02 * c01 - c00 * c12) * id;
        Cm[8] = (c00 * c11 - c01 * c01) * id;
      } else {
        fallback = 1;
      }
    }
    double G[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        G[3 * a + b] = Fm[3 * a] * Cm[b] + Fm[3 * a + 1] * Cm[3 + b] + Fm[3 * a + 2] * Cm[6 + b];
    // strain rate and rotation rate (Eq. 23-24)
    double E[9], R[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        E[3 * a + b] = 0.5 * (G[3 * a + b] + G[3 * b + a]);
        R[3 * a + b] = 0.5 * (G[3 * a + b] - G[3 * b + a]);
      }
    double e2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) e2 += E[k] * E[k];
    const double Gam = shear_mod(M, rhod, cd);
    double dS[5] = {0, 0, 0, 0, 0};
    if (M.strength) {
      const double Sm[9] = {Sd[0], Sd[2], Sd[3], Sd[2], Sd[1], Sd[4], Sd[3], Sd[4], -Sd[0] - Sd[1]};
      const double tr3 = (E[0] + E[4] + E[8]) / 3.0;
      const double sg = A.p.jaumann == SPH_JAUMANN_PRINTED ? -1.0 : 1.0;
      const int ia[5] = {0, 1, 0, 0, 1}, ib[5] = {0, 1, 1, 2, 2};
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int a = ia[q], b = ib[q];
        double rot = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) rot += R[3 * a + k] * Sm[3 * k + b] - Sm[3 * a + k] * R[3 * k + b];
        dS[q] = 2.0 * Gam * (E[3 * a + b] - (a == b ? tr3 : 0.0)) + sg * rot;
      }
    }
    double gx[3];
    ext_field(A.p, A.s.x[i], A.s.y[i], A.s.z[i], gx, nullptr);
    const double cl = M.strength ? sqrt(cd * cd + 4.0 / 3.0 * Gam / rhod) : cd;
    A.w.vsig[i] = (1.0 + 0.6 * A.p.av_alpha) * cl + 0.6 * A.p.av_beta * (double)mumax;
    A.w.edot2[i] = 0.5 * e2;
    const double axd = (double)ax + gx[0], ayd = (double)ay + gx[1], azd = (double)az + gx[2];
    const double dud = du.get();
    A.s.ax[i] = fixed ? 0.0 : axd;
    A.s.ay[i] = fixed ? 0.0 : ayd;
    A.s.az[i] = fixed ? 0.0 : azd;
    A.s.dudt[i] = fixed ? 0.0 : dud;
    A.s.dsxx[i] = fixed ? 0.0 : dS[0];
    A.s.dsyy[i] = fixed ? 0.0 : dS[1];
    A.s.dsxy[i] = fixed ? 0.0 : dS[2];
    A.s.dsxz[i] = fixed ? 0.0 : dS[3];
    A.s.dsyz[i] = fixed ? 0.0 : dS[4];
    bool fin = isfinite(axd) && isfinite(ayd) && isfinite(azd) && isfinite(dud);
#pragma unroll
    for (int k = 0; k < 5; ++k) fin = fin && isfinite(dS[k]);
    if (!fin) atomicOr(&A.st->err, ERR_NONFINITE);
  }
  const int nfb = __popc(__ballot_sync(kFull, fallback != 0));
  const long long pw = wsum((long long)npairs);
  if (lane == 0) {
    if (nfb) atomicAdd(&A.st->n_cfallback, nfb);
    atomicAdd(&A.st->pairs_force, (unsigned long long)pw);
  }
}

cudaError_t launch_forces(sph_ctx *c) {
  ForceArgs a;
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
    k_forces<float, 256><<<blocks, 32 * kWarpsPerBlock, 0, c->stream>>>(a);
  else
    k_forces<double, 256><<<blocks, 32 * kWarpsPerBlock, 0, c->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sphk
