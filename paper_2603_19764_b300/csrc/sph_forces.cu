// sph_forces.cu -- equation of state, yield and radial return of the
// evaluation stress, and the full-stress pair loop with its per-particle
// finalize (§2.1-§2.3: Eq. 4-8, 13, 18-37).
//
// Pair loop layout: one warp per bucket of 32 cell-sorted particles (one per
// lane), grouped as in the density kernel (sph_pair.cuh). Candidates j from
// the cells overlapping the group's box grown by max(H_group, H_max) are
// kept when within max(H_group, H_j) of the box and staged in shared memory
// as (x, y, z, H^2). Each lane marks the candidates with
// r^2 < max(H_i, H_j)^2 (broadcast reads, one bit per candidate; the H_i
// radius is widened by the guard band of sph_pair.cuh so that the count
// below loses no pair to FP32 rounding), then walks its own set bits
// independently, so the heavy pair body runs only for real neighbours. A pair at r = 0 (the particle itself, or a coincident
// one) contributes nothing to any sum below (every term carries x_ij); the
// walk also counts the neighbours r < H_i of the smoothing-length solve.
//
// The per-pair sums use the algebraically equal contracted forms
//   a_i   += m_j W'_i/r sig~_i x_ij + W'_j/r (m sig~)_j x_ij      (Eq. 4, 18)
//   du_i  += -m_j W'_i/r v_ij . (sig~_i x_ij)                     (Eq. 19, du|_H)
//   F_i   += g_ij v_ij (x) x_ij,  C_i^-1 += g_ij x_ij (x) x_ij      (Eq. 20-21)
// with sig~ = (-P I + S) / (Omega rho^2), W'/r the radial kernel derivative
// over r and g_ij = -1/2 (m_j W'_i/r / (Omega_i rho_i) + W'_j/r m_j /
// (Omega_j rho_j)), since every kernel gradient points along x_ij. In the
// FP32 form the energy and the F, C^-1 sums are Kahan-compensated, and the
// per-particle finalize runs in FP32 as well: FP64 stays in positions,
// integration and global sums.
#include "sph_kick.cuh"
#include "sph_pair.cuh"

namespace sphk {

// ------------------------------------------------------------ EOS + pack
template <typename T> struct Packed;
template <> struct Packed<float> {
  using V4 = float4;
  static __device__ __forceinline__ const float4 *pos(const Work &w) { return w.pos32; }
  static __device__ __forceinline__ float4 *posh(const Work &w) { return w.posh32; }
  static __device__ __forceinline__ float4 *rec(const Work &w) { return w.fj32; }
  static __device__ __forceinline__ float4 *fs(const Work &w, int k) { return w.fs32[k]; }
};
template <> struct Packed<double> {
  using V4 = double4_32a;
  static __device__ __forceinline__ const double4_32a *pos(const Work &w) { return w.pos64; }
  static __device__ __forceinline__ double4_32a *posh(const Work &w) { return w.posh64; }
  static __device__ __forceinline__ double4_32a *rec(const Work &w) { return w.fj64; }
  static __device__ __forceinline__ double4_32a *fs(const Work &w, int k) { return w.fs64[k]; }
};

// Per particle: the evaluation state (predict = 1: v, u, S at i from the
// half-step values of the read view src and the derivatives at i-1, Eq. 40;
// predict = 0: the state as it stands), EOS at (rho, u_eval), yield, radial
// return of the evaluation stress, and the packed neighbour / own data of
// the pair loop:
//   posh = (x, y, z, H), and the neighbour record of 4 consecutive vectors
//   rec0 = (v, m)   rec1 = m/(Omega rho^2) (sxx, syy, szz, sxy), s = -P I + S
//   rec2 = (m sxz', m syz', m/(Omega rho), c)   rec3 = (rho/2, 1/H, cG/H^5, H/2)
//   fs0 = (Sxx, Syy, Sxy, Sxz)   fs1 = (Syz, Gamma, c_L, 0)   fs2 = (g, 0)
// This kernel's own conversions use the conversion instructions: it is not
// bound by the FP64 unit that runs them (the integer-pipe forms of to_t and
// from_t serve the kernels that are), and they need no branch.
template <typename T> __device__ __forceinline__ T cvt_t(double d) { return (T)d; }
// Six blocks per SM (40 registers): latency-bound, so more resident warps
// help (3 % over five blocks at 48 registers; eight spill).
template <typename T>
__global__ void __launch_bounds__(kBlock, 6) k_eos_pack(sph_state s, sph_state src, Work w,
                                                    int64_t n, KParams P, int predict) {
  using V = V4T<T>;
  const typename V::type *pos = Packed<T>::pos(w);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // offset from the half step: dt / 2, or with rungs the time from the
    // midpoint of the particle's own step to the end of this substep
    const bool fixed = s.flags[i] & SPH_FLAG_FIXED;
    double k = 0.0;
    if (predict && !fixed) {
      const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, i) : 0;
      k = predict_offset(P, i, P.dt[sy] * P.sub_scale);
    }
    const double ud = src.u[i] + k * src.dudt[i];
    const MatT<T> &M = mat_t<T>(P, s.mat[i]);
    const double rhod = s.rho[i];
    const EosT<T> e = eos_t<T>(M, rhod, ud);
    s.pres[i] = (double)e.P;
    s.cs[i] = (double)e.c;
    const T Y = yield_t<T>(M, e.P, cvt_t<T>(ud));
    T S[5] = {cvt_t<T>(src.sxx[i] + k * src.dsxx[i]), cvt_t<T>(src.syy[i] + k * src.dsyy[i]),
              cvt_t<T>(src.sxy[i] + k * src.dsxy[i]), cvt_t<T>(src.sxz[i] + k * src.dsxz[i]),
              cvt_t<T>(src.syz[i] + k * src.dsyz[i])};
    if (!M.strength) {
      S[0] = S[1] = S[2] = S[3] = S[4] = T(0);
    } else {
      const T f = radial_factor_t<T>(S, Y, P.yield_norm);
#pragma unroll
      for (int k = 0; k < 5; ++k) S[k] *= f;
    }
    const typename V::type pp = pos[i];
    const T rho = cvt_t<T>(rhod), om = cvt_t<T>(s.omega[i]), m = cvt_t<T>(s.m[i]),
            H = cvt_t<T>(s.h[i]);
    const T inv = quot(m, om * rho * rho);
    const T ih = quot(T(1), H);
    const T ih2 = ih * ih;
    const T K = T(cG) * ih2 * ih2 * ih;
    const T Gam = M.strength ? shear_mod_t<T>(M, rho, e.c) : T(0);
    const T cl = M.strength ? root(e.c * e.c + quot(T(4.0 / 3.0) * Gam, rho)) : e.c;
    T gx[3];
    ext_field_t<T>(P, s.x[i], s.y[i], s.z[i], gx, nullptr);
    Packed<T>::posh(w)[i] = V::make(pp.x, pp.y, pp.z, H);
    typename V::type *rec = Packed<T>::rec(w) + 4 * i;
    rec[0] = V::make(cvt_t<T>(src.vx[i] + k * src.ax[i]), cvt_t<T>(src.vy[i] + k * src.ay[i]),
                     cvt_t<T>(src.vz[i] + k * src.az[i]), m);
    rec[1] =
        V::make((S[0] - e.P) * inv, (S[1] - e.P) * inv, (-S[0] - S[1] - e.P) * inv, S[2] * inv);
    rec[2] = V::make(S[3] * inv, S[4] * inv, quot(m, om * rho), e.c);
    // halves (exact) for the pair means of Eq. 5-8: rho_i/2 + rho_j/2 is
    // the rounded (rho_i + rho_j)/2 bit for bit
    rec[3] = V::make(T(0.5) * rho, ih, K, T(0.5) * H);
    Packed<T>::fs(w, 0)[i] = V::make(S[0], S[1], S[2], S[3]);
    Packed<T>::fs(w, 1)[i] = V::make(S[4], Gam, cl, T(0));
    Packed<T>::fs(w, 2)[i] = V::make(gx[0], gx[1], gx[2], T(0));
  }
}

cudaError_t launch_eos_pack(sph_ctx *c, int predict) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  // v, u, S and the derivatives at i-1 through the step's read view (the
  // permuted copies when they were not copied back)
  if (c->kp.precision == SPH_FP32K)
    k_eos_pack<float><<<(int)b, kBlock, 0, c->stream>>>(c->st, c->src, c->w, c->n, c->kp,
                                                        predict);
  else
    k_eos_pack<double><<<(int)b, kBlock, 0, c->stream>>>(c->st, c->src, c->w, c->n, c->kp,
                                                         predict);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------- pair loop
// Running sums of the pair loop. FP64 form: plain. FP32 form, energy and
// velocity-gradient sums (du, F): compensated in blocks -- the terms of
// kSumBlock consecutive pairs are added plainly, then each block sum enters
// a Kahan sum, which bounds the error by a block's rounding (kSumBlock ulp
// of the block's terms) at an eighth of the cost of compensating every
// term. The correction-tensor sums C^-1 = sum g x x (Eq. 21) are added
// plainly in both forms: their diagonal terms share one sign, and their
// rounding error is a few ulp of the matrix norm.
constexpr int kSumBlock = 8;
template <typename T> struct Acc {
  T s = 0;
  __device__ __forceinline__ void add(T v) { s += v; }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ T get() const { return s; }
};
template <> struct Acc<float> {
  float p = 0.f, s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) { p += v; }
  __device__ __forceinline__ void flush() {
    const float y = p - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
    p = 0.f;
  }
  __device__ __forceinline__ float get() const { return s - c; }
};
template <typename T> struct Plain {
  T s = 0;
  __device__ __forceinline__ void add(T v) { s += v; }
  __device__ __forceinline__ T get() const { return s; }
};

template <typename T> struct FList;
template <> struct FList<float> {
  template <int S> static __device__ __forceinline__ ViewPlanes<S> at(void *p) {
    return ViewPlanes<S>{reinterpret_cast<float *>(p)};
  }
};
template <> struct FList<double> {
  template <int S> static __device__ __forceinline__ ViewAoS<double4_32a> at(void *p) {
    return ViewAoS<double4_32a>{reinterpret_cast<double4_32a *>(p)};
  }
};

struct ForceArgs {
  sph_state s;
  Work w;
  int64_t n;
  const int *cell_start, *cell_end;
  KParams p;
  Status *st;
  // global steps: kick each particle once its derivatives are formed (v,
  // u, S and the strain invariant read from src, written to s; its terms
  // of the step's sums to the work arrays)
  int kick;
  sph_state src;
  // buckets [b_begin, min(b_end, bucket count)) taken through *counter
  int b_begin, b_end;
  unsigned *counter;
};

// Three 4-warp blocks per SM: the pair body and its compensated sums fit in
// the ~170 registers a thread then has, without spilling (at four blocks,
// 128 registers, they spill and the kernel runs 1.5 % slower).
// UF: staging depth, the chunks of 32 stream positions located and loaded
// at once (kDepths; the lists do not depend on it)
template <typename T, int CAP, bool PER, int UF>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 3) k_forces(ForceArgs A) {
  constexpr bool REL = std::is_same<T, float>::value;
  using V = V4T<T>;
  using V4 = typename V::type;
  using PK = Packed<T>;
  __shared__ V4 s_rec[kWarpsPerBlock][CAP];
  __shared__ int s_idx[kWarpsPerBlock][CAP];
  __shared__ unsigned s_mask[kWarpsPerBlock][CAP / 32][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the candidate list: planes in the FP32 form (packed mask tests),
  // one record per candidate in the FP64 form
  const auto Lr = FList<T>::template at<CAP>(s_rec[wib]);
  int *Li = s_idx[wib];
  unsigned(*Lm)[32] = s_mask[wib];
  // persistent warps: each takes the next bucket of 32 particles
  const int n_act = A.p.act ? A.st->n_active : 0;
  const int nbuckets = bucket_count(A.p, n_act);
  long long w_pairs = 0, w_cand = 0;
  int w_fb = 0, w_groups = 0, w_upd = 0;
  unsigned w_box = 0;
  // a periodic box must be wider than twice every search radius
  const T box_min = PER ? (T)fmin(fmin(A.p.box_len[0], A.p.box_len[1]), A.p.box_len[2]) : T(0);
  for (;;) {
  unsigned bk = 0;
  if (lane == 0) bk = (unsigned)A.b_begin + atomicAdd(A.counter, 1u);
  bk = __shfl_sync(kFull, bk, 0);
  if ((int)bk >= nbuckets || (int)bk >= A.b_end) break;
  // the bucket's system and its sorted range
  const BucketLane bl = bucket_lane(A.p, n_act, bk, lane, A.n, &A.st->err);
  const int sy = bl.sy;
  const SysRec &R = A.p.sys[sy];
  const int64_t i = bl.i;
  // with hierarchical steps only particles whose step ends get derivatives
  const bool valid = bl.valid && rung_active(A.p, i);
  const int64_t ic = bl.ic;
  const V4 *posh = PK::posh(A.w);
  const V4 *rec = PK::rec(A.w);   // 4 consecutive vectors per particle

  if (A.kick && valid) {
    // the kick in this bucket's epilogue reads these: ask L2 for them now,
    // so that their DRAM latency passes while the pair loop runs
    const void *const pf[] = {A.src.vx + i, A.src.vy + i, A.src.vz + i, A.src.u + i,
                              A.src.sxx + i, A.src.syy + i, A.src.sxy + i, A.src.sxz + i,
                              A.src.syz + i, A.src.eps_ii + i, A.s.m + i, A.s.rho + i,
                              A.s.x + i, A.s.y + i, A.s.z + i, A.s.mat + i};
#pragma unroll
    for (const void *q : pf) prefetch_l2(q);
  }
  const Grid g = R.grid;
  const T Lt = grid_L<T>(g), invL = grid_invL<T>(g);
  const int cc = A.w.cc[ic];
  const int cx = cc & 1023, cy = (cc >> 10) & 1023, cz = (cc >> 20) & 1023;
  const T hmax_all = to_t<T>(dec_d(R.hmax2_enc));

  // particle i (evaluation state, packed)
  const V4 p = V::ld(posh, ic);
  const V4 a0 = V::ld(rec, 4 * ic), a1 = V::ld(rec, 4 * ic + 1), a2 = V::ld(rec, 4 * ic + 2),
           a3 = V::ld(rec, 4 * ic + 3);
  const T im = T(1) / a0.w;
  const T sxx = a1.x * im, syy = a1.y * im, szz = a1.z * im, sxy = a1.w * im;
  // iOr: the H_i weight of Eq. 20-21 over Omega_i rho_i
  const T sxz = a2.x * im, syz = a2.y * im,
          iOr = a2.z * im * pconst<T>(A.p.grad_wi, A.p.grad_wi_f);
  const T Hi = p.w, Hi2 = p.w * p.w, invHi = a3.y, Ki = a3.z;
  const T gi = guard_band(Hi, Lt);   // r^2 band the FP32 sum cannot decide
  const T vix = a0.x, viy = a0.y, viz = a0.z, ci = a2.w, rhoi_h = a3.x, Hi_h = T(0.5) * Hi;
  // neighbour count of particle i (r < H_i by the canonical predicate):
  // the density solve may close on an expanded sum and leave it to this pass
  int nngb = 0;
  const T al = pconst<T>(A.p.av_alpha, A.p.av_alpha_f);
  const T be = pconst<T>(A.p.av_beta, A.p.av_beta_f);
  const T ep = pconst<T>(A.p.av_eps, A.p.av_eps_f);

  T ax = 0, ay = 0, az = 0, mumax = 0;
  Acc<T> du, F0, F1, F2, F3, F4, F5, F6, F7, F8;
  Plain<T> C0, C1, C2, C3, C4, C5;
  int npairs = 0, blk = 0;
  long long cand = 0;

  unsigned todo = __ballot_sync(kFull, valid);
  while (todo) {
    const Group G = next_group(todo, cx, cy, cz, A.p.span_f);
    ++w_groups;
    const bool act = G.member;
    const T xi = REL ? rel_coord(p.x, cx - G.rx, Lt) : p.x;
    const T yi = REL ? rel_coord(p.y, cy - G.ry, Lt) : p.y;
    const T zi = REL ? rel_coord(p.z, cz - G.rz, Lt) : p.z;
    const T Rb = wmax(act ? Hi : T(0));
    // lists and masks reach r^2 < H_i^2 + gi: no pair with r < H_i by the
    // FP64 predicate escapes the count
    const T gmax = guard_band(Rb, Lt);
    // (hmax_all includes the staging skin of a substep that kept the last
    // order: every radius it bounds was raised by the skin)
    const T Rf = tmax(Rb, hmax_all) + T(1e-5) * tmax(Rb, Lt);
    if (PER && !(T(2) * Rf < box_min)) w_box = 1u;
    const Box<T> bx = group_box(act, xi, yi, zi);
    auto sg = make_stager_for<T, REL, PER>(bx, Rf, g, invL, A.p, G.rx, G.ry, G.rz);
    for (;;) {
      // stage candidates
      const int nl = stage_list<UF, false, T, REL>(
          sg, g, A.cell_start, A.cell_end, Lt, A.p, G.rx, G.ry, G.rz, 0, CAP, A.n, &A.st->err,
          [&](bool ok, int j) { return ok ? V::ld(posh, j) : V::make(0, 0, 0, 0); },
          [&](bool ok, const V4 &q, T ox, T oy, T oz, T &xj, T &yj, T &zj) {
            xj = add_rn(q.x, ox);
            yj = add_rn(q.y, oy);
            zj = add_rn(q.z, oz);
            const T R = tmax(Rb, q.w);
            return ok &&
                   box_d2(xj, yj, zj, bx.x0, bx.x1, bx.y0, bx.y1, bx.z0, bx.z1) < R * R + gmax;
          },
          [&](int at, T xj, T yj, T zj, const V4 &q, int j) {
            Lr.put(at, xj, yj, zj, q.w * q.w);
            Li[at] = j;
          });
      cand += nl;
      __syncwarp();
      // membership bits: r^2 < max(H_i^2 + gi, H_j^2)
      const int nw = (nl + 31) >> 5;
      for (int wd = 0; wd < nw; ++wd) {
        const int kb = wd << 5;
        const T Hi2g = Hi2 + gi;
        const unsigned mk = mask_word(Lr, kb, min(32, nl - kb), xi, yi, zi,
                                      [Hi2g](T w) { return tmax(Hi2g, w); });
        Lm[wd][lane] = act ? mk : 0u;
      }
      __syncwarp();
      // each lane walks its own neighbours, independently of the others.
      // FP32 form: the next neighbour's 64-byte record is loaded one pair
      // ahead, so that its latency overlaps the current pair's arithmetic
      // (the FP64 record would take 32 more registers and spill)
      constexpr bool PF = REL;
      int wd = 0;
      unsigned mk = nw > 0 ? Lm[0][lane] : 0u;
      while (mk == 0u && ++wd < nw) mk = Lm[wd][lane];
      bool more = mk != 0u;
      int kn = 0, jn = 0;
      V4 g0, g1, g2, g3;   // the prefetched record, in two 32-byte loads
      if (more) {
        kn = (wd << 5) + take_next(mk);
        jn = (int)checked(Li[kn], A.n, &A.st->err);
        if (PF) {
          V::ld2(rec + 4 * jn, g0, g1);
          V::ld2(rec + 4 * jn + 2, g2, g3);
        }
      }
      while (more) {
        {
          const int k = kn, j = jn;
          V4 f0, f1, f2, f3;
          if (PF) {
            f0 = g0; f1 = g1; f2 = g2; f3 = g3;
          } else {
            V::ld2(rec + 4 * j, f0, f1);
            V::ld2(rec + 4 * j + 2, f2, f3);
          }
          while (mk == 0u && ++wd < nw) mk = Lm[wd][lane];
          more = mk != 0u;
          if (PF) {
            // without a branch: after the lane's last pair the index stays
            // at the current pair and its record is loaded once more
            const int b = take_next(mk);   // mk stays 0 after the last pair
            kn = more ? (wd << 5) + b : kn;
            jn = (int)checked(Li[kn], A.n, &A.st->err);
            V::ld2(rec + 4 * jn, g0, g1);
            V::ld2(rec + 4 * jn + 2, g2, g3);
          } else if (more) {
            kn = (wd << 5) + take_next(mk);
            jn = (int)checked(Li[kn], A.n, &A.st->err);
          }
          T qx, qy, qz, qw;   // qw = H_j^2
          Lr.get(k, qx, qy, qz, qw);
          const T dx = xi - qx, dy = yi - qy, dz = zi - qz;
          // the mask test's rounding order, so that the walk and the marks
          // agree on every pair
          const T r2 = dist2(dx, dy, dz);
          {
            bool inH;
            if (REL) {
              inH = r2 < Hi2;
              if (fabs(r2 - Hi2) < gi) {   // rare: decide in FP64
                const double h = A.s.h[i];
                const double ex = A.s.x[i] - A.s.x[j], ey = A.s.y[i] - A.s.y[j],
                             ez = A.s.z[i] - A.s.z[j];
                inH = (PER ? r2_canon_periodic(ex, ey, ez, A.p.box_len) : r2_canon(ex, ey, ez)) <
                      __dmul_rn(h, h);
              }
            } else {
              const double h = A.s.h[i];
              const double h2 = __dmul_rn(h, h);
              const double c2 = r2_canon((double)dx, (double)dy, (double)dz);
              inH = c2 < h2;
              // a shifted image's coordinate was rounded once more than the
              // minimum image of x_i - x_j: decide the rare pair at the
              // boundary with the canonical arithmetic
              if (PER && fabs(c2 - h2) < 1e-12 * h * fmax(h, (double)box_min))
                inH = r2_canon_periodic(A.s.x[i] - A.s.x[j], A.s.y[i] - A.s.y[j],
                                        A.s.z[i] - A.s.z[j], A.p.box_len) < h2;
            }
            nngb += inH ? 1 : 0;   // the particle itself included, taken off below
          }
          // a pair marked only for the count (r^2 in the band past both
          // radii) has no say in the signal velocity and no place in the
          // pair statistics; its kernel weights are zero up to the rounding
          // of r / H (below 1e-20 of a neighbour's)
          const bool inR = r2 < tmax(Hi2, qw);
          // a pair at r = 0 (the particle itself, or a coincident one)
          // contributes nothing below: every term carries x_ij
          const T r = root(r2);
          const T ti = tmax(T(1) - r * invHi, T(0));
          const T tj = tmax(T(1) - r * f3.y, T(0));
          const T Wi = Ki * ti * ti * ti;   // W'(r, H_i) / r
          const T Wj = f3.z * tj * tj * tj; // W'(r, H_j) / r
          const T mj = f0.w;
          const T vx = vix - f0.x, vy = viy - f0.y, vz = viz - f0.z;
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
          // Eq. 5-8 for approaching pairs. FP32 form: evaluated for every pair
          // with mu = 0 for the others (cheaper than the divergent branch);
          // FP64 form: branched, its divides being costly
          const bool av = vr < T(0) && inR;
          if (REL || av) {
            const T hb = Hi_h + f3.w;   // (H_i + H_j) / 2
            const T mu0 = quot(hb * vr, r2 + ep * hb * hb);
            const T mu = av ? mu0 : T(0);
            const T Pi = quot((be * mu - al * T(0.5) * (ci + f2.w)) * mu, rhoi_h + f3.x);
            const T t = T(0.5) * mj * Pi * (Wi + Wj);
            ax -= t * dx;
            ay -= t * dy;
            az -= t * dz;
            dsum += T(0.5) * t * vr;
            mumax = tmax(mumax, -mu);
          }
          du.add(dsum);
          // Eq. 20-21 weight (the one-sided form: H_j weight 0)
          const T gs = mWi * iOr + Wj * (f2.z * pconst<T>(A.p.grad_wj, A.p.grad_wj_f));
          const T gvx = gs * vx, gvy = gs * vy, gvz = gs * vz;
          F0.add(gvx * dx); F1.add(gvx * dy); F2.add(gvx * dz);
          F3.add(gvy * dx); F4.add(gvy * dy); F5.add(gvy * dz);
          F6.add(gvz * dx); F7.add(gvz * dy); F8.add(gvz * dz);
          const T gx = gs * dx, gy = gs * dy;
          C0.add(gx * dx); C1.add(gx * dy); C2.add(gx * dz);
          C3.add(gy * dy); C4.add(gy * dz); C5.add(gs * dz * dz);
          npairs += inR ? 1 : 0;   // the particle itself included, taken off below
          if (++blk == kSumBlock) {   // lanes stay in step: one pair per pass each
            blk = 0;
            du.flush(); F0.flush(); F1.flush(); F2.flush(); F3.flush();
            F4.flush(); F5.flush(); F6.flush(); F7.flush(); F8.flush();
          }
        }
      }
      __syncwarp();
      if (stager_finished(sg)) break;
    }
  }

  du.flush(); F0.flush(); F1.flush(); F2.flush(); F3.flush();
  F4.flush(); F5.flush(); F6.flush(); F7.flush(); F8.flush();
  // ---------------------------------------- finalize (Eq. 21-29, 38-39)
  int fallback = 0;
  if (valid) {
    // the walk counted the particle itself (r = 0, always in range)
    nngb -= 1;
    npairs -= 1;
    const V4 s0 = V::ld(PK::fs(A.w, 0), i), s1 = V::ld(PK::fs(A.w, 1), i),
             s2 = V::ld(PK::fs(A.w, 2), i);
    const bool fixed = A.s.flags[i] & SPH_FLAG_FIXED;
    const T F[9] = {F0.get(), F1.get(), F2.get(), F3.get(), F4.get(),
                    F5.get(), F6.get(), F7.get(), F8.get()};
    const T c00 = C0.get(), c01 = C1.get(), c02 = C2.get();
    const T c11 = C3.get(), c12 = C4.get(), c22 = C5.get();
    T Cm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (A.p.correction) {
      // inverse of the symmetric C^-1 by cofactors (Eq. 21-22)
      const T k00 = c11 * c22 - c12 * c12, k01 = c02 * c12 - c01 * c22,
              k02 = c01 * c12 - c02 * c11;
      const T det = c00 * k00 + c01 * k01 + c02 * k02;
      if (nngb >= 8 && fabs(det) >= T(1e-3)) {
        const T id = T(1) / det;
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
    T G[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        G[3 * a + b] = F[3 * a] * Cm[b] + F[3 * a + 1] * Cm[3 + b] + F[3 * a + 2] * Cm[6 + b];
    T E[9], R[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        E[3 * a + b] = T(0.5) * (G[3 * a + b] + G[3 * b + a]);
        R[3 * a + b] = T(0.5) * (G[3 * a + b] - G[3 * b + a]);
      }
    T e2 = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) e2 += E[k] * E[k];
    // Eq. 13 with R S - S R (objective) or S R - R S (Eq. 25-29 as printed)
    const T Gam = s1.y;
    const T Sm[9] = {s0.x, s0.z, s0.w, s0.z, s0.y, s1.x, s0.w, s1.x, -s0.x - s0.y};
    const T tr3 = (E[0] + E[4] + E[8]) / T(3);
    const T sg = A.p.jaumann == SPH_JAUMANN_PRINTED ? T(-1) : T(1);
    T dS[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int a = q == 1 || q == 4 ? 1 : 0;
      const int b = q == 0 ? 0 : (q == 1 || q == 2 ? 1 : 2);
      T rot = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) rot += R[3 * a + k] * Sm[3 * k + b] - Sm[3 * a + k] * R[3 * k + b];
      dS[q] = T(2) * Gam * (E[3 * a + b] - (a == b ? tr3 : T(0))) + sg * rot;
    }
    KickIn kd;
    kd.vsig = from_t((T(1) + T(0.6) * al) * s1.z + T(0.6) * be * mumax);
    kd.edot2 = from_t(T(0.5) * e2);
    A.w.vsig[i] = kd.vsig;
    A.s.nngb[i] = nngb;
    A.w.edot2[i] = kd.edot2;
    if (A.w.divv) A.w.divv[i] = (float)(E[0] + E[4] + E[8]);
    const T axt = ax + s2.x, ayt = ay + s2.y, azt = az + s2.z;
    const T dud = du.get();
    kd.a[0] = fixed ? 0.0 : from_t(axt);
    kd.a[1] = fixed ? 0.0 : from_t(ayt);
    kd.a[2] = fixed ? 0.0 : from_t(azt);
    kd.dudt = fixed ? 0.0 : from_t(dud);
#pragma unroll
    for (int k = 0; k < 5; ++k) kd.dS[k] = fixed ? 0.0 : from_t(dS[k]);
    A.s.ax[i] = kd.a[0];
    A.s.ay[i] = kd.a[1];
    A.s.az[i] = kd.a[2];
    A.s.dudt[i] = kd.dudt;
    A.s.dsxx[i] = kd.dS[0];
    A.s.dsyy[i] = kd.dS[1];
    A.s.dsxy[i] = kd.dS[2];
    A.s.dsxz[i] = kd.dS[3];
    A.s.dsyz[i] = kd.dS[4];
    bool fin = isfinite(axt) && isfinite(ayt) && isfinite(azt) && isfinite(dud);
#pragma unroll
    for (int k = 0; k < 5; ++k) fin = fin && isfinite(dS[k]);
    if (!fin) atomicOr(&A.st->err, ERR_NONFINITE);
    // the kicks of a global step (§2.4): particle i's derivatives are final
    // here, and no other warp of this pass reads its v, u or S
    if (A.kick) {
      double term[kNSum], tcr;
      kick_particle<T>(A.s, A.src, A.w, A.p, i, true, A.p.dt[sy], true, A.src.vx != A.s.vx, kd,
                       term, &tcr, w_upd, nullptr);
      // left for the reduction kernels, which add them in the kick
      // kernel's order
#pragma unroll
      for (int k = 0; k < kNSum; ++k) A.w.terms[k][i] = term[k];
      A.w.tcrit[i] = tcr;
    }
  }
  w_fb += fallback;
  w_pairs += npairs;
  w_cand += cand;
  }  // bucket loop
  const int nfb = wsum(w_fb);
  const int nupd = wsum(w_upd);
  const long long pw = wsum(w_pairs);
  const bool box_bad = PER && __any_sync(kFull, w_box);
  if (lane == 0) {
    if (box_bad) atomicOr(&A.st->err, ERR_CAPACITY);
    if (nfb) atomicAdd(&A.st->n_cfallback, nfb);
    if (nupd) atomicAdd(&A.st->updates, (unsigned long long)nupd);
    atomicAdd(&A.st->pairs_force, (unsigned long long)pw);
    atomicAdd(&A.st->cand_force, (unsigned long long)w_cand);
    atomicAdd(&A.st->groups_force, (unsigned long long)w_groups);
  }
}

template <typename K> int grid_for_buckets(const sph_ctx *c, K kernel, int64_t buckets) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * kWarpsPerBlock, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t need = (buckets + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const int64_t have = (int64_t)per_sm * c->num_sms;
  return (int)(need < have ? (need > 0 ? need : 1) : have);
}

template <typename T, int CAP, bool PER, int UF>
void launch_forces_t(const ForceArgs &a, const sph_ctx *c, int64_t buckets, cudaStream_t stream) {
  k_forces<T, CAP, PER, UF><<<grid_for_buckets(c, k_forces<T, CAP, PER, UF>, buckets),
                              32 * kWarpsPerBlock, 0, stream>>>(a);
}

// The pair loop over buckets [b0, b1) (b1 < 0: to the last bucket), taken
// through the counter *ctr, which must be zero, on `stream`.
cudaError_t launch_forces_range(sph_ctx *c, int b0, int b1, unsigned *ctr, cudaStream_t stream) {
  ForceArgs a;
  a.s = c->st;
  a.w = c->w;
  a.n = c->n;
  a.cell_start = c->cell_start;
  a.cell_end = c->cell_end;
  a.p = c->kp;
  a.st = c->d_status;
  a.kick = c->fuse_kick;
  a.src = c->src;
  a.b_begin = b0;
  a.b_end = b1 < 0 ? 0x7fffffff : b1;
  a.counter = ctr;
  const int64_t buckets = (b1 < 0 ? c->kp.nbuckets : b1) - b0;
  if (c->kp.precision == SPH_FP32K) {
    const bool d4 = c->depth_f == 4;
    if (c->kp.periodic) {
      if (d4) launch_forces_t<float, 800, true, 4>(a, c, buckets, stream);
      else launch_forces_t<float, 800, true, 3>(a, c, buckets, stream);
    } else {
      if (d4) launch_forces_t<float, 800, false, 4>(a, c, buckets, stream);
      else launch_forces_t<float, 800, false, 3>(a, c, buckets, stream);
    }
  } else {
    if (c->kp.periodic) launch_forces_t<double, 256, true, kDepthForces>(a, c, buckets, stream);
    else launch_forces_t<double, 256, false, kDepthForces>(a, c, buckets, stream);
  }
  c->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_forces(sph_ctx *c) {
  cudaError_t e = cudaMemsetAsync(&c->d_status->next_bucket[1], 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return e;
  return launch_forces_range(c, 0, -1, &c->d_status->next_bucket[1], c->stream);
}

}  // namespace sphk
