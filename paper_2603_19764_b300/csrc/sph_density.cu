// sph_density.cu -- position packing and the density / smoothing-length
// solve (§2.1, Eq. 1-3).
//
// One warp owns a bucket of 32 consecutive (cell-sorted) particles, one
// particle per lane, processed group by group (sph_pair.cuh). A group stages
// every particle within 1.05 R of its bounding box (R the largest H of its
// unconverged lanes) into shared memory once; each lane then marks, in a
// private bit mask, the staged particles within 1.05 H_i of itself and walks
// only those, testing r < H_i exactly. Newton sweeps reuse the staged list
// and the masks until some H outgrows them. The density of particle i
// depends on H_i alone, so every particle's iteration runs inside the kernel
// without global synchronisation.
//
// FP64 form: absolute positions, canonical predicate r^2 = (dx dx + dy dy) +
// dz dz without fused multiply-add. FP32 form: positions relative to the
// group's reference cell, FP32 sums and Newton arithmetic, the radius
// included (stored as FP64); pairs with |r^2 - H^2| inside the guard band
// (sph_pair.cuh) are re-decided with the FP64 predicate against the exact
// square of that radius, so that neighbour counts stay exact.
#include "sph_pair.cuh"

namespace sphk {

// Position packing for the pair kernels: in the FP32 form each particle's
// position relative to the origin of its cell, with its mass; in the FP64
// form the absolute position. (The evaluation state that the predictor
// forms from the half-step values is made where it is read, in k_eos_pack.)
__global__ void __launch_bounds__(kBlock) k_pack(sph_state s, Work w, int64_t n, KParams P,
                                                int fp32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = s.x[i], y = s.y[i], z = s.z[i], m = s.m[i];
    if (fp32) {
      const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, i) : 0;
      const Grid &g = P.sys[sy].grid;
      const int c = w.cc[i];
      // the cell index as a double through FP32 (exact below 2^24), so
      // that no conversion runs on the FP64 unit
      const double ox = g.lo[0] + f2d((float)(c & 1023)) * g.L;
      const double oy = g.lo[1] + f2d((float)((c >> 10) & 1023)) * g.L;
      const double oz = g.lo[2] + f2d((float)((c >> 20) & 1023)) * g.L;
      w.pos32[i] = make_float4(d2f(x - ox), d2f(y - oy), d2f(z - oz), d2f(m));
    } else {
      w.pos64[i] = make_double4_32a(x, y, z, m);
    }
  }
}

cudaError_t launch_pack(sph_ctx *c) {
  int64_t b = (c->n + kBlock - 1) / kBlock;
  if (b > 148 * 16) b = 148 * 16;
  k_pack<<<(int)b, kBlock, 0, c->stream>>>(c->st, c->w, c->n, c->kp,
                                          c->kp.precision == SPH_FP32K);
  c->nlaunch += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- density
struct DensArgs {
  sph_state s;
  Work w;
  int64_t n;
  const int *cell_start, *cell_end;
  KParams p;
  Status *st;
  void *spill;      // per-warp overflow of the candidate lists (kSpill entries)
  int expand;       // close Newton steps by the expansion (FP32 form, full steps)
  const double *h_in;   // H before the solve (the step's read view); h is written to s.h
  int spill_warps;      // warps the overflow region has room for
};

// Candidates beyond the shared-memory list of a warp continue in a private
// global-memory region of kSpill entries (positions, indices, mask words),
// so that a list of up to CAP + kSpill candidates stays resident across the
// Newton sweeps instead of being staged again for every sweep.
constexpr int kSpill = 1024;


// FP32 form within a full step: a Newton step of at most kExpand H is
// accepted without a new evaluation of the sums when the second-order
// expansion of rho(H) about the evaluated H already meets the tolerance at
// the new H. The kernel sum is C^3 in H (the Wendland C2 kernel's (1-q)^4
// factor), so the omitted third-order term is ~1e-8 of rho, below FP32
// rounding; pairs entering or leaving the support between the two radii
// weigh (dH/H)^4. The neighbour count at the accepted H is the force pass's
// (it visits every pair within max(H_i, H_j)).
constexpr double kExpand = 3e-3;

template <typename V4> struct SpillView {
  V4 *p;
  int *i;
  unsigned (*m)[32];
};
template <typename V4>
__device__ __forceinline__ SpillView<V4> spill_view(void *base, int warp) {
  const size_t per = (size_t)kSpill * (sizeof(V4) + 2 * sizeof(int));
  char *b = (char *)base + per * warp;
  SpillView<V4> v;
  v.p = (V4 *)b;
  v.i = (int *)(b + (size_t)kSpill * sizeof(V4));
  v.m = (unsigned(*)[32])(b + (size_t)kSpill * (sizeof(V4) + sizeof(int)));
  return v;
}

template <typename T> struct PosPtr;
template <> struct PosPtr<float> {
  static __device__ __forceinline__ const float4 *get(const Work &w) { return w.pos32; }
};
template <> struct PosPtr<double> {
  static __device__ __forceinline__ const double4_32a *get(const Work &w) { return w.pos64; }
};


// Candidate list layout over a buffer of S candidates: planes in the FP32
// form (packed mask tests, bank-spread walk reads), one record per
// candidate in the FP64 form.
template <typename T> struct DList;
template <> struct DList<float> {
  template <int S> using view = ViewPlanes<S>;
  template <int S> static __device__ __forceinline__ ViewPlanes<S> at(void *p) {
    return ViewPlanes<S>{reinterpret_cast<float *>(p)};
  }
};
template <> struct DList<double> {
  template <int S> using view = ViewAoS<double4_32a>;
  template <int S> static __device__ __forceinline__ ViewAoS<double4_32a> at(void *p) {
    return ViewAoS<double4_32a>{reinterpret_cast<double4_32a *>(p)};
  }
};

// Per-lane bit masks over the staged list (mask_word's layout): candidate k
// marked when r_k^2 < R2.
// Lanes with store = false compute but keep their previous words.
template <typename T, typename LV>
__device__ __forceinline__ void build_masks(const LV &Lp, unsigned (*Lm)[32],
                                            int nl, T xi, T yi, T zi, T R2, bool store, int lane) {
  const int nw = (nl + 31) >> 5;
  for (int wd = 0; wd < nw; ++wd) {
    const int kb = wd << 5;
    const unsigned mk = mask_word(Lp, kb, min(32, nl - kb), xi, yi, zi,
                                  [R2](T) { return R2; });
    if (store) Lm[wd][lane] = mk;
  }
}

// Walk one lane's marked candidates: membership r < H_i, then the kernel
// sums of Eq. 1 (rs) and Eq. 3 (rhs) without their constant factors.
// FP32 form: membership by the FP32 r^2; a pair within the guard band gb of
// H^2 sets `near`, and density_recount then corrects the count with the
// FP64 predicate (the kernel weight of such a pair is ~(gb / H^2)^4 of a
// neighbour's, below the rounding of the sums, so only the count depends on
// the decision).
template <typename T, bool REL, bool PER, typename LV>
__device__ __forceinline__ void density_walk(const LV &Lp, const int *Li,
                                             unsigned (*Lm)[32],
                                             int nl, int lane, T xi, T yi, T zi, T invH, T H2,
                                             T gb, T H, double xi64, double yi64, double zi64,
                                             const sph_state &s, const double *blen,
                                             T &rs, T &rhs, T &rhs2, int &cnt, bool &near,
                                             int64_t n_all, unsigned *err) {
  // every lane advances through its own words: lanes do not wait for each
  // other at word boundaries
  const int nw = (nl + 31) >> 5;
  int wd = 0;
  unsigned mk = nw > 0 ? Lm[0][lane] : 0u;
  for (;;) {
    while (mk == 0u && ++wd < nw) mk = Lm[wd][lane];
    if (mk == 0u) break;
    {
      const int k = (wd << 5) + take_next(mk);
      T qx, qy, qz, qm;
      Lp.get(k, qx, qy, qz, qm);
      const T dx = xi - qx, dy = yi - qy, dz = zi - qz;
      T r2;
      bool in;
      // (Lp, Li, Lm: the shared-memory list or its global overflow; neither
      // is read through the read-only path, the kernel writes both)
      if (REL) {
        r2 = dist2(dx, dy, dz);
        in = r2 < H2;
        near = near || fabs(r2 - H2) < gb;   // rare: the count is corrected afterwards
      } else {
        r2 = (T)r2_canon((double)dx, (double)dy, (double)dz);
        in = r2 < H2;
        // a shifted image's coordinate was rounded once more than the
        // minimum image of x_i - x_j: decide the rare pair at the boundary
        // with the canonical arithmetic
        if (PER && fabs(r2 - H2) < gb) {
          const int j = (int)checked(Li[k], n_all, err);
          in = r2_canon_periodic(xi64 - s.x[j], yi64 - s.y[j], zi64 - s.z[j], blen) < (double)H2;
        }
      }
      // FP64 form: out-of-range candidates skip the (FP64) kernel terms.
      // FP32 form: every marked candidate forms them, a candidate out of
      // range with weight t = 0 (exact zeros, the sums unchanged), which
      // costs less than the branch (the marks reach only 1.005 H)
      if (!REL && !in) continue;
      const T qq = root0(r2) * invH;
      const T t = in ? tmax(T(1) - qq, T(0)) : T(0);
      const T mW = qm * t * t * t;
      rs += mW * t * (T(1) + T(4) * qq);
      rhs += mW * (T(-3) + qq * (T(-9) + T(32) * qq));
      if (REL)   // H^5 d2W/dH2 / cW = (1-q)^2 (12 + 24q - 264q^2 + 288q^3)
        rhs2 += qm * t * t * (T(12) + qq * (T(24) + qq * (T(-264) + T(288) * qq)));
      // the particle itself is among the lane's candidates and in range
      // (r = 0 exactly, see rel_coord): counted here, taken off once by
      // the caller
      cnt += in ? 1 : 0;
    }
  }
}

// FP32 form, after density_walk set `near`: walk the same marks again and
// move every pair within the guard band from the FP32 decision to the FP64
// predicate's, so that the count is that of the canonical predicate.
// Returns the change of the count.
template <bool PER, typename LV>
__device__ __forceinline__ int density_recount(const LV &Lp, const int *Li, unsigned (*Lm)[32],
                                               int nl, int lane, float xi, float yi, float zi,
                                               float H2, float gb, float H, double xi64,
                                               double yi64, double zi64, const double *sx,
                                               const double *sy, const double *sz,
                                               const double *blen, int64_t n_all,
                                               unsigned *err) {
  int cnt = 0;
  const int nw = (nl + 31) >> 5;
  for (int wd = 0; wd < nw; ++wd) {
    unsigned mk = Lm[wd][lane];
    while (mk) {
      const int k = (wd << 5) + take_next(mk);
      float qx, qy, qz, qm;
      Lp.get(k, qx, qy, qz, qm);
      const float r2 = dist2(xi - qx, yi - qy, zi - qz);
      if (fabs(r2 - H2) < gb) {
        const bool in = fp64_within<PER>(sx, sy, sz, xi64, yi64, zi64,
                                         (int)checked(Li[k], n_all, err), blen, (double)H);
        cnt += (in ? 1 : 0) - (r2 < H2 ? 1 : 0);
      }
    }
  }
  return cnt;
}

// Both parts of a list (shared memory and its overflow), out of line: the
// walks stay free of the FP64 predicate and its registers.
template <bool PER, int S1, int S2>
__device__ __noinline__ int recount_lists(ViewPlanes<S1> L1, const int *I1, unsigned (*M1)[32],
                                          int n1, ViewPlanes<S2> L2, const int *I2,
                                          unsigned (*M2)[32], int n2, int lane, float xi,
                                          float yi, float zi, float H2, float gb, float H,
                                          double xi64, double yi64, double zi64,
                                          const double *sx, const double *sy, const double *sz,
                                          const double *blen, int64_t n_all, unsigned *err) {
  return density_recount<PER>(L1, I1, M1, n1, lane, xi, yi, zi, H2, gb, H, xi64, yi64, zi64, sx,
                              sy, sz, blen, n_all, err) +
         density_recount<PER>(L2, I2, M2, n2, lane, xi, yi, zi, H2, gb, H, xi64, yi64, zi64, sx,
                              sy, sz, blen, n_all, err);
}

// UD: staging depth, the chunks of 32 stream positions located and loaded
// at once (kDepths; the lists do not depend on it)
template <typename T, int CAP, bool PER, int UD>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 4) k_density(DensArgs A) {
  constexpr bool REL = std::is_same<T, float>::value;
  using V = V4T<T>;
  using V4 = typename V::type;
  __shared__ V4 s_pos[kWarpsPerBlock][CAP];
  __shared__ int s_idx[kWarpsPerBlock][CAP];
  __shared__ unsigned s_mask[kWarpsPerBlock][CAP / 32][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the list in this warp's shared buffer, and its overflow in global memory
  const auto Lp = DList<T>::template at<CAP>(s_pos[wib]);
  int *Li = s_idx[wib];
  unsigned(*Lm)[32] = s_mask[wib];
  const SpillView<V4> Sv0 =
      spill_view<V4>(A.spill, (int)checked(blockIdx.x * kWarpsPerBlock + wib, A.spill_warps,
                                           &A.st->err));
  const auto Sp = DList<T>::template at<kSpill>(Sv0.p);
  struct {
    int *i;
    unsigned (*m)[32];
  } const Sv = {Sv0.i, Sv0.m};
  constexpr int TCAP = CAP + kSpill;
  // persistent warps: each takes the next bucket of 32 particles
  const int n_act = A.p.act ? A.st->n_active : 0;
  const int nbuckets = bucket_count(A.p, n_act);
  long long w_pairs = 0, w_cand = 0;
  int w_sw = 0, w_nu = 0, w_ncap = 0, w_groups = 0, w_exp = 0;
  long long w_swt = 0;
  unsigned w_bad = 0, w_box = 0;
  // a periodic box must be wider than twice every search radius
  const T box_min = PER ? (T)fmin(fmin(A.p.box_len[0], A.p.box_len[1]), A.p.box_len[2]) : T(0);
  for (;;) {
  unsigned bk = 0;
  if (lane == 0) bk = atomicAdd(&A.st->next_bucket[0], 1u);
  bk = __shfl_sync(kFull, bk, 0);
  if ((int)bk >= nbuckets) break;
  // the bucket's system and its sorted range
  const BucketLane bl = bucket_lane(A.p, n_act, bk, lane, A.n, &A.st->err);
  const int sy = bl.sy;
  const SysRec &R = A.p.sys[sy];
  const int64_t i = bl.i;
  const bool valid = bl.valid;
  // with hierarchical steps only particles whose step ends are solved; the
  // others keep H, rho, Omega and their count
  const bool solve = valid && rung_active(A.p, i);
  const int64_t ic = bl.ic;
  const V4 *pos = PosPtr<T>::get(A.w);

  const Grid g = R.grid;
  const T Lt = grid_L<T>(g), invL = grid_invL<T>(g);
  const int cc = A.w.cc[ic];
  const int cx = cc & 1023, cy = (cc >> 10) & 1023, cz = (cc >> 20) & 1023;
  const V4 p = V::ld(pos, ic);
  const T mi = p.w;
  const MatT<T> &Mt = mat_t<T>(A.p, A.s.mat[ic]);
  const T target = (T)A.p.n_ngb * mi;
  const T tol = pconst<T>(A.p.h_tol, A.p.h_tol_f);
  // the Newton state is kept in T: the FP32 form's radius carries 24 bits,
  // far below h_tol, and its FP64 predicate uses the exact square of it.
  // Cap: h_cap_factor times the lattice radius (3 n_ngb m / (4 pi rho0))^(1/3)
  const T Hcap = Mt.hcap_f * cbrt(Mt.hcap_k * mi);
  // starting radius: the previous H, or the proposal of the learned form
  // (one with 0 < H <= inf, tested on its bits)
  T H = to_t<T>(A.h_in[ic]);
  if (A.p.h_guess) {
    const double hg = A.p.h_guess[ic];
    const long long hb = __double_as_longlong(hg);
    if (hb > 0 && hb <= 0x7ff0000000000000LL) H = to_t<T>(hg);
  }
  H = tmin(H, Hcap);
  const double xi64 = A.s.x[ic], yi64 = A.s.y[ic], zi64 = A.s.z[ic];
  // Newton state: 0 running, 1 converged, 2 capped, 3 gave up, 4 idle lane
  int state = solve ? 0 : 4;
  T lo = T(0), hi = T(INFINITY), H_o = H;
  T rho_o = T(0), om_o = T(1);
  int cnt_o = 0, sweeps_o = 0;
  long long pairs = 0, cand = 0;

  unsigned todo = __ballot_sync(kFull, solve);
  while (todo) {
    const Group G = next_group(todo, cx, cy, cz, A.p.span_d);
    ++w_groups;
    const T xi = REL ? rel_coord(p.x, cx - G.rx, Lt) : p.x;
    const T yi = REL ? rel_coord(p.y, cy - G.ry, Lt) : p.y;
    const T zi = REL ? rel_coord(p.z, cz - G.rz, Lt) : p.z;
    bool complete = false;   // the list holds every particle within Rl of the box
    T Rl = T(0), Hm = T(0);  // list radius; this lane's mask radius
    int nl = 0;

    for (int sweep = 1; sweep <= A.p.max_sweeps; ++sweep) {
      const bool act = G.member && state == 0;
      if (!__any_sync(kFull, act)) break;
      const T Ht = H;
      const T invHt = T(1) / Ht;
      const T H2 = REL ? Ht * Ht : (T)__dmul_rn((double)Ht, (double)Ht);
      // FP64 form in a periodic box: the band of the shifted images' extra
      // rounding (far below the FP32 band)
      const T gb = REL ? guard_band(Ht, Lt) : T(1e-12) * Ht * tmax(Ht, box_min);
      // smallest mask radius: Hq^2 > H^2 + gb, so that no pair with r < H
      // by the FP64 predicate falls outside the mask or the list
      const T Hq = Ht * T(1.0001) + T(1e-5) * tmax(Ht, Lt);
      const T Rneed = wmax(act ? Hq : T(0));
      T rs = T(0), rhs = T(0), rhs2 = T(0);
      int cnt = 0;
      const bool resident = complete && Rneed <= Rl;
      if (!resident) {
        Rl = Rneed * T(1.02);
        if (PER && !(T(2) * Rl < box_min)) w_box = 1u;
        const Box<T> bx = group_box(act, xi, yi, zi);
        // the cells within Rl of the box plus the skin (a hierarchical substep
        // that kept the last order: the particles moved since that sort)
        auto sg = make_stager_for<T, REL, PER>(bx, Rl + sys_skin<T>(R), g, invL, A.p, G.rx,
                                               G.ry, G.rz);
        Hm = T(0);
        complete = false;
        for (int seg = 0;; ++seg) {
          nl = stage_list<UD, true, T, REL>(
              sg, g, A.cell_start, A.cell_end, Lt, A.p, G.rx, G.ry, G.rz, 0, TCAP, A.n,
              &A.st->err,
              [&](bool ok, int j) { return ok ? V::ld(pos, j) : V::make(0, 0, 0, 0); },
              [&](bool ok, const V4 &q, T ox, T oy, T oz, T &xj, T &yj, T &zj) {
                xj = add_rn(q.x, ox);
                yj = add_rn(q.y, oy);
                zj = add_rn(q.z, oz);
                return ok &&
                       box_d2(xj, yj, zj, bx.x0, bx.x1, bx.y0, bx.y1, bx.z0, bx.z1) < Rl * Rl;
              },
              [&](int at, T xj, T yj, T zj, const V4 &q, int j) {
                if (at < CAP) {
                  Lp.put(at, xj, yj, zj, q.w);
                  Li[at] = j;
                } else {
                  Sp.put(at - CAP, xj, yj, zj, q.w);
                  Sv.i[at - CAP] = j;
                }
              });
          cand += nl;
          if (seg == 0 && stager_finished(sg)) {
            complete = true;
            break;
          }
          // list longer than both buffers: evaluate this segment exactly
          const int n1 = min(nl, CAP), n2 = nl - n1;
          __syncwarp();
          build_masks<T>(Lp, Lm, n1, xi, yi, zi, Hq * Hq, act, lane);
          build_masks<T>(Sp, Sv.m, n2, xi, yi, zi, Hq * Hq, act, lane);
          __syncwarp();
          if (act) {
            bool near = false;
            density_walk<T, REL, PER>(Lp, Li, Lm, n1, lane, xi, yi, zi, invHt, H2, gb, Ht, xi64,
                                          yi64, zi64, A.s, A.p.box_len, rs, rhs, rhs2,
                                          cnt, near, A.n, &A.st->err);
            density_walk<T, REL, PER>(Sp, Sv.i, Sv.m, n2, lane, xi, yi, zi, invHt, H2, gb, Ht,
                                          xi64, yi64, zi64, A.s, A.p.box_len, rs, rhs,
                                          rhs2, cnt, near, A.n, &A.st->err);
            if constexpr (REL)
              if (near)   // rare
                cnt += recount_lists<PER>(Lp, Li, Lm, n1, Sp, Sv.i, Sv.m, n2, lane, xi, yi, zi, H2,
                                          gb, Ht, xi64, yi64, zi64, A.s.x, A.s.y, A.s.z,
                                          A.p.box_len, A.n, &A.st->err);
          }
          __syncwarp();
          if (stager_finished(sg)) break;
        }
      }
      if (complete) {
        // resident list: refresh the masks of lanes whose H outgrew them
        const bool rebuild = act && !(Hm >= Hq);
        const int n1 = min(nl, CAP), n2 = nl - n1;
        if (__any_sync(kFull, rebuild)) {
          const T Hn = rebuild ? tmax(Ht * T(1.005), Hq) : Hm;
          __syncwarp();
          build_masks<T>(Lp, Lm, n1, xi, yi, zi, Hn * Hn, rebuild, lane);
          build_masks<T>(Sp, Sv.m, n2, xi, yi, zi, Hn * Hn, rebuild, lane);
          __syncwarp();
          Hm = Hn;
        }
        if (act) {
          bool near = false;
          density_walk<T, REL, PER>(Lp, Li, Lm, n1, lane, xi, yi, zi, invHt, H2, gb, Ht, xi64,
                                        yi64, zi64, A.s, A.p.box_len, rs, rhs, rhs2,
                                        cnt, near, A.n, &A.st->err);
          density_walk<T, REL, PER>(Sp, Sv.i, Sv.m, n2, lane, xi, yi, zi, invHt, H2, gb, Ht,
                                        xi64, yi64, zi64, A.s, A.p.box_len, rs, rhs,
                                        rhs2, cnt, near, A.n, &A.st->err);
          if constexpr (REL)
            if (near)   // rare
              cnt += recount_lists<PER>(Lp, Li, Lm, n1, Sp, Sv.i, Sv.m, n2, lane, xi, yi, zi, H2,
                                        gb, Ht, xi64, yi64, zi64, A.s.x, A.s.y, A.s.z,
                                        A.p.box_len, A.n, &A.st->err);
        }
      }

      if (act) {
        // Eq. 1 and Eq. 3 with the kernel constants applied once; the
        // residual is relative to the target kernel mass n_ngb m_i
        const T ih = invHt;
        const T ih3 = ih * ih * ih;
        const T rho = T(cW) * ih3 * rs;
        const T rhoH = T(cW) * ih3 * ih * rhs;
        const T om = T(1) + Ht / (T(3) * rho) * rhoH;
        const T gq = T(4.0 * kPi / 3.0) * Ht * Ht * Ht * rho / target - T(1);
        rho_o = rho;
        om_o = om;
        cnt_o = cnt - 1;   // the walk counted the particle itself
        H_o = H;
        sweeps_o = sweep;
        pairs += cnt - 1;
        if (fabs(gq) <= tol) {
          state = 1;
        } else if (gq < T(0) && H >= Hcap) {
          state = 2;
          om_o = T(1);   // Eq. 3 tends to 0 without neighbours (0 for a lone particle)
        } else {
          if (gq < T(0)) lo = H;
          else hi = H;
          const T gp = T(4.0 * kPi) * Ht * Ht * rho * om / target;
          T Hn = gp > T(0) ? H - gq / gp : (gq < T(0) ? T(1.25) * H : T(0.75) * H);
          if (!(Hn >= T(0.75) * H)) Hn = T(0.75) * H;
          if (!(Hn <= T(1.25) * H)) Hn = T(1.25) * H;
          if (hi < T(INFINITY) && (Hn <= lo || Hn >= hi)) Hn = T(0.5) * (lo + hi);
          if (Hn > Hcap) Hn = Hcap;
          if (REL && A.expand && fabs(Hn - H) <= T(kExpand) * H) {
            // rho, d rho / dH at Hn from the second-order expansion about H
            const T d = Hn - H;
            const T rho2 = T(cW) * ih3 * ih * ih * rhs2;
            const T r1 = rho + d * (rhoH + T(0.5) * rho2 * d);
            const T H1 = Hn;
            const T gq1 = T(4.0 * kPi / 3.0) * H1 * H1 * H1 * r1 / target - T(1);
            const T om1 = T(1) + H1 / (T(3) * r1) * (rhoH + rho2 * d);
            // the estimate's error in d rho / dH reaches Omega scaled by
            // |1 - Omega| / Omega, and the forces carry 1 / Omega: a
            // particle with few neighbours (small Omega) is closed only on
            // an exact sum
            if (fabs(gq1) <= tol && r1 > T(0) && om1 >= T(0.5)) {
              rho_o = r1;
              om_o = om1;
              H_o = Hn;
              state = 1;
              ++w_exp;
            }
          }
          H = Hn;
        }
      }
    }
    if (G.member && state == 0) state = 3;
  }

  if (solve) {
    A.s.h[i] = from_t(H_o);
    A.s.rho[i] = from_t(rho_o);
    A.s.omega[i] = from_t(om_o);
    A.s.nngb[i] = cnt_o;
  }
  w_sw = max(w_sw, solve ? sweeps_o : 0);
  w_swt += solve ? sweeps_o : 0;
  w_nu += state == 3;
  w_ncap += state == 2;
  w_bad |= (solve && !(isfinite(rho_o) && isfinite(om_o) && rho_o > T(0))) ? 1u : 0u;
  {
    // every particle's radius bounds the force pass's search, solved or not
    // (the maximum of the order-preserving encodings), widened by the
    // staging skin (0 after a sort)
    const unsigned long long hb =
        wmax(enc_d(valid ? (solve ? from_t(H_o) : A.h_in[i]) + R.skin : 0.0));
    if (lane == 0) atomicMax(&A.p.sys[sy].hmax2_enc, hb);
  }
  w_pairs += pairs;
  w_cand += cand;
  }  // bucket loop
  const int sw = wmax(w_sw);
  const int nu = wsum(w_nu);
  const int ncap = wsum(w_ncap);
  const unsigned nbad = __ballot_sync(kFull, w_bad != 0u);
  const long long pw = wsum(w_pairs);
  const long long swt = wsum(w_swt);
  const int nexp = wsum(w_exp);
  if (lane == 0) {
    atomicMax(&A.st->max_sweeps, sw);
    if (nexp) atomicAdd(&A.st->n_expanded, nexp);
    atomicAdd(&A.st->sweeps_total, (unsigned long long)swt);
    if (nu) {
      atomicAdd(&A.st->n_unconv, nu);
      atomicOr(&A.st->err, ERR_NOCONV);
    }
    if (ncap) atomicAdd(&A.st->n_capped, ncap);
    if (nbad) atomicOr(&A.st->err, ERR_NONFINITE);
    if (PER && __any_sync(kFull, w_box)) atomicOr(&A.st->err, ERR_CAPACITY);
    atomicAdd(&A.st->pairs_density, (unsigned long long)pw);
    atomicAdd(&A.st->cand_density, (unsigned long long)w_cand);
    atomicAdd(&A.st->groups_density, (unsigned long long)w_groups);
  }
}

template <typename T, int CAP, bool PER, int UD>
void launch_density_t(sph_ctx *c, const DensArgs &a) {
  k_density<T, CAP, PER, UD><<<resident_grid(c, k_density<T, CAP, PER, UD>),
                               32 * kWarpsPerBlock, 0, c->stream>>>(a);
}

cudaError_t launch_density(sph_ctx *c, int expand) {
  DensArgs a;
  a.expand = expand;
  a.s = c->st;
  a.w = c->w;
  a.n = c->n;
  a.cell_start = c->cell_start;
  a.cell_end = c->cell_end;
  a.p = c->kp;
  a.st = c->d_status;
  a.spill = c->dens_spill;
  a.h_in = c->src.h;
  a.spill_warps = c->spill_warps;
  cudaError_t e = cudaMemsetAsync(&c->d_status->next_bucket[0], 0, sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return e;
  if (c->kp.precision == SPH_FP32K) {
    const bool d4 = c->depth_d == 4;
    if (c->kp.periodic) {
      if (d4) launch_density_t<float, 576, true, 4>(c, a);
      else launch_density_t<float, 576, true, 3>(c, a);
    } else {
      if (d4) launch_density_t<float, 576, false, 4>(c, a);
      else launch_density_t<float, 576, false, 3>(c, a);
    }
  } else {
    if (c->kp.periodic) launch_density_t<double, 256, true, kDepthDensity>(c, a);
    else launch_density_t<double, 256, false, kDepthDensity>(c, a);
  }
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace sphk

namespace sphk {

// Overflow region of the density lists: one kSpill-entry region per warp
// that can be resident, at most one warp per bucket.
cudaError_t alloc_density_spill(sph_ctx *c) {
  // sized for the variant with the most resident blocks (closed or
  // periodic box), so that every launched warp owns a region
  int per_sm = 0;
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
    int k = 0;
    const bool per = v & 1, d4 = v & 2;
    if (c->kp.precision == SPH_FP32K)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &k,
          per ? (d4 ? k_density<float, 576, true, 4> : k_density<float, 576, true, 3>)
              : (d4 ? k_density<float, 576, false, 4> : k_density<float, 576, false, 3>),
          32 * kWarpsPerBlock, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &k, per ? k_density<double, 256, true, kDepthDensity>
                  : k_density<double, 256, false, kDepthDensity>,
          32 * kWarpsPerBlock, 0);
    per_sm = k > per_sm ? k : per_sm;
  }
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t need = ((int64_t)c->kp.nbuckets + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int64_t blocks = (int64_t)per_sm * c->num_sms;
  if (blocks > need) blocks = need;
  const size_t v4 = c->kp.precision == SPH_FP32K ? sizeof(float4) : sizeof(double4_32a);
  const size_t per = (size_t)kSpill * (v4 + 2 * sizeof(int));
  c->spill_warps = (int)(blocks * kWarpsPerBlock);
  return cudaMalloc(&c->dens_spill, per * (size_t)(blocks * kWarpsPerBlock));
}

}  // namespace sphk
