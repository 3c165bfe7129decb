// sph_mlp.cu -- the smoothing-length network of the learned form: its
// device object, inference, loss and gradient by back-propagation on the
// tensor cores, Adam, feature normalisation, and the per-step kernel that
// records training samples and proposes each particle's next support radius.
//
// The paper's smoothing-length solve (§2.1, Eq. 2-3) starts from the
// previous radius; the network moves only that starting point, and the
// exact Newton solve that follows decides H and the neighbour count.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sph_internal.cuh"
#include "sph_mlp.cuh"

using namespace sphk;
using namespace sphk::mlp;

struct sph_mlp {
  cudaStream_t stream;
  float *theta, *mom, *vel;      // FP32 master parameters and Adam moments
  float *norm;                   // NNORM
  __nv_bfloat16 *wb;             // w1b | w2b | w2tb
  float *grad;                   // reduced gradient (NPARAM) + loss + count
  float *partials;               // per-block gradient partials
  double *nsum;                  // normalisation partial sums
  float *h_out;                  // pinned: loss, count
  int adam_t;
  char err[256];
};

namespace {

constexpr int kThreads = 128;            // 4 warps, 64 samples per block pass
constexpr int kWarps = kThreads / 32;
constexpr int kGradBlocks = 2 * 148;     // training grid
constexpr int kPart = NPARAM + 2;        // gradient, loss, sample count

Net net_of(const sph_mlp *m) {
  Net n;
  if (!m) {
    memset(&n, 0, sizeof(n));
    return n;
  }
  n.theta = m->theta;
  n.norm = m->norm;
  n.w1b = m->wb;
  n.w2b = m->wb + NH * LD1;
  n.w2tb = m->wb + NH * LD1 + NH * LD2;
  return n;
}

// bf16 operand copies of W1 and W2 from the master parameters.
__global__ void k_refresh_bf16(const float *theta, __nv_bfloat16 *wb) {
  __nv_bfloat16 *w1 = wb, *w2 = wb + NH * LD1, *w2t = wb + NH * LD1 + NH * LD2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NH * LD2; k += gridDim.x * blockDim.x) {
    const int r = k / LD2, c = k % LD2;
    w2[k] = __float2bfloat16_rn(c < NH ? theta[OFF_W2 + r * NH + c] : 0.f);
    w2t[k] = __float2bfloat16_rn(c < NH ? theta[OFF_W2 + c * NH + r] : 0.f);
    if (k < NH * LD1) {
      const int r1 = k / LD1, c1 = k % LD1;
      w1[k] = __float2bfloat16_rn(c1 < NIN ? theta[OFF_W1 + r1 * NIN + c1] : 0.f);
    }
  }
}

// Standardised, bf16-rounded features of sample rows into a warp's
// [16][LD1] tile (columns NIN.. stay zero), and the standardised targets.
// Training (y given): a row with any non-finite feature or target is
// masked, its features staged as zeros so that it adds nothing.
__device__ __forceinline__ void stage_rows(const Smem &S, __nv_bfloat16 *xs, const float *X,
                                           const float *y, const int64_t *idx, int64_t base,
                                           int64_t m, float *yh, int *ok) {
  const int lane = threadIdx.x & 31;
  if (lane < 16) {
    const int64_t s = base + lane;
    float v = 0.f;
    int good = 0;
    if (s < m) {
      const int64_t q = idx ? idx[s] : s;
      good = 1;
      for (int f = 0; f < NIN; ++f) good &= isfinite(X[q * NIN + f]) ? 1 : 0;
      if (y) {
        const float yv = y[q];
        good &= isfinite(yv) ? 1 : 0;
        v = good ? (yv - S.ymu) / S.ysd : 0.f;
      }
    }
    yh[lane] = v;
    ok[lane] = good;
  }
  __syncwarp();
  for (int e = lane; e < 16 * NIN; e += 32) {
    const int r = e / NIN, f = e % NIN;
    const int64_t s = base + r;
    float v = 0.f;
    if (s < m && (ok[r] || !y)) {
      const int64_t q = idx ? idx[s] : s;
      v = (X[q * NIN + f] - S.mu[f]) * S.isd[f];
    }
    xs[r * LD1 + f] = __float2bfloat16_rn(v);
  }
  __syncwarp();
}

// ------------------------------------------------------------- inference
__global__ void __launch_bounds__(kThreads) k_forward(Net N, const float *X, int64_t m,
                                                      float *pred) {
  __shared__ __align__(16) Smem S;
  __shared__ __align__(16) __nv_bfloat16 xs[kWarps][16 * LD1];
  __shared__ float yh[kWarps][16];
  __shared__ int ok[kWarps][16];
  load_net(S, N, false);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = lane; e < 16 * LD1; e += 32) xs[w][e] = __float2bfloat16_rn(0.f);
  __syncthreads();
  const int64_t ntiles = (m + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * kWarps + w; tile < ntiles;
       tile += (int64_t)gridDim.x * kWarps) {
    stage_rows(S, xs[w], X, nullptr, nullptr, tile * 16, m, yh[w], ok[w]);
    uint32_t ax[4];
    load_a(xs[w], LD1, 0, 0, ax);
    Tile T;
    forward_tile(S, ax, T);
    const int g = lane >> 2;
    if ((lane & 3) == 0) {
      const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
      if (r0 < m) pred[r0] = S.ymu + S.ysd * T.out[0];
      if (r1 < m) pred[r1] = S.ymu + S.ysd * T.out[1];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------- loss + gradient
// Per block: passes over groups of 64 samples (16 per warp). Forward in
// registers, back-propagation of the output error through the layers, and
// the weight gradients dW2 = d2^T a1 and dW1 = d1^T x as tensor-core
// products over the block's 64 samples, each warp owning 16 rows of both.
// Samples with a non-finite target carry no weight. Each block writes its
// partial gradient; k_grad_final adds them in block order.
struct GradSmem {
  __nv_bfloat16 xs[kWarps][16 * LD1];
  __nv_bfloat16 d2T[NH * LD2];     // [unit o][sample s]
  __nv_bfloat16 a1T[NH * LD2];     // [unit i][sample s]
  __nv_bfloat16 d1T[NH * LD2];
  __nv_bfloat16 xT[8 * LD2];       // [feature][sample], rows NIN.. zero
  float yh[kWarps][16];
  int ok[kWarps][16];
  float red[kWarps][3][NH];        // per-warp column sums: b1, b2, W3
  float sc[kWarps][3];             // per-warp b3, loss, count
};

constexpr size_t kSmemOff = (sizeof(Smem) + 127) / 128 * 128;
constexpr size_t kGradSmem = kSmemOff + sizeof(GradSmem);

__global__ void __launch_bounds__(kThreads) k_loss_grad(Net N, const float *X, const float *y,
                                                        const int64_t *idx, int64_t m,
                                                        float *partials) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(smem_raw);
  GradSmem &G = *reinterpret_cast<GradSmem *>(smem_raw + kSmemOff);
  load_net(S, N, true);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int e = lane; e < 16 * LD1; e += 32) G.xs[w][e] = __float2bfloat16_rn(0.f);
  for (int e = threadIdx.x; e < 8 * LD2; e += kThreads) G.xT[e] = __float2bfloat16_rn(0.f);
  __syncthreads();

  // persistent accumulators
  float gw2[8][4], gw1[4] = {0.f, 0.f, 0.f, 0.f};
  float gb1[16], gb2[16], gw3[16];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int j = 0; j < 4; ++j) gw2[nt][j] = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) gb1[q] = gb2[q] = gw3[q] = 0.f;
  float gb3 = 0.f, loss = 0.f, cnt = 0.f;

  const int64_t ngroups = (m + 63) / 64;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t base = grp * 64 + 16 * w;
    stage_rows(S, G.xs[w], X, y, idx, base, m, G.yh[w], G.ok[w]);
    uint32_t ax[4];
    load_a(G.xs[w], LD1, 0, 0, ax);
    Tile T;
    forward_tile(S, ax, T);
    // output error of rows g and g + 8 (zero for masked rows)
    const float e0 = G.ok[w][g] ? T.out[0] - G.yh[w][g] : 0.f;
    const float e1 = G.ok[w][g + 8] ? T.out[1] - G.yh[w][g + 8] : 0.f;
    if (t == 0) {
      loss += e0 * e0 + e1 * e1;
      gb3 += e0 + e1;
      cnt += (float)(G.ok[w][g] + G.ok[w][g + 8]);
    }
    float d2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = 8 * nt + 2 * t;
      gw3[2 * nt] += T.a2[nt][0] * e0 + T.a2[nt][2] * e1;
      gw3[2 * nt + 1] += T.a2[nt][1] * e0 + T.a2[nt][3] * e1;
      d2[nt][0] = e0 * S.w3[col] * (1.f - T.a2[nt][0] * T.a2[nt][0]);
      d2[nt][1] = e0 * S.w3[col + 1] * (1.f - T.a2[nt][1] * T.a2[nt][1]);
      d2[nt][2] = e1 * S.w3[col] * (1.f - T.a2[nt][2] * T.a2[nt][2]);
      d2[nt][3] = e1 * S.w3[col + 1] * (1.f - T.a2[nt][3] * T.a2[nt][3]);
      gb2[2 * nt] += d2[nt][0] + d2[nt][2];
      gb2[2 * nt + 1] += d2[nt][1] + d2[nt][3];
    }
    uint32_t d2f[4][4];
    to_a(d2, d2f);
    // error at the first layer: (d2 W2) * (1 - a1^2)
    float d1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        uint32_t b0, b1;
        load_b(S.w2t, LD2, 8 * nt, 16 * kt, b0, b1);
        mma16816(c, d2f[kt], b0, b1);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) d1[nt][j] = c[j] * (1.f - T.a1[nt][j] * T.a1[nt][j]);
      gb1[2 * nt] += d1[nt][0] + d1[nt][2];
      gb1[2 * nt + 1] += d1[nt][1] + d1[nt][3];
    }
    // stage the block's 64 samples transposed for the weight products
    const int s0 = 16 * w + g;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = 8 * nt + 2 * t + (j & 1), s = s0 + (j >> 1) * 8;
        G.d2T[col * LD2 + s] = __float2bfloat16_rn(d2[nt][j]);
        G.a1T[col * LD2 + s] = __float2bfloat16_rn(T.a1[nt][j]);
        G.d1T[col * LD2 + s] = __float2bfloat16_rn(d1[nt][j]);
      }
    for (int e = lane; e < 16 * NIN; e += 32) {
      const int r = e / NIN, f = e % NIN;
      G.xT[f * LD2 + 16 * w + r] = G.xs[w][r * LD1 + f];
    }
    __syncthreads();
    // dW2 rows 16w..16w+15 and dW1 rows likewise, over the 64 samples
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      uint32_t a[4], b0, b1;
      load_a(G.d2T, LD2, 16 * w, 16 * kt, a);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        load_b(G.a1T, LD2, 8 * nt, 16 * kt, b0, b1);
        mma16816(gw2[nt], a, b0, b1);
      }
      load_a(G.d1T, LD2, 16 * w, 16 * kt, a);
      load_b(G.xT, LD2, 0, 16 * kt, b0, b1);
      mma16816(gw1, a, b0, b1);
    }
    __syncthreads();
  }

  // ---- block partial: column sums over the row groups, then the warps
#pragma unroll
  for (int q = 0; q < 16; ++q) {
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
      gb1[q] += __shfl_xor_sync(0xffffffffu, gb1[q], off);
      gb2[q] += __shfl_xor_sync(0xffffffffu, gb2[q], off);
      gw3[q] += __shfl_xor_sync(0xffffffffu, gw3[q], off);
    }
  }
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int col = 8 * nt + 2 * t + j;
        G.red[w][0][col] = gb1[2 * nt + j];
        G.red[w][1][col] = gb2[2 * nt + j];
        G.red[w][2][col] = gw3[2 * nt + j];
      }
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    gb3 += __shfl_xor_sync(0xffffffffu, gb3, off);
    loss += __shfl_xor_sync(0xffffffffu, loss, off);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  }
  if (lane == 0) {
    G.sc[w][0] = gb3;
    G.sc[w][1] = loss;
    G.sc[w][2] = cnt;
  }
  float *P = partials + (size_t)blockIdx.x * kPart;
  // W2 and W1 rows owned by this warp
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int o = 16 * w + g + (j >> 1) * 8, i = 8 * nt + 2 * t + (j & 1);
      P[OFF_W2 + o * NH + i] = gw2[nt][j];
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = 16 * w + g + (j >> 1) * 8, f = 2 * t + (j & 1);
    if (f < NIN) P[OFF_W1 + o * NIN + f] = gw1[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < NH; col += kThreads) {
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int q = 0; q < kWarps; ++q) {
      s1 += G.red[q][0][col];
      s2 += G.red[q][1][col];
      s3 += G.red[q][2][col];
    }
    P[OFF_B1 + col] = s1;
    P[OFF_B2 + col] = s2;
    P[OFF_W3 + col] = s3;
  }
  if (threadIdx.x == 0) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int q = 0; q < kWarps; ++q) {
      s0 += G.sc[q][0];
      s1 += G.sc[q][1];
      s2 += G.sc[q][2];
    }
    P[OFF_B3] = s0;
    P[NPARAM] = s1;
    P[NPARAM + 1] = s2;
  }
}

// Sum of the block partials in block order; the gradient and the loss are
// divided by the number of weighted samples (loss = 1/(2m) sum e^2).
__global__ void k_grad_final(const float *partials, int nblocks, float *grad) {
  __shared__ float inv_m;
  if (threadIdx.x == 0) {
    float c = 0.f;
    for (int b = 0; b < nblocks; ++b) c += partials[(size_t)b * kPart + NPARAM + 1];
    inv_m = c > 0.f ? 1.f / c : 0.f;
    grad[NPARAM + 1] = c;
  }
  __syncthreads();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= NPARAM; k += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * kPart + k];
    grad[k] = k < NPARAM ? s * inv_m : 0.5f * s * inv_m;
  }
}

// One Adam update (Kingma & Ba 2015, Algorithm 1), then the bf16 copies.
__global__ void k_adam(float *theta, float *mom, float *vel, const float *grad, float lr,
                       float beta1, float beta2, float eps, float c1, float c2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
    const float gk = grad[k];
    const float mk = beta1 * mom[k] + (1.f - beta1) * gk;
    const float vk = beta2 * vel[k] + (1.f - beta2) * gk * gk;
    mom[k] = mk;
    vel[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  }
}

// Normalisation: FP64 sums of each feature, its square, the target and its
// square over the samples with a finite target, per block; then the means
// and standard deviations (floored) in block order.
constexpr int kNormCols = 2 * (NIN + 1) + 1;
__global__ void __launch_bounds__(256) k_norm_partials(const float *X, const float *y, int64_t m,
                                                       double *part) {
  double acc[kNormCols];
#pragma unroll
  for (int k = 0; k < kNormCols; ++k) acc[k] = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < m;
       s += (int64_t)gridDim.x * blockDim.x) {
    const float yv = y[s];
    if (!isfinite(yv)) continue;
#pragma unroll
    for (int f = 0; f < NIN; ++f) {
      const double v = X[s * NIN + f];
      acc[2 * f] += v;
      acc[2 * f + 1] += v * v;
    }
    acc[2 * NIN] += yv;
    acc[2 * NIN + 1] += (double)yv * yv;
    acc[2 * NIN + 2] += 1.0;
  }
  __shared__ double red[kNormCols][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNormCols; ++k) {
    double v = wsum(acc[k]);
    if (lane == 0) red[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNormCols) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[threadIdx.x][q];
    part[(size_t)blockIdx.x * kNormCols + threadIdx.x] = v;
  }
}

__global__ void k_norm_final(const double *part, int nblocks, float *norm, float floor_sd) {
  if (threadIdx.x != 0) return;
  double s[kNormCols];
  for (int k = 0; k < kNormCols; ++k) {
    s[k] = 0.0;
    for (int b = 0; b < nblocks; ++b) s[k] += part[(size_t)b * kNormCols + k];
  }
  const double n = s[2 * NIN + 2] > 0.0 ? s[2 * NIN + 2] : 1.0;
  for (int f = 0; f <= NIN; ++f) {
    const double mu = s[2 * f] / n;
    const double var = fmax(s[2 * f + 1] / n - mu * mu, 0.0);
    const float sd = fmaxf((float)sqrt(var), floor_sd);
    if (f < NIN) {
      norm[f] = (float)mu;
      norm[NIN + f] = sd;
    } else {
      norm[2 * NIN] = (float)mu;
      norm[2 * NIN + 1] = sd;
    }
  }
}

sph_status mfail(sph_mlp *m, const char *what, cudaError_t e) {
  if (m) snprintf(m->err, sizeof(m->err), "%s: %s", what, cudaGetErrorString(e));
  return SPH_E_CUDA;
}

#define MCK(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return mfail(m, #call, e_); \
  } while (0)

int grid_for(int64_t work, int per_block, int cap) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  return (int)(b > cap ? cap : b);
}

// Enqueue loss and gradient over samples idx[0..m) (or 0..m) into m->grad.
sph_status enqueue_loss_grad(sph_mlp *m, const float *X, const float *y, const int64_t *idx,
                             int64_t n) {
  const int nb = grid_for(n, 64, kGradBlocks);
  k_loss_grad<<<nb, kThreads, kGradSmem, m->stream>>>(net_of(m), X, y, idx, n, m->partials);
  MCK(cudaGetLastError());
  k_grad_final<<<grid_for(NPARAM + 1, 256, 64), 256, 0, m->stream>>>(m->partials, nb, m->grad);
  MCK(cudaGetLastError());
  return SPH_OK;
}

sph_status enqueue_adam(sph_mlp *m, const float *grad, float lr, float b1, float b2, float eps) {
  m->adam_t += 1;
  const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
  k_adam<<<grid_for(NPARAM, 256, 64), 256, 0, m->stream>>>(m->theta, m->mom, m->vel, grad, lr, b1,
                                                          b2, eps, c1, c2);
  MCK(cudaGetLastError());
  k_refresh_bf16<<<grid_for(NH * LD2, 256, 64), 256, 0, m->stream>>>(m->theta, m->wb);
  MCK(cudaGetLastError());
  return SPH_OK;
}

}  // namespace

// --------------------------------------------------------- in-step kernel
namespace sphk {

// After the force pass of a step (sorted order): the features of every
// particle from its converged H, count, density, Omega, dt div v and the
// H of the previous step (per-particle arrays the sort permutes); with
// recording on, the previous step's features and the target
// log(H_now / H_prev) as a training sample; with a guess mode, the starting
// radius of the next step's solve: H exp(-dt div v / 3) (continuity) or
// H exp(network) (learned), the ratio limited to [0.8, 1.25].
// NET: the network guess (the network in shared memory); otherwise the
// kernel needs no shared memory and keeps more warps in flight.
struct LearnSmem {
  Smem S;
  __nv_bfloat16 xs[4][32 * LD1];
  float outs[4][32];
};

template <bool NET>
__global__ void __launch_bounds__(128) k_learn(sph_state s, int64_t n, KParams P, LearnArgs L,
                                               Net N) {
  extern __shared__ __align__(16) unsigned char learn_smem[];
  LearnSmem &Q = *reinterpret_cast<LearnSmem *>(learn_smem);
  Smem &S = Q.S;
  const bool use_net = NET;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (NET) {
    load_net(S, N, false);
    for (int e = lane; e < 32 * LD1; e += 32) Q.xs[w][e] = __float2bfloat16_rn(0.f);
    __syncthreads();
  }
  const int64_t nchunks = (n + 31) / 32;
  for (int64_t ch = (int64_t)blockIdx.x * 4 + w; ch < nchunks; ch += (int64_t)gridDim.x * 4) {
    const int64_t i = ch * 32 + lane;
    const bool valid = i < n;
    const int64_t ic = valid ? i : ch * 32;
    const int64_t id = s.id[ic];
    const int sy = P.nsys > 1 ? sys_lookup(P.sys_begin, P.nsys, ic) : 0;
    // the features are FP32 quantities: ratios, logarithms and the cube
    // root in FP32
    const double H = s.h[ic];
    const float Hf = d2f(H);
    const float dtdiv = d2f(P.dt[sy]) * L.divv[ic];
    const double hp = L.hprev[ic];
    const bool have_prev = __double_as_longlong(hp) > 0;   // hp > 0 on the integer pipe
    const MatT<float> &M = mat_t<float>(P, s.mat[ic]);
    // (no FP64 division or conversion: both run on the FP64 unit at 1/64
    // of the FP32 rate; d2f rounds on the integer pipe)
    const float rho0 = M.rho0;
    const float hbar = cbrtf(P.lattice_k_f * (d2f(s.m[ic]) / rho0));
    const float lhp = have_prev ? logf(Hf / d2f(hp)) : 0.f;
    float f[NIN];
    f[0] = logf(Hf / hbar);
    f[1] = (float)s.nngb[ic] / (float)P.n_ngb - 1.f;
    f[2] = logf(d2f(s.rho[ic]) / rho0);
    f[3] = dtdiv;
    f[4] = lhp;
    f[5] = d2f(s.omega[ic]) - 1.f;
    if (valid && L.record) {
      float *xo = L.x_out + id * NIN;
      const bool have = have_prev;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 fp = L.feat[k][ic];
        xo[2 * k] = have ? fp.x : NAN;
        xo[2 * k + 1] = have ? fp.y : NAN;
      }
      L.y_out[id] = have ? lhp : NAN;
#pragma unroll
      for (int k = 0; k < 3; ++k) L.feat[k][ic] = make_float2(f[2 * k], f[2 * k + 1]);
    }
    float r = 0.f;
    if (L.guess == SPH_GUESS_CONTINUITY) r = -dtdiv / 3.f;
    if (use_net) {
#pragma unroll
      for (int k = 0; k < NIN; ++k)
        Q.xs[w][lane * LD1 + k] = __float2bfloat16_rn((f[k] - S.mu[k]) * S.isd[k]);
      __syncwarp();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t ax[4];
        load_a(Q.xs[w], LD1, 16 * half, 0, ax);
        float o[2];
        infer_tile(S, ax, o);
        if ((lane & 3) == 0) {
          Q.outs[w][16 * half + (lane >> 2)] = o[0];
          Q.outs[w][16 * half + (lane >> 2) + 8] = o[1];
        }
      }
      __syncwarp();
      r = S.ymu + S.ysd * Q.outs[w][lane];
      __syncwarp();
    }
    if (valid) {
      if (L.guess != SPH_GUESS_PREVIOUS) {
        const float lo = -0.22314355f, hi = 0.22314355f;   // log 0.8, log 1.25
        r = isfinite(r) ? fminf(fmaxf(r, lo), hi) : 0.f;
        L.hprop[ic] = H * f2d(expf(r));
      }
      L.hprev[ic] = H;
    }
  }
}

cudaError_t launch_learn(sph_ctx *c) {
  if (!c->learn.hprev) return cudaSuccess;
  const int blocks = (int)((c->n + 127) / 128 < 148 * 8 ? (c->n + 127) / 128 : 148 * 8);
  if (c->learn.guess == SPH_GUESS_NETWORK)
    k_learn<true><<<blocks, 128, sizeof(LearnSmem), c->stream>>>(c->st, c->n, c->kp, c->learn,
                                                                 net_of(c->net));
  else
    k_learn<false><<<blocks, 128, 0, c->stream>>>(c->st, c->n, c->kp, c->learn, net_of(c->net));
  c->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace sphk

// ------------------------------------------------------------- C entry points
extern "C" {

sph_status sph_mlp_create(sph_mlp **out, void *stream) {
  if (!out) return SPH_E_ARG;
  *out = nullptr;
  sph_mlp *m = (sph_mlp *)calloc(1, sizeof(sph_mlp));
  if (!m) return SPH_E_ARG;
  m->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  auto al = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  };
  al((void **)&m->theta, sizeof(float) * NPARAM);
  al((void **)&m->mom, sizeof(float) * NPARAM);
  al((void **)&m->vel, sizeof(float) * NPARAM);
  al((void **)&m->norm, sizeof(float) * NNORM);
  al((void **)&m->wb, sizeof(__nv_bfloat16) * (NH * LD1 + 2 * NH * LD2));
  al((void **)&m->grad, sizeof(float) * kPart);
  al((void **)&m->partials, sizeof(float) * kPart * kGradBlocks);
  al((void **)&m->nsum, sizeof(double) * kNormCols * 148 * 4);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&m->h_out, sizeof(float) * 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGradSmem);
  if (e != cudaSuccess) {
    sph_mlp_destroy(m);
    return SPH_E_CUDA;
  }
  *out = m;
  return SPH_OK;
}

sph_status sph_mlp_destroy(sph_mlp *m) {
  if (!m) return SPH_OK;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  void *p[] = {m->theta, m->mom, m->vel, m->norm, m->wb, m->grad, m->partials, m->nsum};
  for (void *q : p)
    if (q) cudaFree(q);
  if (m->h_out) cudaFreeHost(m->h_out);
  free(m);
  return SPH_OK;
}

const char *sph_mlp_last_error(const sph_mlp *m) { return m ? m->err : "no network"; }

sph_status sph_mlp_set(sph_mlp *m, const float *theta, const float *norm) {
  if (!m || !theta || !norm) return SPH_E_ARG;
  for (int k = NIN; k < 2 * NIN + 2; ++k)
    if (k != 2 * NIN && !(norm[k] > 0.f)) return SPH_E_ARG;   // standard deviations
  MCK(cudaMemcpyAsync(m->theta, theta, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaMemcpyAsync(m->norm, norm, sizeof(float) * NNORM, cudaMemcpyHostToDevice, m->stream));
  MCK(cudaMemsetAsync(m->mom, 0, sizeof(float) * NPARAM, m->stream));
  MCK(cudaMemsetAsync(m->vel, 0, sizeof(float) * NPARAM, m->stream));
  m->adam_t = 0;
  k_refresh_bf16<<<grid_for(NH * LD2, 256, 64), 256, 0, m->stream>>>(m->theta, m->wb);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(m->stream));
  return SPH_OK;
}

sph_status sph_mlp_get(const sph_mlp *mc, float *theta, float *norm) {
  sph_mlp *m = const_cast<sph_mlp *>(mc);
  if (!m) return SPH_E_ARG;
  if (theta)
    MCK(cudaMemcpyAsync(theta, m->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
  if (norm)
    MCK(cudaMemcpyAsync(norm, m->norm, sizeof(float) * NNORM, cudaMemcpyDeviceToHost, m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  return SPH_OK;
}

sph_status sph_mlp_fit_norm(sph_mlp *m, const float *X, const float *y, int64_t n) {
  if (!m || !X || !y || n < 1) return SPH_E_ARG;
  const int nb = grid_for(n, 256, 148 * 4);
  k_norm_partials<<<nb, 256, 0, m->stream>>>(X, y, n, m->nsum);
  MCK(cudaGetLastError());
  k_norm_final<<<1, 32, 0, m->stream>>>(m->nsum, nb, m->norm, 1e-6f);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(m->stream));
  return SPH_OK;
}

sph_status sph_mlp_forward(sph_mlp *m, const float *X, int64_t n, float *pred) {
  if (!m || !X || !pred || n < 1) return SPH_E_ARG;
  const int nb = grid_for(n, 16 * kWarps, 148 * 8);
  k_forward<<<nb, kThreads, 0, m->stream>>>(net_of(m), X, n, pred);
  MCK(cudaGetLastError());
  return SPH_OK;
}

sph_status sph_mlp_loss_grad(sph_mlp *m, const float *X, const float *y, const int64_t *idx,
                             int64_t n, float *loss, float *grad) {
  if (!m || !X || !y || n < 1) return SPH_E_ARG;
  sph_status s = enqueue_loss_grad(m, X, y, idx, n);
  if (s != SPH_OK) return s;
  if (grad)
    MCK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice,
                        m->stream));
  MCK(cudaMemcpyAsync(m->h_out, m->grad + NPARAM, sizeof(float) * 2, cudaMemcpyDeviceToHost,
                      m->stream));
  MCK(cudaStreamSynchronize(m->stream));
  if (loss) *loss = m->h_out[0];
  return SPH_OK;
}

sph_status sph_mlp_adam_step(sph_mlp *m, const float *grad, float lr, float beta1, float beta2,
                             float eps) {
  if (!m || !grad || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return SPH_E_ARG;
  sph_status s = enqueue_adam(m, grad, lr, beta1, beta2, eps);
  if (s != SPH_OK) return s;
  MCK(cudaStreamSynchronize(m->stream));
  return SPH_OK;
}

sph_status sph_mlp_train_epoch(sph_mlp *m, const float *X, const float *y, const int64_t *perm,
                               int64_t n, int32_t batch, float lr, float *mean_loss) {
  if (!m || !X || !y || !perm || n < 1 || batch < 16 || !(lr > 0.f)) return SPH_E_ARG;
  // the loss of every minibatch is kept on the device and summed at the end
  double total = 0.0;
  int nbatch = 0;
  for (int64_t b0 = 0; b0 < n; b0 += batch) {
    const int64_t cnt = n - b0 < batch ? n - b0 : batch;
    sph_status s = enqueue_loss_grad(m, X, y, perm + b0, cnt);
    if (s == SPH_OK) s = enqueue_adam(m, m->grad, lr, 0.9f, 0.999f, 1e-8f);
    if (s != SPH_OK) return s;
    MCK(cudaMemcpyAsync(m->h_out, m->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost,
                        m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    total += m->h_out[0];
    ++nbatch;
  }
  if (mean_loss) *mean_loss = (float)(total / nbatch);
  return SPH_OK;
}

}  // extern "C"
