// sph_mlp.cuh -- warp-level tensor-core evaluation of the smoothing-length
// network (the learned form): 6 standardised features -> 64 tanh -> 64 tanh
// -> 1 linear output, bf16 operands and FP32 accumulation through
// mma.sync m16n8k16. One warp evaluates a tile of 16 rows; the layers stay
// in registers, the accumulator fragment of one layer being repacked as the
// operand fragment of the next.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace sphk {
namespace mlp {

constexpr int NIN = 6;                   // features
constexpr int NH = 64;                   // hidden units per layer
constexpr int OFF_W1 = 0;                // W1[64][6], row = hidden unit
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;      // W2[64][64], row = unit of layer 2
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;
constexpr int NPARAM = OFF_B3 + 1;       // 4673
constexpr int NNORM = 2 * NIN + 2;       // x_mu[6], x_sd[6], y_mu, y_sd
// shared-memory row strides (bf16 elements) chosen so that the eight row
// groups of a fragment load fall in distinct banks
constexpr int LD1 = 24;                  // W1 and the feature tiles: 16 used
constexpr int LD2 = 72;                  // 64-wide matrices

// Device copy of a network: FP32 master parameters, normalisation and the
// bf16 operand copies the kernels read.
struct Net {
  const float *theta;
  const float *norm;
  const __nv_bfloat16 *w1b;    // [NH][LD1]: W1 with the inputs padded to 16
  const __nv_bfloat16 *w2b;    // [NH][LD2]: W2
  const __nv_bfloat16 *w2tb;   // [NH][LD2]: W2 transposed
};

// Block-shared copy.
struct Smem {
  __nv_bfloat16 w1[NH * LD1];
  __nv_bfloat16 w2[NH * LD2];
  __nv_bfloat16 w2t[NH * LD2];
  float b1[NH], b2[NH], w3[NH];
  float mu[NIN], isd[NIN];
  float b3, ymu, ysd, pad_;
};

// Cooperative copy of the network into shared memory (all threads of the
// block; followed by a barrier in the caller).
__device__ __forceinline__ void load_net(Smem &S, const Net &N, bool with_transpose) {
  const uint4 *s1 = reinterpret_cast<const uint4 *>(N.w1b);
  const uint4 *s2 = reinterpret_cast<const uint4 *>(N.w2b);
  const uint4 *s3 = reinterpret_cast<const uint4 *>(N.w2tb);
  uint4 *d1 = reinterpret_cast<uint4 *>(S.w1);
  uint4 *d2 = reinterpret_cast<uint4 *>(S.w2);
  uint4 *d3 = reinterpret_cast<uint4 *>(S.w2t);
  constexpr int n1 = NH * LD1 * 2 / 16, n2 = NH * LD2 * 2 / 16;
  for (int k = threadIdx.x; k < n1; k += blockDim.x) d1[k] = s1[k];
  for (int k = threadIdx.x; k < n2; k += blockDim.x) {
    d2[k] = s2[k];
    if (with_transpose) d3[k] = s3[k];
  }
  for (int k = threadIdx.x; k < NH; k += blockDim.x) {
    S.b1[k] = N.theta[OFF_B1 + k];
    S.b2[k] = N.theta[OFF_B2 + k];
    S.w3[k] = N.theta[OFF_W3 + k];
  }
  if (threadIdx.x < NIN) {
    S.mu[threadIdx.x] = N.norm[threadIdx.x];
    S.isd[threadIdx.x] = 1.0f / N.norm[NIN + threadIdx.x];
  }
  if (threadIdx.x == 0) {
    S.b3 = N.theta[OFF_B3];
    S.ymu = N.norm[2 * NIN];
    S.ysd = N.norm[2 * NIN + 1];
  }
}

// tanh x = 1 - 2 / (e^(2x) + 1), an identity of the hyperbolic functions,
// evaluated with the hardware exponential and the fast divide: about six
// instructions where the library tanhf takes several times more, with an
// absolute error of a few 1e-7 (the first layer is rounded to bf16, 4e-3
// relative, right after). Saturates to +-1 when e^(2x) overflows or
// underflows.
__device__ __forceinline__ float tanh_fast(float x) {
  return 1.f - __fdividef(2.f, __expf(2.f * x) + 1.f);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // lo in the low half
  return *reinterpret_cast<uint32_t *>(&v);
}

// D += A B for one 16x8 tile, A 16x16 row-major, B 16x8 column-major.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of columns n0..n0+7, rows k0..k0+15 of a matrix stored with
// one row per column n ([n][k], stride ld).
__device__ __forceinline__ void load_b(const __nv_bfloat16 *W, int ld, int n0, int k0,
                                       uint32_t &b0, uint32_t &b1) {
  const int lane = threadIdx.x & 31;
  const __nv_bfloat16 *p = W + (n0 + (lane >> 2)) * ld + k0 + 2 * (lane & 3);
  b0 = *reinterpret_cast<const uint32_t *>(p);
  b1 = *reinterpret_cast<const uint32_t *>(p + 8);
}

// A fragment of rows m0..m0+15, columns k0..k0+15 of a row-major [m][k]
// matrix with stride ld.
__device__ __forceinline__ void load_a(const __nv_bfloat16 *X, int ld, int m0, int k0,
                                       uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31;
  const __nv_bfloat16 *p = X + (m0 + (lane >> 2)) * ld + k0 + 2 * (lane & 3);
  a[0] = *reinterpret_cast<const uint32_t *>(p);
  a[1] = *reinterpret_cast<const uint32_t *>(p + 8 * ld);
  a[2] = *reinterpret_cast<const uint32_t *>(p + 8);
  a[3] = *reinterpret_cast<const uint32_t *>(p + 8 * ld + 8);
}

// Accumulator fragments of a 16x64 layer (8 column tiles) repacked as the
// four 16x16 operand fragments of the next product.
__device__ __forceinline__ void to_a(const float (&c)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    a[kt][0] = pack_bf16(c[2 * kt][0], c[2 * kt][1]);
    a[kt][1] = pack_bf16(c[2 * kt][2], c[2 * kt][3]);
    a[kt][2] = pack_bf16(c[2 * kt + 1][0], c[2 * kt + 1][1]);
    a[kt][3] = pack_bf16(c[2 * kt + 1][2], c[2 * kt + 1][3]);
  }
}

// Layers of one 16-row tile. Lane (g, t) = (lane / 4, lane % 4) holds rows
// g and g + 8, columns 8 nt + 2 t + {0, 1} of every 16x64 layer.
struct Tile {
  float a1[8][4];   // first hidden layer (FP32)
  float a2[8][4];   // second hidden layer (FP32)
  float out[2];     // standardised output of rows g and g + 8
};

__device__ __forceinline__ void forward_tile(const Smem &S, const uint32_t (&ax)[4], Tile &T) {
  const int t = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t b0, b1;
    load_b(S.w1, LD1, 8 * nt, 0, b0, b1);
    mma16816(c, ax, b0, b1);
    const int col = 8 * nt + 2 * t;
    T.a1[nt][0] = tanh_fast(c[0] + S.b1[col]);
    T.a1[nt][1] = tanh_fast(c[1] + S.b1[col + 1]);
    T.a1[nt][2] = tanh_fast(c[2] + S.b1[col]);
    T.a1[nt][3] = tanh_fast(c[3] + S.b1[col + 1]);
  }
  uint32_t a1f[4][4];
  to_a(T.a1, a1f);
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      uint32_t b0, b1;
      load_b(S.w2, LD2, 8 * nt, 16 * kt, b0, b1);
      mma16816(c, a1f[kt], b0, b1);
    }
    const int col = 8 * nt + 2 * t;
    T.a2[nt][0] = tanh_fast(c[0] + S.b2[col]);
    T.a2[nt][1] = tanh_fast(c[1] + S.b2[col + 1]);
    T.a2[nt][2] = tanh_fast(c[2] + S.b2[col]);
    T.a2[nt][3] = tanh_fast(c[3] + S.b2[col + 1]);
    p0 += T.a2[nt][0] * S.w3[col] + T.a2[nt][1] * S.w3[col + 1];
    p1 += T.a2[nt][2] * S.w3[col] + T.a2[nt][3] * S.w3[col + 1];
  }
  // the four lanes of a row group hold the row's partial dot products
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  T.out[0] = p0 + S.b3;
  T.out[1] = p1 + S.b3;
}

// Inference only (the in-step guess): both hidden layers through the
// hardware tanh on bf16 pairs, one special-function instruction per two
// units. The first layer's result is then already the bf16 operand of the
// second product; the second layer's pairs are widened to FP32 for the
// output's dot product. bf16 activations put about 4e-3 relative error on
// the proposal of log(H_n+1 / H_n), a few 1e-5 on H itself, which the
// Newton solve that follows removes. Training and the forward entry point
// keep FP32 activations (tanh_fast).
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t v) {
  uint32_t y;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(v));
  return y;
}

__device__ __forceinline__ void infer_tile(const Smem &S, const uint32_t (&ax)[4], float (&out)[2]) {
  const int t = threadIdx.x & 3;
  uint32_t a1f[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t b0, b1;
    load_b(S.w1, LD1, 8 * nt, 0, b0, b1);
    mma16816(c, ax, b0, b1);
    const int col = 8 * nt + 2 * t;
    // rows g and g + 8 of columns col, col + 1: the A-fragment halves of
    // the next product (see to_a)
    a1f[nt >> 1][2 * (nt & 1)] = tanh_bf16x2(pack_bf16(c[0] + S.b1[col], c[1] + S.b1[col + 1]));
    a1f[nt >> 1][2 * (nt & 1) + 1] =
        tanh_bf16x2(pack_bf16(c[2] + S.b1[col], c[3] + S.b1[col + 1]));
  }
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      uint32_t b0, b1;
      load_b(S.w2, LD2, 8 * nt, 16 * kt, b0, b1);
      mma16816(c, a1f[kt], b0, b1);
    }
    const int col = 8 * nt + 2 * t;
    const uint32_t lo = tanh_bf16x2(pack_bf16(c[0] + S.b2[col], c[1] + S.b2[col + 1]));
    const uint32_t hi = tanh_bf16x2(pack_bf16(c[2] + S.b2[col], c[3] + S.b2[col + 1]));
    p0 += __uint_as_float(lo << 16) * S.w3[col] + __uint_as_float(lo & 0xffff0000u) * S.w3[col + 1];
    p1 += __uint_as_float(hi << 16) * S.w3[col] + __uint_as_float(hi & 0xffff0000u) * S.w3[col + 1];
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  out[0] = p0 + S.b3;
  out[1] = p1 + S.b3;
}

}  // namespace mlp
}  // namespace sphk
