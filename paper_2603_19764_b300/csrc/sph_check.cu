// sph_check.cu -- self-check of the integer-pipe FP64 <-> FP32 conversions
// the per-particle kernels use, against the hardware conversion.
#include "sph_internal.cuh"

namespace {
__global__ void k_check_conversions(const double *in, int64_t n, unsigned long long *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = in[i];
    const float a = sphk::d2f(d), h = __double2float_rn(d);
    const bool same = __float_as_uint(a) == __float_as_uint(h) || (isnan(a) && isnan(h));
    const double ba = sphk::f2d(h), bh = (double)h;
    const bool back = __double_as_longlong(ba) == __double_as_longlong(bh) || (isnan(ba) && isnan(bh));
    if (!same || !back) atomicAdd(bad, 1ull);
  }
}
}  // namespace

extern "C" sph_status sph_check_conversions(const double *in, int64_t n, int64_t *mismatches,
                                            void *cuda_stream) {
  if (!in || !mismatches || n < 1) return SPH_E_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned long long *d = nullptr, h = 0;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return SPH_E_CUDA;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(*d), stream);
  if (e == cudaSuccess) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    k_check_conversions<<<(int)blocks, 256, 0, stream>>>(in, n, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(d);
  if (e != cudaSuccess) return SPH_E_CUDA;
  *mismatches = (int64_t)h;
  return SPH_OK;
}

// ------------------------------------------------------------------------
// FMA throughput of the GPU (the denominator of the pair kernels' ALU
// roofline, measured rather than taken from unit counts): every thread runs
// kChains independent chains a <- a * b + c, kUnroll FMAs deep per loop trip,
// so that the issue rate, not the FMA latency, bounds the loop. Block 0's
// thread 0 reads the SM cycle counter and the global nanosecond timer at
// both ends: cycles per nanosecond is the SM clock while the launch ran.
namespace {
constexpr int kChains = 8, kUnroll = 8, kPeakThreads = 256, kPeakBlocksPerSm = 4;

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int64_t trips, T b, T c, T *sink,
                                                          long long *clk) {
  long long c0 = 0, t0 = 0;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  if (timer) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
  for (int64_t it = 0; it < trips; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma_rn(a[k], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-1.5) sink[0] = s;   // never true for these b, c; keeps the chains live
  if (timer) {
    long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = clock64() - c0;
    clk[1] = t1 - t0;
  }
}

template <typename T>
sph_status fma_peak(int64_t trips, int32_t launches, sph_peak_report *out, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPH_E_CUDA;
  const int blocks = nsm * kPeakBlocksPerSm;
  void *buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) return SPH_E_CUDA;
  T *sink = (T *)buf;
  long long *clk = (long long *)((char *)buf + 32);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const T b = (T)0.999999, c = (T)1e-6;
  if (e == cudaSuccess) {
    k_fma_peak<T><<<blocks, kPeakThreads, 0, stream>>>(trips, b, c, sink, clk);   // warm-up
    e = cudaEventRecord(e0, stream);
  }
  for (int32_t l = 0; l < launches && e == cudaSuccess; ++l) {
    k_fma_peak<T><<<blocks, kPeakThreads, 0, stream>>>(trips, b, c, sink, clk);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
  long long hclk[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return SPH_E_CUDA;
  const double flops =
      2.0 * kChains * kUnroll * (double)trips * (double)blocks * kPeakThreads;
  out->ms = ms / launches;
  out->flops = flops;
  out->tflops = flops / (out->ms * 1e-3) * 1e-12;
  out->sm_mhz = hclk[1] > 0 ? 1e3 * (double)hclk[0] / (double)hclk[1] : 0.0;
  out->n_sm = nsm;
  return SPH_OK;
}
}  // namespace

extern "C" sph_status sph_measure_fma_peak(int32_t precision, int32_t launches,
                                           sph_peak_report *out, void *cuda_stream) {
  if (!out || launches < 1 || launches > 10000 || (precision != 0 && precision != 1))
    return SPH_E_ARG;
  // about 4 ms a launch at the FP32 unit-count rate; FP64 runs 1/32 of the
  // trips (about 8 ms at 1/64 of the FP32 rate)
  return precision == 1 ? fma_peak<float>(16384, launches, out, (cudaStream_t)cuda_stream)
                        : fma_peak<double>(512, launches, out, (cudaStream_t)cuda_stream);
}
