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
