// sph_noalloc.cu -- global sums of a particle state without any allocation.
//
// The per-step diagnostics of sph_step reduce per-block partial sums through
// scratch that sph_init allocates. This file offers the same reduction to
// callers that may not allocate device memory at all: code that runs inside
// a host application which has already committed the whole device heap to
// its own caching allocator or a fixed memory budget, and monitoring hooks
// that must not change the device's allocation state between steps. Their
// scratch is a fixed, file-scope device array instead.
#include <mutex>

#include "sph_internal.cuh"

namespace {

constexpr int kDiagBlocks = 148 * 8;   // at most this many partial-sum blocks
constexpr int kDiagSums = 8;           // e_kin, e_int, p[3], L[3]
constexpr int kDiagThreads = 256;
constexpr int kMaxDevices = 64;

// Block partial sums shared by every call on a device: 1184 x 8 doubles
// (75,776 bytes). Every GPU that loads the library holds this array until
// the process exits. Each call overwrites the slots of the blocks it
// launches before it reads them, so nothing has to start at zero.
static __device__ __align__(256) double g_diag_scratch[kDiagBlocks * kDiagSums];

// Device address of g_diag_scratch per device: looked up by every call made
// outside a stream capture; a captured call uses the last address found.
std::mutex g_diag_mutex;
double *g_diag_addr[kMaxDevices];

__global__ void __launch_bounds__(kDiagThreads) k_diag_partials(sph_state s, int64_t n,
                                                              double *partials) {
  __shared__ double red[kDiagSums][kDiagThreads / 32];
  double acc[kDiagSums] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double m = s.m[i], vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
    const double x = s.x[i], y = s.y[i], z = s.z[i];
    acc[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    acc[1] += m * s.u[i];
    acc[2] += m * vx;
    acc[3] += m * vy;
    acc[4] += m * vz;
    acc[5] += m * (y * vz - z * vy);
    acc[6] += m * (z * vx - x * vz);
    acc[7] += m * (x * vy - y * vx);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagSums; ++k) acc[k] = sphk::wsum(acc[k]);
  if (lane == 0)
    for (int k = 0; k < kDiagSums; ++k) red[k][w] = acc[k];
  __syncthreads();
  if (threadIdx.x < kDiagSums) {
    double t = 0.0;
    for (int q = 0; q < kDiagThreads / 32; ++q) t += red[threadIdx.x][q];
    partials[blockIdx.x * kDiagSums + threadIdx.x] = t;
  }
}

// Fixed-order sum of the partials of the blocks just launched.
__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double *partials, int nblocks,
                                                           double *out) {
  __shared__ double red[kDiagThreads / 32];
  for (int k = 0; k < kDiagSums; ++k) {
    double t = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) t += partials[b * kDiagSums + k];
    t = sphk::wsum(t);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int q = 0; q < kDiagThreads / 32; ++q) sum += red[q];
      out[k] = sum;
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" sph_status sph_diagnostics_noalloc(const sph_state *st, int64_t n, double *sums,
                                              void *cuda_stream) {
  if (!st || !sums || n < 1 || n > SPH_NOALLOC_MAX_N) return SPH_E_ARG;
  if (!st->x || !st->y || !st->z || !st->vx || !st->vy || !st->vz || !st->u || !st->m)
    return SPH_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SPH_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SPH_E_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // An error left pending by earlier, unrelated work is not this call's.
  (void)cudaGetLastError();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) return SPH_E_CUDA;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_diag_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
      // Looked up again on every call outside a capture: after a device
      // reset the module, and so the array, may sit at another address.
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_diag_scratch) != cudaSuccess || !p) return SPH_E_CUDA;
      g_diag_addr[dev] = (double *)p;
    } else if (!g_diag_addr[dev]) {
      return SPH_E_STATE;   // the first call on a device must not be captured
    }
    scratch = g_diag_addr[dev];
  }
  int64_t blocks = (n + kDiagThreads - 1) / kDiagThreads;
  if (blocks > kDiagBlocks) blocks = kDiagBlocks;
  k_diag_partials<<<(int)blocks, kDiagThreads, 0, stream>>>(*st, n, scratch);
  if (cudaGetLastError() != cudaSuccess) return SPH_E_CUDA;
  k_diag_final<<<1, kDiagThreads, 0, stream>>>(scratch, (int)blocks, sums);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
