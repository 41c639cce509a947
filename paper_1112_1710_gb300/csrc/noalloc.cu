// noalloc.cu -- conservation sums that allocate nothing.
//
// mhd_conservation_sums_static computes exactly what mhd_conservation_sums
// computes (the same per-block partial sums in the same fixed reduction
// order, so the same bits), but it needs no context and allocates no device
// or host memory: the per-block partial sums live in the file-scope array
// below, and the patch descriptors travel as a kernel parameter.
//
// It exists for callers that cannot allocate: code whose device memory is
// owned by another allocator that has reserved all of it (a serving
// framework's caching pool), code that must not call cudaMalloc/cudaFree
// because those calls can synchronise the device and stall work on other
// streams in a latency-critical loop, and plugin or embedded hosts that are
// not permitted to allocate at all.
//
// The array is a static __device__ object: every GPU that loads this library
// holds it (kMaxBlocks * 8 doubles, 1 MiB) until the process exits, and all
// calls on a device share it.  Each call overwrites the partials of the
// blocks it launches and reads only those, so nothing has to start at zero;
// two calls that overlap on the GPU (different streams, no ordering between
// them) race on the array and may return wrong sums.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "mhd_gpu.h"

namespace {

using mhd::DPatch;
using mhd::kThreads;

constexpr int kMaxBlocks = 16384;  // 16384 blocks x 256 cells = 4,194,304 cells
constexpr int kMaxPatches = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxBlocks * 8];

struct StaticSumArgs {
  DPatch p[kMaxPatches];
  int32_t first_block[kMaxPatches + 1];  // block b works on patch p with first_block[p] <= b < first_block[p+1]
  int32_t npatch;
  int32_t dtype;
};

// Host-side address of g_partials, looked up once per device with that device
// current (in host code the symbol itself is only a stand-in), together with
// the CUDA context it belongs to: after cudaDeviceReset (or any other end of
// the device's primary context) the module is loaded again, possibly at
// another address, so a change of the current context triggers a new lookup.
std::mutex g_mu;
bool g_ready[kMaxDevices] = {};
double* g_addr[kMaxDevices] = {};
CUcontext g_ctx[kMaxDevices] = {};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_sums_static(StaticSumArgs a, double* partials) {
  int p = 0;
  while (p + 1 < a.npatch && (int)blockIdx.x >= a.first_block[p + 1]) ++p;
  const DPatch& d = a.p[p];
  const int e = (blockIdx.x - a.first_block[p]) * kThreads + threadIdx.x;
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = 0.0;
  if (e < d.n[0] * d.n[1] * d.n[2]) {
    const int i = d.g + e % d.n[0], j = d.g + (e / d.n[0]) % d.n[1], k = d.g + e / (d.n[0] * d.n[1]);
    const int64_t x = (int64_t)i + (int64_t)j * d.s1 + (int64_t)k * d.s2;
    const double dv = d.dx[0] * d.dx[1] * d.dx[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = (double)((const R*)d.U[q])[x] * dv;
#pragma unroll
    for (int c = 0; c < 3; ++c) v[5 + c] = (double)((const R*)d.B[c])[x] * dv;
  }
  __shared__ double sh[8][kThreads];
#pragma unroll
  for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) partials[(int64_t)blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads) k_sums_static_final(const double* partials, int nblocks,
                                                                double* out) {
  __shared__ double sh[8][kThreads];
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = v[q] + partials[(int64_t)b * 8 + q];
#pragma unroll
  for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < 8; ++q) sh[q][threadIdx.x] = sh[q][threadIdx.x] + sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 8) out[threadIdx.x] = sh[threadIdx.x][0];
}

bool describe(const mhd_patch_desc& d, DPatch& o) {
  if (d.dtype != MHD_F64 && d.dtype != MHD_F32) return false;
  if (d.nghost < 0 || d.nghost > 64 || d.stride[0] != 1) return false;
  std::memset(&o, 0, sizeof o);
  int64_t N[3];
  for (int a = 0; a < 3; ++a) {
    const int64_t n = (int64_t)d.interior.hi[a] - d.interior.lo[a] + 1;
    if (n < 1 || n > (1 << 20) || !(d.dx[a] > 0.0)) return false;
    N[a] = n + 2 * d.nghost;
    o.n[a] = (int32_t)n;
    o.N[a] = (int32_t)N[a];
    o.dx[a] = d.dx[a];
  }
  if (d.stride[1] < N[0] + 1 || d.stride[2] < d.stride[1] * (N[1] + 1)) return false;
  for (int q = 0; q < 5; ++q) {
    if (!d.U[q]) return false;
    o.U[q] = d.U[q];
  }
  for (int a = 0; a < 3; ++a) {
    if (!d.B[a]) return false;
    o.B[a] = d.B[a];
  }
  o.s1 = d.stride[1];
  o.s2 = d.stride[2];
  o.g = d.nghost;
  return true;
}

}  // namespace

extern "C" mhd_status mhd_conservation_sums_static(const mhd_patch_desc* patches, int32_t n,
                                                   double* d_out8, void* stream) {
  if (n < 1 || !patches || !d_out8) return MHD_EINVAL;
  if (n > kMaxPatches) return MHD_ETOOBIG;
  StaticSumArgs a;
  std::memset(&a, 0, sizeof a);
  a.npatch = n;
  a.dtype = patches[0].dtype;
  int64_t blocks = 0;
  for (int p = 0; p < n; ++p) {
    if (patches[p].dtype != a.dtype || !describe(patches[p], a.p[p])) return MHD_EINVAL;
    a.first_block[p] = (int32_t)blocks;
    const int64_t cells = (int64_t)a.p[p].n[0] * a.p[p].n[1] * a.p[p].n[2];
    blocks += (cells + kThreads - 1) / kThreads;
    if (blocks > kMaxBlocks) return MHD_ETOOBIG;
  }
  a.first_block[n] = (int32_t)blocks;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MHD_ECUDA;
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    // cuCtxGetCurrent through the runtime's driver entry points (the library
    // does not link the driver library itself)
    static CUresult (*ctx_current)(CUcontext*) = nullptr;
    if (!ctx_current) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return MHD_ECUDA;
      }
      ctx_current = (CUresult(*)(CUcontext*))fn;
    }
    CUcontext cur = nullptr;
    if (ctx_current(&cur) != CUDA_SUCCESS) return MHD_ECUDA;
    if (!g_ready[dev] || cur == nullptr || cur != g_ctx[dev]) {
      void* ptr = nullptr;
      // (with no context current yet, this lookup makes the device's primary
      // context current; the context is read again afterwards)
      if (cudaGetSymbolAddress(&ptr, g_partials) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return MHD_ECUDA;
      }
      if (ctx_current(&cur) != CUDA_SUCCESS || cur == nullptr) return MHD_ECUDA;
      g_addr[dev] = (double*)ptr;
      g_ctx[dev] = cur;
      g_ready[dev] = true;
    }
    partials = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (a.dtype == MHD_F64)
    k_sums_static<double><<<(int)blocks, kThreads, 0, s>>>(a, partials);
  else
    k_sums_static<float><<<(int)blocks, kThreads, 0, s>>>(a, partials);
  k_sums_static_final<<<1, kThreads, 0, s>>>(partials, (int)blocks, d_out8);
  return cudaGetLastError() == cudaSuccess ? MHD_OK : MHD_ECUDA;
}
