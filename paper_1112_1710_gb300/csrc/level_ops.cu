// level_ops.cu -- per-level operations that feed the patch advance: the CFL
// time-step reduction, the list-driven ghost fill and the FP64 conservation
// sums.  Built with --fmad=false (the CFL candidate is compared bit for bit).
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "launch.h"
#include "physics.cuh"

namespace mhd {

// ---------------------------------------------------------------- CFL dt
// Per interior cell: t = min_d dx_d / (|v_d| + c_f,d), in the patch's
// arithmetic type.  The block minimum of t (warp shuffles, then shared
// memory; a block lies in one patch) becomes the candidate (cfl * t) * scale
// in FP64 once per block, and one atomicMin on its IEEE bits (positive, so
// integer order is value order) reduces over blocks.  x -> (cfl x) scale is
// monotone, so this equals the minimum of the per-cell candidates.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_cfl(const DPatch* __restrict__ P,
                                                  const BlockTask* __restrict__ T, double gamma_d,
                                                  double cfl, unsigned long long* out,
                                                  int* status) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  const int e = t.start + threadIdx.x;
  const R inf = R(1) / R(0);
  R m = inf;
  if (e < p.n[0] * p.n[1] * p.n[2]) {
    int i, j, k;
    if (p.n[0] * p.n[1] * p.n[2] < (1 << 24)) {
      int ri, rj;
      const int q = divmod24(e, p.n[0], ri);
      k = divmod24(q, p.n[1], rj);
      i = ri;
      j = rj;
    } else {
      i = e % p.n[0];
      j = (e / p.n[0]) % p.n[1];
      k = e / (p.n[0] * p.n[1]);
    }
    const int64_t x = (int64_t)(p.g + i) + (int64_t)(p.g + j) * p.s1 + (int64_t)(p.g + k) * p.s2;
    const R gamma = (R)gamma_d, gm1 = gamma - R(1);
    R u[8], w[8];
#pragma unroll
    for (int q = 0; q < 5; ++q) u[q] = ((const R*)p.U[q])[x];
    u[5] = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
    u[6] = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
    u[7] = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
    cons2prim(u, gm1, w);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      R cf = fast_speed(w[0], w[4], w[5 + d], w[5 + t1], w[5 + t2], gamma);
      R tt = dx_of<R>(p, d) / (Tr<R>::abs(w[1 + d]) + cf);
      m = rmin(m, tt);
    }
    if (!(w[0] > R(0)) || !(w[4] > R(0))) raise_status(status, -4);
  }
  for (int o = 16; o > 0; o >>= 1) {
    R u2 = __shfl_down_sync(0xffffffffu, m, o);
    m = (u2 < m) ? u2 : m;
  }
  __shared__ R red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : inf;
    for (int o = 16; o > 0; o >>= 1) {
      R u2 = __shfl_down_sync(0xffffffffu, m, o);
      m = (u2 < m) ? u2 : m;
    }
    if (threadIdx.x == 0) {
      const double v = (cfl * (double)m) * p.cfl_scale;
      if (v == v) atomicMin(out, (unsigned long long)__double_as_longlong(v));
    }
  }
}

__global__ void k_set_inf(unsigned long long* out) {
  *out = 0x7FF0000000000000ULL;
}

cudaError_t cfl_dt_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks,
                          double gamma, double cfl, double* d_out, int* d_status,
                          const KernelTimer* tm, cudaStream_t s) {
  MHD_TIMED(tm, K_CFL, s, (k_set_inf<<<1, 1, 0, s>>>((unsigned long long*)d_out)));
  if (nblocks > 0) {
    if (dtype == 0)
      MHD_TIMED(tm, K_CFL, s, (k_cfl<double><<<nblocks, kThreads, 0, s>>>(
                                  patches, tasks, gamma, cfl, (unsigned long long*)d_out, d_status)));
    else
      MHD_TIMED(tm, K_CFL, s, (k_cfl<float><<<nblocks, kThreads, 0, s>>>(
                                  patches, tasks, gamma, cfl, (unsigned long long*)d_out, d_status)));
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sums
// Two passes with a fixed reduction tree, so the result is reproducible.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_sums(const DPatch* __restrict__ P,
                                                   const BlockTask* __restrict__ T,
                                                   double* partials) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  const int e = t.start + threadIdx.x;
  double v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = 0.0;
  if (e < p.n[0] * p.n[1] * p.n[2]) {
    const int i = p.g + e % p.n[0], j = p.g + (e / p.n[0]) % p.n[1], k = p.g + e / (p.n[0] * p.n[1]);
    const int64_t x = (int64_t)i + (int64_t)j * p.s1 + (int64_t)k * p.s2;
    const double dv = p.dx[0] * p.dx[1] * p.dx[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = (double)((const R*)p.U[q])[x] * dv;
#pragma unroll
    for (int a = 0; a < 3; ++a) v[5 + a] = (double)((const R*)p.B[a])[x] * dv;
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

__global__ void __launch_bounds__(kThreads) k_sums_final(const double* partials, int nblocks,
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

cudaError_t sums_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks,
                        double* partials, double* d_out8, const KernelTimer* tm, cudaStream_t s) {
  if (nblocks > 0) {
    if (dtype == 0)
      MHD_TIMED(tm, K_SUMS, s, (k_sums<double><<<nblocks, kThreads, 0, s>>>(patches, tasks, partials)));
    else
      MHD_TIMED(tm, K_SUMS, s, (k_sums<float><<<nblocks, kThreads, 0, s>>>(patches, tasks, partials)));
  }
  MHD_TIMED(tm, K_SUMS, s, (k_sums_final<<<1, kThreads, 0, s>>>(partials, nblocks, d_out8)));
  return cudaGetLastError();
}

}  // namespace mhd
