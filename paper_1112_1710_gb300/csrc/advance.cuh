// advance.cuh -- the staged patch advance (A of the paper's Sec. 2.2 life
// cycle) over a batch of patches, templated on the arithmetic type R.
//
// One step of a patch updates the cells of its update box UB = interior grown
// by k layers (Sec. 2.3 extended ghosts) and the faces of those cells; it reads
// data on UB grown by 2.  The stages, each one thread per element, every
// block working inside one patch (BlockTask):
//   k_prim    UB+2 cells : primitives W, cell EMF E^n = -v x Bc
//   k_pred    UB+1 cells : limited slopes, face values, positivity rule,
//                          Hancock predictor, predicted face states, E_ref
//   k_edge    UB+2 cells : E^n at the cell's three edges (mean of the four
//                          cells; FP64 builds)
//   k_flux    faces      : CT half-step normal field, HLLD flux, contact side
//   k_emf     UB+2 cells : Gardiner-Stone (or arithmetic) EMF of the cell's
//                          three edges (FP64 builds)
//   k_update  UB         : conservative cell update and CT face update
// The FP32 build computes the edge averages inside k_flux and the edge EMFs
// inside k_update, from the cell and face values around each edge (measured
// on GB300: a launch fewer pays in FP32, while in FP64 the recomputation of
// edges shared by several faces costs more than the launch).
// Intermediates live in a per-patch scratch region with the patch's own
// strides, so every stage addresses them like the state arrays.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "launch.h"
#include "physics.cuh"

// Each translation unit that instantiates the advance names its own inner
// namespace, so that instantiations built with different floating-point
// flags (FP64 with and without multiply-add contraction) never share a
// symbol.
#ifndef MHD_ADVANCE_NS
#error "define MHD_ADVANCE_NS before including advance.cuh"
#endif
// Resident blocks per SM the FP32 predictor is compiled for.
#ifndef MHD_PRED_MINB
#define MHD_PRED_MINB 3
#endif
#ifndef MHD_FAST_RECIP
#error "define MHD_FAST_RECIP (0: divide as the oracle does; 1: reciprocal form of HLLD)"
#endif

namespace mhd {
namespace MHD_ADVANCE_NS {

// HLLD in the reciprocal form (FP32 and contracted FP64 builds) or with the
// oracle's divisions (parity build).
constexpr bool kFastRecip = MHD_FAST_RECIP != 0;

// Launch regions of the predictor / flux stages (UB grown by kM1) and of the
// update stages ([lo - kMu, hi + kMuT]); see region_m1 / region_mu.
template <typename R> constexpr int kM1 = region_m1(sizeof(R));
template <typename R> constexpr int kMu = region_mu(sizeof(R));
template <typename R> constexpr int kMuT = region_mu_top(sizeof(R));

// Where the edge averages of E^n and the edge EMFs are computed: inside the
// kernels that use them (k_flux and k_update, FP32) or by k_edge and k_emf
// into scratch planes (FP64).
template <typename R> constexpr bool kInlineEdges = sizeof(R) == 4;

template <typename R> struct SolverConsts {
  R gamma, gm1, igm1, eps_up;
  int limiter, emf;
  R p_floor, rho_floor;
};

struct Cell {
  int i, j, k;
};

// Decomposes element e of the launch region [lo - M, hi + MT]^3 of patch p
// (lo, hi: the update box UB) into a cell; false if e is beyond the region.
// The primitives (and in FP64 the edge averages) launch over UB+2; the other
// stages over the regions of launch.h (region_m1, region_mu).
template <int M, int MT>
__device__ __forceinline__ bool region_cell(const DPatch& p, int e, Cell& c) {
  const int ex = p.n[0] + 2 * p.k + M + MT, ey = p.n[1] + 2 * p.k + M + MT, ez = p.n[2] + 2 * p.k + M + MT;
  if (e >= ex * ey * ez) return false;
  const int lo = p.g - p.k - M;
  if (ex * ey * ez < (1 << 24)) {
    int rx, ry;
    const int qx = divmod24(e, ex, rx);
    const int qy = divmod24(qx, ey, ry);
    c.i = lo + rx;
    c.j = lo + ry;
    c.k = lo + qy;
  } else {  // very large patches: exact integer division
    c.i = lo + e % ex;
    c.j = lo + (e / ex) % ey;
    c.k = lo + e / (ex * ey);
  }
  return true;
}

// Is index v along axis d inside [lo_d + a, hi_d + b] of the update box?
__device__ __forceinline__ bool in_ub(const DPatch& p, int d, int v, int a, int b) {
  const int lo = p.g - p.k, hi = p.g + p.n[d] - 1 + p.k;
  return v >= lo + a && v <= hi + b;
}

__device__ __forceinline__ int64_t lin(const DPatch& p, const Cell& c) {
  return (int64_t)c.i + (int64_t)c.j * p.s1 + (int64_t)c.k * p.s2;
}

__device__ __forceinline__ int64_t stride_of(const DPatch& p, int d) {
  return d == 0 ? (int64_t)1 : (d == 1 ? p.s1 : p.s2);
}

template <typename R> __device__ __forceinline__ R* arr(R* scr, const DPatch& p, int a) {
  return scr + p.scr + (int64_t)a * p.snelem;
}

// Vector groups of scratch slots: the 8 slots from slot a on hold 8 values
// per element as vectors, FP32 in two float4 planes (values 0-3 in slots
// a..a+3 as one plane of float4, values 4-7 in slots a+4..a+7), FP64 in four
// double2 planes; one vector access moves 16 bytes per thread.  The primitives
// W and the predicted face states use them.  The planes are aligned: arena
// offsets and the plane stride (snelem) are multiples of 8 elements.  A face
// state is stored in its face's rotated frame (rho, v_n, v_t1, v_t2, p, B_t1,
// B_t2) as 7 values and a zero; the eighth slot of its group is never read.  The face
// fluxes of each axis form one group too (the 8 components in the order of
// the state, slot 5 + d carrying the contact side).
template <typename R> struct VecIO;
template <> struct VecIO<float> {
  static __device__ __forceinline__ void load8(const float* g, int64_t sn, int64_t x, float (&v)[8]) {
    const float4 a = reinterpret_cast<const float4*>(g)[x];
    const float4 b = reinterpret_cast<const float4*>(g + 4 * sn)[x];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void store8(float* g, int64_t sn, int64_t x, const float (&v)[8]) {
    reinterpret_cast<float4*>(g)[x] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(g + 4 * sn)[x] = make_float4(v[4], v[5], v[6], v[7]);
  }
  static __device__ __forceinline__ void load7(const float* g, int64_t sn, int64_t x, float (&v)[7]) {
    const float4 a = reinterpret_cast<const float4*>(g)[x];
    const float4 b = reinterpret_cast<const float4*>(g + 4 * sn)[x];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z;
  }
  // whole vectors (the eighth value 0): a partly written sector would be
  // filled from DRAM first
  static __device__ __forceinline__ void store7(float* g, int64_t sn, int64_t x, const float (&v)[7]) {
    reinterpret_cast<float4*>(g)[x] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(g + 4 * sn)[x] = make_float4(v[4], v[5], v[6], 0.0f);
  }
  static __device__ __forceinline__ void load5(const float* g, int64_t sn, int64_t x, float (&v)[5]) {
    const float4 a = reinterpret_cast<const float4*>(g)[x];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = reinterpret_cast<const float4*>(g + 4 * sn)[x].x;
  }
};
template <> struct VecIO<double> {
  static __device__ __forceinline__ void load8(const double* g, int64_t sn, int64_t x, double (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 a = reinterpret_cast<const double2*>(g + 2 * k * sn)[x];
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
  }
  static __device__ __forceinline__ void store8(double* g, int64_t sn, int64_t x, const double (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) reinterpret_cast<double2*>(g + 2 * k * sn)[x] = make_double2(v[2 * k], v[2 * k + 1]);
  }
  static __device__ __forceinline__ void load7(const double* g, int64_t sn, int64_t x, double (&v)[7]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 a = reinterpret_cast<const double2*>(g + 2 * k * sn)[x];
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
    v[6] = reinterpret_cast<const double2*>(g + 6 * sn)[x].x;
  }
  static __device__ __forceinline__ void store7(double* g, int64_t sn, int64_t x, const double (&v)[7]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) reinterpret_cast<double2*>(g + 2 * k * sn)[x] = make_double2(v[2 * k], v[2 * k + 1]);
    reinterpret_cast<double2*>(g + 6 * sn)[x] = make_double2(v[6], 0.0);
  }
  static __device__ __forceinline__ void load5(const double* g, int64_t sn, int64_t x, double (&v)[5]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double2 a = reinterpret_cast<const double2*>(g + 2 * k * sn)[x];
      v[2 * k] = a.x;
      v[2 * k + 1] = a.y;
    }
    v[4] = (g + 4 * sn)[2 * x];
  }
};

// Stores the face state pw (primitives, xyz order) of the axis-d face in its
// rotated frame.
template <typename R>
__device__ __forceinline__ void store_face_state(R* g, int64_t sn, int64_t x, int d, const R (&pw)[8]) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const R v[7] = {pw[0], pw[1 + d], pw[1 + t1], pw[1 + t2], pw[4], pw[5 + t1], pw[5 + t2]};
  VecIO<R>::store7(g, sn, x, v);
}

// Per-patch step constants dt, dt/(2 dx_d), dt/dx_d, computed once per call by
// k_stepc (one thread per patch) so that no stage thread touches the double
// dt scalar, the double dt scale or the double cell widths (on this GPU the
// FP64 pipe is 64x narrower than the FP32 one).
constexpr int kStepConsts = 8;

template <typename R>
__global__ void k_stepc(const DPatch* __restrict__ P, int npatch, const double* d_dt, R* K) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npatch) return;
  const R dt = (R)((*d_dt) * P[p].dt_scale);
  const R hdt = R(0.5) * dt;
  R* k = K + (int64_t)p * kStepConsts;
  k[0] = dt;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    k[1 + d] = hdt / (R)P[p].dx[d];
    k[4 + d] = dt / (R)P[p].dx[d];
  }
}

template <typename R> struct StepDt {
  R dt, hdtdx[3], dtdx[3];
  __device__ __forceinline__ StepDt(const R* __restrict__ K, int patch) {
    const R* k = K + (int64_t)patch * kStepConsts;
    dt = k[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      hdtdx[d] = k[1 + d];
      dtdx[d] = k[4 + d];
    }
  }
};

// ---------------------------------------------------------------- k_prim
// Primitives and cell EMFs on UB+2.  With Cfl, also the CFL time step of the
// step (the quantity mhd_cfl_dt computes, with the same expressions): each
// interior cell's candidate min_d dx_d / (|v_d| + c_f,d) from the same
// primitives, the block minimum (warp shuffles, then shared memory), and one
// atomicMin per block on the IEEE bits of (cfl * min) * cfl_scale in FP64
// (positive doubles order as their bits), into *dt_bits, which must hold
// +infinity before the launch.
template <typename R, bool Cfl>
__global__ void __launch_bounds__(kThreads) k_prim(const DPatch* __restrict__ P,
                                                   const BlockTask* __restrict__ T, R* scr,
                                                   SolverConsts<R> sc, int* status, double cfl,
                                                   unsigned long long* dt_bits) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  const bool act = region_cell<2, 2>(p, t.start + threadIdx.x, c);
  if (!Cfl && !act) return;
  const R inf = R(1) / R(0);
  R m = inf;
  if (act) {
    const int64_t x = lin(p, c);
    R u[8];
#pragma unroll
    for (int q = 0; q < 5; ++q) u[q] = ((const R*)p.U[q])[x];
    u[5] = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
    u[6] = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
    u[7] = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
    R w[8];
    cons2prim(u, sc.gm1, w);
    if constexpr (Cfl) {
      // the CFL candidate from the unfloored primitives (as mhd_cfl_dt)
      const bool interior = c.i >= p.g && c.i < p.g + p.n[0] && c.j >= p.g && c.j < p.g + p.n[1] &&
                            c.k >= p.g && c.k < p.g + p.n[2];
      if (interior) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          R cf = fast_speed(w[0], w[4], w[5 + d], w[5 + t1], w[5 + t2], sc.gamma);
          R tt = dx_of<R>(p, d) / (Tr<R>::abs(w[1 + d]) + cf);
          m = rmin(m, tt);
        }
      }
    }
    // the floors (when set) bound the primitives the step reads, ghost cells
    // included
    if (sc.rho_floor > R(0) && !(w[0] >= sc.rho_floor)) w[0] = sc.rho_floor;
    if (sc.p_floor > R(0) && !(w[4] >= sc.p_floor)) w[4] = sc.p_floor;
    VecIO<R>::store8(arr(scr, p, SC_W), p.snelem, x, w);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, cc = (a + 2) % 3;
      arr(scr, p, SC_EN + a)[x] = w[1 + cc] * w[5 + b] - w[1 + b] * w[5 + cc];
    }
    if (!(w[0] > R(0)) || !(w[4] > R(0))) raise_status(status, -4);
  }
  if constexpr (Cfl) {
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
        if (v == v) atomicMin(dt_bits, (unsigned long long)__double_as_longlong(v));
      }
    }
  }
}

// Sets the FP64 time step the CFL reduction of k_prim lowers to +infinity.
__global__ void k_dt_reset(unsigned long long* dt_bits) { *dt_bits = 0x7FF0000000000000ull; }

// ---------------------------------------------------------------- k_edge
template <typename R, int a> __device__ __forceinline__ void edge_avg(const DPatch& p, const Cell& c, R* scr);

template <typename R>
__global__ void __launch_bounds__(kThreads) k_edge(const DPatch* __restrict__ P,
                                                   const BlockTask* __restrict__ T, R* scr) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<2, 2>(p, t.start + threadIdx.x, c)) return;
  // the three edges stored at this cell, one index decomposition
  edge_avg<R, 0>(p, c, scr);
  edge_avg<R, 1>(p, c, scr);
  edge_avg<R, 2>(p, c, scr);
}

// E^n at the axis-a edge stored at element x: the mean of the cell EMFs of
// the four cells around it.
template <typename R, int a> __device__ __forceinline__ R edge_avg_at(const DPatch& p, int64_t x, const R* scr) {
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  const int64_t sb = stride_of(p, b), sc_ = stride_of(p, cc);
  const R* En = arr(scr, p, SC_EN + a);
  R e00 = En[x - sb - sc_];
  R e10 = En[x - sc_];
  R e01 = En[x - sb];
  R e11 = En[x];
  return R(0.25) * (e00 + e10 + e01 + e11);
}

template <typename R, int a> __device__ __forceinline__ void edge_avg(const DPatch& p, const Cell& c, R* scr) {
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  const int id[3] = {c.i, c.j, c.k};
  if (!in_ub(p, a, id[a], -1, 1) || !in_ub(p, b, id[b], -1, 2) || !in_ub(p, cc, id[cc], -1, 2)) return;
  const int64_t x = lin(p, c);
  arr(scr, p, SC_EE + a)[x] = edge_avg_at<R, a>(p, x, scr);
}

// ---------------------------------------------------------------- k_pred
// Limited slopes of one cell held in registers (dw[axis][component]).
template <typename R> struct RegSlopes {
  const R (&dw)[3][8];
  __device__ __forceinline__ void get(int d, R (&out)[8]) const {
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q] = dw[d][q];
  }
};

// Limited slopes of one cell parked in shared memory: six float4 rows of
// kThreads entries (axis d: rows 2d and 2d + 1), each thread its own column.
// The stores and loads are volatile asm, so that the compiler neither
// forwards the stored values in registers nor moves a load above its store;
// the slopes then do not stay live across the Hancock increment, which is
// what holds the FP32 predictor's registers down.
__device__ __forceinline__ void sts4(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}
__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
struct SmemSlopes {
  uint32_t base;  // shared address of row 0, this thread's column
  __device__ __forceinline__ void put(int d, const float (&v)[8]) const {
    sts4(base + (2 * d) * kThreads * 16, v[0], v[1], v[2], v[3]);
    sts4(base + (2 * d + 1) * kThreads * 16, v[4], v[5], v[6], v[7]);
  }
  __device__ __forceinline__ void get(int d, float (&out)[8]) const {
    const float4 a = lds4(base + (2 * d) * kThreads * 16), b = lds4(base + (2 * d + 1) * kThreads * 16);
    out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
  }
};

// First positivity rule on the face values of rho and p along one axis:
// true if a face value is not positive.
template <typename R> __device__ __forceinline__ bool face_rule1(const R (&w)[8], const R (&dw)[8]) {
  const R rm = w[0] - R(0.5) * dw[0], rp = w[0] + R(0.5) * dw[0];
  const R pm = w[4] - R(0.5) * dw[4], pp = w[4] + R(0.5) * dw[4];
  return !(rm > R(0)) || !(rp > R(0)) || !(pm > R(0)) || !(pp > R(0));
}

// The predictor of one cell from its primitives w and limited slopes (S),
// given the first positivity rule's verdict `bad` over the three axes:
// Hancock increment, the six predicted face states (second positivity rule)
// and, for the upwinded EMF average, the reference cell EMF, stored at
// element x.
template <typename R, typename S>
__device__ __forceinline__ void predict_cell(const DPatch& p, int64_t x, R* scr, const SolverConsts<R>& sc,
                                             const StepDt<R>& st, const R (&w)[8], const S& slopes, bool bad) {
  // Hancock increment
  R du[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) du[q] = R(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R dw[8], fwm[8], fwp[8], fm[8], fp[8];
    slopes.get(d, dw);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      fwm[q] = bad ? w[q] : w[q] - R(0.5) * dw[q];
      fwp[q] = bad ? w[q] : w[q] + R(0.5) * dw[q];
    }
    flux_xyz(d, fwp, sc.igm1, fp);
    flux_xyz(d, fwm, sc.igm1, fm);
#pragma unroll
    for (int q = 0; q < 8; ++q) du[q] = du[q] - st.hdtdx[d] * (fp[q] - fm[q]);
  }
  // predicted face states and the second positivity rule
  bool bad2 = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R dw[8];
    slopes.get(d, dw);
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      R fw[8], u[8], pw[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) fw[q] = bad ? w[q] : (sd ? w[q] + R(0.5) * dw[q] : w[q] - R(0.5) * dw[q]);
      prim2cons(fw, sc.igm1, u);
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = u[q] + du[q];
      cons2prim(u, sc.gm1, pw);
      if (!(pw[0] > R(0)) || !(pw[4] > R(0))) bad2 = true;
      store_face_state(arr(scr, p, SC_WF + (d * 2 + sd) * 8), p.snelem, x, d, pw);
    }
  }
  R duk[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) duk[q] = du[q];
  if (bad2) {
#pragma unroll
    for (int f = 0; f < 6; ++f) store_face_state(arr(scr, p, SC_WF + f * 8), p.snelem, x, f / 2, w);
#pragma unroll
    for (int q = 0; q < 8; ++q) duk[q] = R(0);
  }
  // reference cell EMF from U^{n+1/2} (read only by the upwinded EMF average)
  if (sc.emf == 1) return;
  R uc[8], uh[8];
  prim2cons(w, sc.igm1, uc);
#pragma unroll
  for (int q = 0; q < 8; ++q) uh[q] = uc[q] + duk[q];
  R ir = R(1) / uh[0];
  R v[3] = {uh[1] * ir, uh[2] * ir, uh[3] * ir};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    arr(scr, p, SC_ER + a)[x] = v[cc] * uh[5 + b] - v[b] * uh[5 + cc];
  }
}

// One thread per cell of UB+1; the stencil of W is read from the scratch
// planes through the caches.  FP32 parks the slopes in shared memory
// (SmemSlopes) and is held at 80 registers, three blocks per SM (measured on
// GB300: 132 us against 136 us with the slopes in registers at 117 registers
// and two blocks); FP64 keeps them in registers at one block per SM, its
// time being set by the FP64 pipe.  The FP32 flux kernel is held at 64
// registers (four blocks per SM): past that the compiler's choice drops a
// block per SM and the kernel, bound by the latency of its loads, slows down.
template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? MHD_PRED_MINB : 1) k_pred(const DPatch* __restrict__ P,
                                                   const BlockTask* __restrict__ T, R* scr,
                                                   SolverConsts<R> sc, const R* __restrict__ K) {
  constexpr bool smem = sizeof(R) == 4;
  __shared__ float4 sdw[smem ? 6 : 1][smem ? kThreads : 1];
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<kM1<R>, kM1<R>>(p, t.start + threadIdx.x, c)) return;
  if (kM1<R> > 1 && (!in_ub(p, 0, c.i, -1, 1) || !in_ub(p, 1, c.j, -1, 1) || !in_ub(p, 2, c.k, -1, 1))) return;
  const StepDt<R> st(K, t.patch);
  const int64_t x = lin(p, c);
  R w[8], dw[3][8];
  const R* Wg = arr(scr, p, SC_W);
  VecIO<R>::load8(Wg, p.snelem, x, w);
  SmemSlopes ss{(uint32_t)__cvta_generic_to_shared(&sdw[0][smem ? threadIdx.x : 0])};
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t sd = stride_of(p, d);
    R wm[8], wp[8];
    VecIO<R>::load8(Wg, p.snelem, x - sd, wm);
    VecIO<R>::load8(Wg, p.snelem, x + sd, wp);
#pragma unroll
    for (int q = 0; q < 8; ++q) dw[d][q] = limiter(sc.limiter, w[q] - wm[q], wp[q] - w[q]);
    if (face_rule1(w, dw[d])) bad = true;
    if constexpr (smem) ss.put(d, dw[d]);
  }
  if constexpr (smem) predict_cell(p, x, scr, sc, st, w, ss, bad);
  else predict_cell(p, x, scr, sc, st, w, RegSlopes<R>{dw}, bad);
}

// Tiled predictor: a block owns a TX x TY x TZ tile of UB+1 cells (its task's
// `start` is the tile index within the patch), stages W on the tile grown by
// one cell in shared memory with coalesced row loads, then runs the same
// per-cell predictor from shared memory.
template <typename R> struct PredTile;
template <> struct PredTile<float> {
  static constexpr int TX = kPredTile32[0], TY = kPredTile32[1], TZ = kPredTile32[2];
};
template <> struct PredTile<double> {
  static constexpr int TX = kPredTile64[0], TY = kPredTile64[1], TZ = kPredTile64[2];
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_pred_tiled(const DPatch* __restrict__ P,
                                                         const BlockTask* __restrict__ T, R* scr,
                                                         SolverConsts<R> sc, const R* __restrict__ K) {
  constexpr int TX = PredTile<R>::TX, TY = PredTile<R>::TY, TZ = PredTile<R>::TZ;
  constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2, HN = HX * HY * HZ;
  static_assert(TX * TY * TZ == kThreads, "one thread per tile cell");
  __shared__ R sw[8][HN];
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  // the UB+1 region and this block's tile in it
  const int lo = p.g - p.k - 1;
  const int ex = p.n[0] + 2 * p.k + 2, ey = p.n[1] + 2 * p.k + 2, ez = p.n[2] + 2 * p.k + 2;
  const int ntx = (ex + TX - 1) / TX, nty = (ey + TY - 1) / TY;
  int rx, ry;
  const int q1 = divmod24(t.start, ntx, rx);
  const int tz = divmod24(q1, nty, ry);
  const int x0 = lo + rx * TX, y0 = lo + ry * TY, z0 = lo + tz * TZ;
  // stage W on the tile grown by one (always inside UB+2, where W is valid)
  const int hx_hi = min(HX, ex - rx * TX + 1), hy_hi = min(HY, ey - ry * TY + 1), hz_hi = min(HZ, ez - tz * TZ + 1);
  for (int e = threadIdx.x; e < HN; e += kThreads) {
    int hx, hy;
    const int q2 = divmod24(e, HX, hx);
    const int hz = divmod24(q2, HY, hy);
    if (hx > hx_hi || hy > hy_hi || hz > hz_hi) continue;
    const int64_t x = (int64_t)(x0 - 1 + hx) + (int64_t)(y0 - 1 + hy) * p.s1 + (int64_t)(z0 - 1 + hz) * p.s2;
    R v[8];
    VecIO<R>::load8(arr(scr, p, SC_W), p.snelem, x, v);
#pragma unroll
    for (int q = 0; q < 8; ++q) sw[q][e] = v[q];
  }
  __syncthreads();
  const int ix = threadIdx.x % TX, iy = (threadIdx.x / TX) % TY, iz = threadIdx.x / (TX * TY);
  if (rx * TX + ix >= ex || ry * TY + iy >= ey || tz * TZ + iz >= ez) return;
  const StepDt<R> st(K, t.patch);
  const int s = (ix + 1) + HX * ((iy + 1) + HY * (iz + 1));
  const int sd[3] = {1, HX, HX * HY};
  R w[8], dw[3][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) w[q] = sw[q][s];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      R a = w[q] - sw[q][s - sd[d]];
      R b = sw[q][s + sd[d]] - w[q];
      dw[d][q] = limiter(sc.limiter, a, b);
    }
  }
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (face_rule1(w, dw[d])) bad = true;
  const int64_t x = (int64_t)(x0 + ix) + (int64_t)(y0 + iy) * p.s1 + (int64_t)(z0 + iz) * p.s2;
  predict_cell(p, x, scr, sc, st, w, RegSlopes<R>{dw}, bad);
}

// ---------------------------------------------------------------- k_flux
// The face direction is a template parameter so that every array index below
// is a compile-time constant (no local-memory arrays).
template <typename R, int d>
__device__ __forceinline__ void flux_face(const DPatch& p, int patch, const Cell& c, R* scr,
                                          const SolverConsts<R>& sc, const R* __restrict__ K) {
  constexpr int b = (d + 1) % 3, cc = (d + 2) % 3;
  const int id[3] = {c.i, c.j, c.k};
  if (!in_ub(p, d, id[d], 0, 1) || !in_ub(p, b, id[b], -1, 1) || !in_ub(p, cc, id[cc], -1, 1)) return;
  const StepDt<R> st(K, patch);
  const int64_t x = lin(p, c);
  const int64_t sd = stride_of(p, d), sb = stride_of(p, b), scc = stride_of(p, cc);
  // CT half step of the face-normal field
  R dEc, dEb;
  if constexpr (kInlineEdges<R>) {
    dEc = edge_avg_at<R, cc>(p, x + sb, scr) - edge_avg_at<R, cc>(p, x, scr);
    dEb = edge_avg_at<R, b>(p, x + scc, scr) - edge_avg_at<R, b>(p, x, scr);
  } else {
    dEc = arr(scr, p, SC_EE + cc)[x + sb] - arr(scr, p, SC_EE + cc)[x];
    dEb = arr(scr, p, SC_EE + b)[x + scc] - arr(scr, p, SC_EE + b)[x];
  }
  R bh = ((const R*)p.B[d])[x] - (st.hdtdx[b] * dEc - st.hdtdx[cc] * dEb);
  R vl[7], vr[7], fr[8], f[8], upw;
  // the face states are stored in the face's rotated frame without their
  // normal field: HLLD takes the CT half-step value bh instead
  VecIO<R>::load7(arr(scr, p, SC_WF + (d * 2 + 1) * 8), p.snelem, x - sd, vl);
  VecIO<R>::load7(arr(scr, p, SC_WF + (d * 2 + 0) * 8), p.snelem, x, vr);
  const R L[8] = {vl[0], vl[1], vl[2], vl[3], vl[4], R(0), vl[5], vl[6]};
  const R Rr[8] = {vr[0], vr[1], vr[2], vr[3], vr[4], R(0), vr[5], vr[6]};
  hlld<R, kFastRecip>(L, Rr, bh, sc.gamma, sc.igm1, sc.eps_up, fr, &upw);
  rot_out(d, fr, f);
  f[5 + d] = upw;
  VecIO<R>::store8(arr(scr, p, SC_F + d * 8), p.snelem, x, f);
}

template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 4 : 2) k_flux(const DPatch* __restrict__ P,
                                                   const BlockTask* __restrict__ T, R* scr,
                                                   SolverConsts<R> sc, const R* __restrict__ K) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<kM1<R>, kM1<R>>(p, t.start + threadIdx.x, c)) return;
  flux_face<R, 0>(p, t.patch, c, scr, sc, K);
  flux_face<R, 1>(p, t.patch, c, scr, sc, K);
  flux_face<R, 2>(p, t.patch, c, scr, sc, K);
}

// ---------------------------------------------------------------- edge EMFs
// Gardiner-Stone (or arithmetic) EMF of one edge from the four face EMFs
// around it (eb_lo, eb_hi, ec_lo, ec_hi), the contact sides of those faces
// and the four reference cell EMFs, in one fixed expression order (the
// staged and the fused advance both use it).
template <typename R>
__device__ __forceinline__ R edge_emf_value(R eb_lo, R eb_hi, R ec_lo, R ec_hi, R r00, R r10, R r01, R r11,
                                            R mb_lo, R mb_hi, R mc_lo, R mc_hi, int emf) {
  R avg = R(0.25) * (eb_lo + eb_hi + ec_lo + ec_hi);
  if (emf == 1) return avg;
  R dc14, dc34, db14, db34;
  if (mb_hi > R(0)) dc14 = r01 - ec_lo;
  else if (mb_hi < R(0)) dc14 = r11 - ec_hi;
  else dc14 = R(0.5) * ((r01 - ec_lo) + (r11 - ec_hi));
  if (mb_lo > R(0)) dc34 = ec_lo - r00;
  else if (mb_lo < R(0)) dc34 = ec_hi - r10;
  else dc34 = R(0.5) * ((ec_lo - r00) + (ec_hi - r10));
  if (mc_hi > R(0)) db14 = r10 - eb_lo;
  else if (mc_hi < R(0)) db14 = r11 - eb_hi;
  else db14 = R(0.5) * ((r10 - eb_lo) + (r11 - eb_hi));
  if (mc_lo > R(0)) db34 = eb_lo - r00;
  else if (mc_lo < R(0)) db34 = eb_hi - r01;
  else db34 = R(0.5) * ((eb_lo - r00) + (eb_hi - r01));
  return avg + R(0.25) * (dc34 - dc14 + db34 - db14);
}

// EMF of the axis-a edge stored at element x: the face EMFs -F_b[B_c] of the
// two b-faces and F_c[B_b] of the two c-faces around it; with the upwinded
// average also the contact sides of those faces and the reference EMFs of
// the four cells around the edge.
template <typename R, int a>
__device__ __forceinline__ R emf_at(const DPatch& p, int64_t x, const R* scr, int emf) {
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  const int64_t sb = stride_of(p, b), scc = stride_of(p, cc);
  const int64_t sn = p.snelem;
  const R* Fb = arr(scr, p, SC_F + b * 8);
  const R* Fc = arr(scr, p, SC_F + cc * 8);
  const R eb_lo = -*vgroup_at(Fb, sn, x - scc, 5 + cc), eb_hi = -*vgroup_at(Fb, sn, x, 5 + cc);
  const R ec_lo = *vgroup_at(Fc, sn, x - sb, 5 + b), ec_hi = *vgroup_at(Fc, sn, x, 5 + b);
  if (emf == 1) return R(0.25) * (eb_lo + eb_hi + ec_lo + ec_hi);
  const R* Er = arr(scr, p, SC_ER + a);
  return edge_emf_value(eb_lo, eb_hi, ec_lo, ec_hi, Er[x - sb - scc], Er[x - scc], Er[x - sb], Er[x],
                        *vgroup_at(Fb, sn, x - scc, 5 + b), *vgroup_at(Fb, sn, x, 5 + b),
                        *vgroup_at(Fc, sn, x - sb, 5 + cc), *vgroup_at(Fc, sn, x, 5 + cc), emf);
}

// FP32 arithmetic-average edge EMF (the same value as emf_at with emf == 1)
// with the induction fluxes read as whole float4 vectors, slots 4-7 of the
// flux groups: one thread's nine edges and its cell update read 24 such
// vectors at repeated positions, which the compiler then loads once each,
// instead of 36 scalars at a 16-byte stride.
template <int i> __device__ __forceinline__ float slot4(const float4& v) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}
template <int a> __device__ __forceinline__ float emf_avg4(const DPatch& p, int64_t y, const float* scr) {
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  const int64_t sb = stride_of(p, b), scc = stride_of(p, cc);
  const float4* Fb = reinterpret_cast<const float4*>(arr(scr, p, SC_F + b * 8) + 4 * p.snelem);
  const float4* Fc = reinterpret_cast<const float4*>(arr(scr, p, SC_F + cc * 8) + 4 * p.snelem);
  const float eb_lo = -slot4<1 + cc>(Fb[y - scc]), eb_hi = -slot4<1 + cc>(Fb[y]);
  const float ec_lo = slot4<1 + b>(Fc[y - sb]), ec_hi = slot4<1 + b>(Fc[y]);
  return 0.25f * (eb_lo + eb_hi + ec_lo + ec_hi);
}

// Is the axis-a edge stored at cell c one of the edges of the update box's
// faces (the edges whose EMF the flux registers capture)?
template <int a> __device__ __forceinline__ bool update_edge(const DPatch& p, const Cell& c) {
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  const int id[3] = {c.i, c.j, c.k};
  return in_ub(p, a, id[a], 0, 0) && in_ub(p, b, id[b], 0, 1) && in_ub(p, cc, id[cc], 0, 1);
}

// ---------------------------------------------------------------- k_emf
// The EMFs of the three update-box edges stored at each cell of [lo, hi + 1].
template <typename R>
__global__ void __launch_bounds__(kThreads) k_emf(const DPatch* __restrict__ P,
                                                  const BlockTask* __restrict__ T, R* scr,
                                                  SolverConsts<R> sc) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<kMu<R>, kMuT<R>>(p, t.start + threadIdx.x, c)) return;
  const int64_t x = lin(p, c);
  const R* cs = scr;
  const bool u0 = update_edge<0>(p, c), u1 = update_edge<1>(p, c), u2 = update_edge<2>(p, c);
  R e0 = R(0), e1 = R(0), e2 = R(0);
  if (u0) e0 = emf_at<R, 0>(p, x, cs, sc.emf);
  if (u1) e1 = emf_at<R, 1>(p, x, cs, sc.emf);
  if (u2) e2 = emf_at<R, 2>(p, x, cs, sc.emf);
  if (u0) arr(scr, p, SC_ED + 0)[x] = e0;
  if (u1) arr(scr, p, SC_ED + 1)[x] = e1;
  if (u2) arr(scr, p, SC_ED + 2)[x] = e2;
}

// ---------------------------------------------------------------- k_update
// One thread per cell of [lo, hi + 1]: the cell's conservative update and the
// CT update of its three lower faces, each face from the EMFs of its four edges.
// EmfInline: the nine distinct edge EMFs a cell's faces need are computed
// here from the face fluxes (an edge is shared by four faces, so its EMF is
// evaluated by up to three threads, always with the same expression), and
// patches that feed flux registers also store the EMF of every update-box
// edge at its element, where the capture kernel reads it; otherwise they are
// read from k_emf's planes.
// At most 51 registers in FP32 (five blocks per SM) and 85 in FP64 (three); the compiler's free choice
// (80-86 in FP32) cost a quarter of the kernel's speed.
template <typename R, bool EmfInline>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 5 : 3) k_update(const DPatch* __restrict__ P,
                                                     const BlockTask* __restrict__ T, R* scr,
                                                     SolverConsts<R> sc, const R* __restrict__ K, int commit) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<kMu<R>, kMuT<R>>(p, t.start + threadIdx.x, c)) return;
  const StepDt<R> st(K, t.patch);
  const int64_t x = lin(p, c);
  const int id[3] = {c.i, c.j, c.k};
  const int64_t s1 = p.s1, s2 = p.s2;
  // every load before the first store: the state and scratch pointers may
  // alias as far as the compiler knows, so a store would order later loads
  const bool cell = in_ub(p, 0, c.i, 0, 0) && in_ub(p, 1, c.j, 0, 0) && in_ub(p, 2, c.k, 0, 0);
  bool face[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    face[a] = in_ub(p, a, id[a], 0, 1) && in_ub(p, b, id[b], 0, 0) && in_ub(p, cc, id[cc], 0, 0);
  }
  // face 0 needs E2 at x, x+s1 and E1 at x, x+s2; face 1 E0 at x, x+s2 and
  // E2 at x, x+1; face 2 E1 at x, x+1 and E0 at x, x+s1
  const R* cs = scr;
  R e0 = R(0), e0y = R(0), e0z = R(0), e1 = R(0), e1x = R(0), e1z = R(0), e2 = R(0), e2x = R(0), e2y = R(0);
  if constexpr (EmfInline && sizeof(R) == 4) {
    if (sc.emf == 1) {
      // every position these read lies in UB+2, inside the planes, so the
      // reads are unconditional and repeated positions are loaded once
      e0 = emf_avg4<0>(p, x, cs);
      e0z = emf_avg4<0>(p, x + s2, cs);
      e0y = emf_avg4<0>(p, x + s1, cs);
      e1 = emf_avg4<1>(p, x, cs);
      e1z = emf_avg4<1>(p, x + s2, cs);
      e1x = emf_avg4<1>(p, x + 1, cs);
      e2 = emf_avg4<2>(p, x, cs);
      e2y = emf_avg4<2>(p, x + s1, cs);
      e2x = emf_avg4<2>(p, x + 1, cs);
    } else {
      if (face[1] || face[2]) e0 = emf_at<R, 0>(p, x, cs, sc.emf);
      if (face[1]) e0z = emf_at<R, 0>(p, x + s2, cs, sc.emf);
      if (face[2]) e0y = emf_at<R, 0>(p, x + s1, cs, sc.emf);
      if (face[0] || face[2]) e1 = emf_at<R, 1>(p, x, cs, sc.emf);
      if (face[0]) e1z = emf_at<R, 1>(p, x + s2, cs, sc.emf);
      if (face[2]) e1x = emf_at<R, 1>(p, x + 1, cs, sc.emf);
      if (face[0] || face[1]) e2 = emf_at<R, 2>(p, x, cs, sc.emf);
      if (face[0]) e2y = emf_at<R, 2>(p, x + s1, cs, sc.emf);
      if (face[1]) e2x = emf_at<R, 2>(p, x + 1, cs, sc.emf);
    }
  } else if constexpr (EmfInline) {
    if (face[1] || face[2]) e0 = emf_at<R, 0>(p, x, cs, sc.emf);
    if (face[1]) e0z = emf_at<R, 0>(p, x + s2, cs, sc.emf);
    if (face[2]) e0y = emf_at<R, 0>(p, x + s1, cs, sc.emf);
    if (face[0] || face[2]) e1 = emf_at<R, 1>(p, x, cs, sc.emf);
    if (face[0]) e1z = emf_at<R, 1>(p, x + s2, cs, sc.emf);
    if (face[2]) e1x = emf_at<R, 1>(p, x + 1, cs, sc.emf);
    if (face[0] || face[1]) e2 = emf_at<R, 2>(p, x, cs, sc.emf);
    if (face[0]) e2y = emf_at<R, 2>(p, x + s1, cs, sc.emf);
    if (face[1]) e2x = emf_at<R, 2>(p, x + 1, cs, sc.emf);
  } else {
    const R* E0 = arr(cs, p, SC_ED + 0);
    const R* E1 = arr(cs, p, SC_ED + 1);
    const R* E2 = arr(cs, p, SC_ED + 2);
    if (face[1] || face[2]) e0 = E0[x];
    if (face[1]) e0z = E0[x + s2];
    if (face[2]) e0y = E0[x + s1];
    if (face[0] || face[2]) e1 = E1[x];
    if (face[0]) e1z = E1[x + s2];
    if (face[2]) e1x = E1[x + 1];
    if (face[0] || face[1]) e2 = E2[x];
    if (face[0]) e2y = E2[x + s1];
    if (face[1]) e2x = E2[x + 1];
  }
  R un[5];
  if (cell) {
    R f0a[5], f0b[5], f1a[5], f1b[5], f2a[5], f2b[5];
    // (FP32: VecIO::load5 reads slot 4 as the x of the plane-2 float4, the
    // vector the inline edge EMFs read too)
    VecIO<R>::load5(arr(scr, p, SC_F + 0 * 8), p.snelem, x, f0a);
    VecIO<R>::load5(arr(scr, p, SC_F + 0 * 8), p.snelem, x + 1, f0b);
    VecIO<R>::load5(arr(scr, p, SC_F + 1 * 8), p.snelem, x, f1a);
    VecIO<R>::load5(arr(scr, p, SC_F + 1 * 8), p.snelem, x + s1, f1b);
    VecIO<R>::load5(arr(scr, p, SC_F + 2 * 8), p.snelem, x, f2a);
    VecIO<R>::load5(arr(scr, p, SC_F + 2 * 8), p.snelem, x + s2, f2b);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      R u = ((const R*)p.U[q])[x];
      un[q] = u - st.dtdx[0] * (f0b[q] - f0a[q]) - st.dtdx[1] * (f1b[q] - f1a[q]) - st.dtdx[2] * (f2b[q] - f2a[q]);
    }
  }
  // B_a^{n+1} = B_a^n - (dt/dx_b (E_c(x + s_b) - E_c(x)) - dt/dx_c (E_b(x + s_c) - E_b(x)))
  R bn[3];
  if (face[0]) bn[0] = ((const R*)p.B[0])[x] - (st.dtdx[1] * (e2y - e2) - st.dtdx[2] * (e1z - e1));
  if (face[1]) bn[1] = ((const R*)p.B[1])[x] - (st.dtdx[2] * (e0z - e0) - st.dtdx[0] * (e2x - e2));
  if (face[2]) bn[2] = ((const R*)p.B[2])[x] - (st.dtdx[0] * (e1x - e1) - st.dtdx[1] * (e0y - e0));
  // edge EMFs for the flux registers
  const bool cap = EmfInline && (p.flags & 1) != 0;
  const bool ce0 = cap && update_edge<0>(p, c), ce1 = cap && update_edge<1>(p, c), ce2 = cap && update_edge<2>(p, c);
  R ec0 = R(0), ec1 = R(0), ec2 = R(0);
  if constexpr (sizeof(R) == 4) {
    if (sc.emf == 1) {  // the values the face updates used
      ec0 = e0;
      ec1 = e1;
      ec2 = e2;
    }
  }
  if (ce0 && !(sizeof(R) == 4 && sc.emf == 1)) ec0 = emf_at<R, 0>(p, x, cs, sc.emf);
  if (ce1 && !(sizeof(R) == 4 && sc.emf == 1)) ec1 = emf_at<R, 1>(p, x, cs, sc.emf);
  if (ce2 && !(sizeof(R) == 4 && sc.emf == 1)) ec2 = emf_at<R, 2>(p, x, cs, sc.emf);
  // without commit the new state goes to the (by now unused) primitive planes
  if (cell) {
#pragma unroll
    for (int q = 0; q < 5; ++q) (commit ? (R*)p.U[q] : arr(scr, p, SC_W + q))[x] = un[q];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (face[a]) (commit ? (R*)p.B[a] : arr(scr, p, SC_W + 5 + a))[x] = bn[a];
  if (ce0) arr(scr, p, SC_ED + 0)[x] = ec0;
  if (ce1) arr(scr, p, SC_ED + 1)[x] = ec1;
  if (ce2) arr(scr, p, SC_ED + 2)[x] = ec2;
}

// ---------------------------------------------------------------- k_floor
// The floors after the update (enabled by p_floor > 0 or rho_floor > 0): one
// thread per cell of the update box.  A density below rho_floor becomes
// rho_floor with M kept and E = p_floor / (gamma - 1) + |M|^2 / (2 rho_floor)
// + |Bc|^2 / 2; otherwise a pressure below p_floor, from the new face field,
// gets E += (p_floor - p) / (gamma - 1).  The oracle's expressions and order.
template <typename R>
__device__ __forceinline__ bool floor_cell(const DPatch& p, int64_t x, const SolverConsts<R>& sc) {
  R u[8], w[8];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = ((const R*)p.U[q])[x];
  u[5] = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
  u[6] = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
  u[7] = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
  cons2prim(u, sc.gm1, w);
  if (sc.rho_floor > R(0) && !(w[0] >= sc.rho_floor)) {
    const R ke = R(0.5) * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / sc.rho_floor;
    const R me = R(0.5) * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
    ((R*)p.U[0])[x] = sc.rho_floor;
    ((R*)p.U[4])[x] = (sc.p_floor / sc.gm1 + ke) + me;
    return true;
  }
  if (sc.p_floor > R(0) && w[4] < sc.p_floor) {
    const R add = (sc.p_floor - w[4]) / sc.gm1;
    ((R*)p.U[4])[x] = u[4] + add;
    return true;
  }
  return false;
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_floor(const DPatch* __restrict__ P, const BlockTask* __restrict__ T,
                                                    SolverConsts<R> sc, unsigned long long* count) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  Cell c;
  if (!region_cell<kMu<R>, kMuT<R>>(p, t.start + threadIdx.x, c)) return;
  const bool f = in_ub(p, 0, c.i, 0, 0) && in_ub(p, 1, c.j, 0, 0) && in_ub(p, 2, c.k, 0, 0) &&
                 floor_cell<R>(p, lin(p, c), sc);
  // one atomic per warp with floored cells
  const unsigned m = __ballot_sync(__activemask(), f);
  if (m && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(count, (unsigned long long)__popc(m));
}

#include "pf.cuh"

// Enqueues the step constants, the fused pass of compiled shape TX x TY and
// the staged EMF / update / floor kernels.
template <typename R, int TX, int TY, int MINB>
cudaError_t launch_pf_shape(const AdvanceArgs& a, R* scr, R* K, const SolverConsts<R>& sc, cudaStream_t s) {
  using L = PfLayout<TX, TY>;
  if (a.npf == 0) return cudaSuccess;
  const size_t smem = sizeof(R) * L::TOTAL;
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    e = cudaFuncSetAttribute(k_pf<R, TX, TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  const KernelTimer* tm = a.timer;
  MHD_TIMED(tm, K_PF, s,
            (k_stepc<R><<<(a.npatches + 127) / 128, 128, 0, s>>>(a.patches, a.npatches, a.d_dt, K),
             k_pf<R, TX, TY, MINB><<<a.npf, L::NT, smem, s>>>(a.patches, a.pf_items, scr, K, sc, a.d_status)));
  constexpr bool inl = kInlineEdges<R>;
  const dim3 gu(a.nblocksu);
  if (!inl) MHD_TIMED(tm, K_EMF, s, (k_emf<R><<<gu, kThreads, 0, s>>>(a.patches, a.tasksu, scr, sc)));
  MHD_TIMED(tm, K_UPDATE, s,
            (k_update<R, inl><<<gu, kThreads, 0, s>>>(a.patches, a.tasksu, scr, sc, K, a.commit ? 1 : 0)));
  if (a.commit && (a.p_floor > 0.0 || a.rho_floor > 0.0))
    MHD_TIMED(tm, K_UPDATE, s, (k_floor<R><<<gu, kThreads, 0, s>>>(a.patches, a.tasksu, sc, a.d_floors)));
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pf(const AdvanceArgs& a, R* scr, R* K, const SolverConsts<R>& sc, cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    static_assert(kNumPf32 == 4 && kPfVariants32[0].tx == 16 && kPfVariants32[1].ty == 12 &&
                      kPfVariants32[2].tx == 24 && kPfVariants32[3].ty == 8,
                  "variant table and dispatch must match");
    switch (a.variant) {
      case 0: return launch_pf_shape<R, 16, 16, 2>(a, scr, K, sc, s);
      case 1: return launch_pf_shape<R, 16, 12, 3>(a, scr, K, sc, s);
      case 2: return launch_pf_shape<R, 24, 8, 3>(a, scr, K, sc, s);
      case 3: return launch_pf_shape<R, 16, 8, 4>(a, scr, K, sc, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    static_assert(kNumPf64 == 1 && kPfVariants64[0].tx == 8, "variant table and dispatch must match");
    if (a.variant != 0) return cudaErrorInvalidValue;
    return launch_pf_shape<R, 8, 8, 2>(a, scr, K, sc, s);
  }
}

// Enqueues the step constants and the stages for the patches of one call;
// K (npatch x kStepConsts elements) is scratch.
template <typename R>
cudaError_t launch_advance(const AdvanceArgs& a, R* scr, R* K, const SolverConsts<R>& sc, cudaStream_t s) {
  if (a.pf) return launch_pf<R>(a, scr, K, sc, s);
  const DPatch* d_patches = a.patches;
  const int npatch = a.npatches, npblocks = a.npblocks;
  const BlockTask *d_tasks = a.tasks, *d_tasks1 = a.tasks1, *d_tasksu = a.tasksu, *d_ptasks = a.ptasks;
  const double* d_dt = a.d_dt;
  int* d_status = a.d_status;
  const KernelTimer* tm = a.timer;
  const bool commit = a.commit;
  if (a.nblocks == 0) return cudaSuccess;
  const dim3 g1(a.nblocks), g1b(a.nblocks1), gu(a.nblocksu);
  if (a.cfl_out) {
    // the step's own CFL dt first (k_prim), then the step constants from it
    MHD_TIMED(tm, K_PRIM, s,
              (k_dt_reset<<<1, 1, 0, s>>>(a.cfl_out),
               k_prim<R, true><<<g1, kThreads, 0, s>>>(d_patches, d_tasks, scr, sc, d_status, a.cfl, a.cfl_out),
               k_stepc<R><<<(npatch + 127) / 128, 128, 0, s>>>(d_patches, npatch, d_dt, K)));
  } else {
    MHD_TIMED(tm, K_PRIM, s,
              (k_stepc<R><<<(npatch + 127) / 128, 128, 0, s>>>(d_patches, npatch, d_dt, K),
               k_prim<R, false><<<g1, kThreads, 0, s>>>(d_patches, d_tasks, scr, sc, d_status, 0.0, nullptr)));
  }
  if (npblocks > 0)
    MHD_TIMED(tm, K_PRED, s, (k_pred_tiled<R><<<npblocks, kThreads, 0, s>>>(d_patches, d_ptasks, scr, sc, K)));
  else
    MHD_TIMED(tm, K_PRED, s, (k_pred<R><<<g1b, kThreads, 0, s>>>(d_patches, d_tasks1, scr, sc, K)));
  constexpr bool inl = kInlineEdges<R>;
  if (!inl) MHD_TIMED(tm, K_EDGE, s, (k_edge<R><<<g1, kThreads, 0, s>>>(d_patches, d_tasks, scr)));
  MHD_TIMED(tm, K_FLUX, s, (k_flux<R><<<g1b, kThreads, 0, s>>>(d_patches, d_tasks1, scr, sc, K)));
  if (!inl) MHD_TIMED(tm, K_EMF, s, (k_emf<R><<<gu, kThreads, 0, s>>>(d_patches, d_tasksu, scr, sc)));
  MHD_TIMED(tm, K_UPDATE, s,
            (k_update<R, inl><<<gu, kThreads, 0, s>>>(d_patches, d_tasksu, scr, sc, K, commit ? 1 : 0)));
  if (commit && (a.p_floor > 0.0 || a.rho_floor > 0.0))
    MHD_TIMED(tm, K_UPDATE, s, (k_floor<R><<<gu, kThreads, 0, s>>>(d_patches, d_tasksu, sc, a.d_floors)));
  return cudaGetLastError();
}

#include "fused.cuh"

// Enqueues the step constants, the fused kernel (as many CTAs as fit on the
// device, at most one per item) and the copy-back of the new state.
template <typename R, int BX, int BY, int NT>
cudaError_t launch_fused(const AdvanceArgs& a, const SolverConsts<R>& sc, cudaStream_t s) {
  if (a.nitems == 0) return cudaSuccess;
  const size_t smem = sizeof(R) * FusedLayout<BX, BY>::TOTAL;
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!configured[dev]) {
    e = cudaFuncSetAttribute(k_fused<R, BX, BY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  int nsm = 0, per_sm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<R, BX, BY, NT>, NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = a.nitems < nsm * per_sm ? a.nitems : nsm * per_sm;
  R* K = (R*)a.stepc;
  MHD_TIMED(a.timer, K_FUSED, s,
            (k_stepc<R><<<(a.npatches + 127) / 128, 128, 0, s>>>(a.patches, a.npatches, a.d_dt, K),
             cudaMemsetAsync(a.counter, 0, sizeof(int), s),
             k_fused<R, BX, BY, NT><<<grid, NT, smem, s>>>(a.patches, a.items, a.nitems, a.counter, (R*)a.scratch,
                                                           K, sc, a.d_status)));
  if (a.commit || a.commit_patches)
    MHD_TIMED(a.timer, K_COMMIT, s,
              (k_commit<R><<<a.nctasks, kThreads, 0, s>>>(a.commit && !a.commit_patches ? a.patches : a.commit_patches,
                                                          a.ctasks, (const R*)a.scratch)));
  if (a.commit && (a.p_floor > 0.0 || a.rho_floor > 0.0))
    MHD_TIMED(a.timer, K_COMMIT, s,
              (k_floor<R><<<a.nctasks, kThreads, 0, s>>>(a.patches, a.ctasks, sc, a.d_floors)));
  return cudaGetLastError();
}

template <typename R> cudaError_t launch_fused_variant(const AdvanceArgs& a, const SolverConsts<R>& sc, cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    static_assert(kNumFused32 == 4, "variant table and dispatch must match");
    switch (a.variant) {
      case 0: return launch_fused<R, 16, 16, 512>(a, sc, s);
      case 1: return launch_fused<R, 16, 16, 384>(a, sc, s);
      case 2: return launch_fused<R, 16, 12, 384>(a, sc, s);
      case 3: return launch_fused<R, 24, 8, 384>(a, sc, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    static_assert(kNumFused64 == 1, "variant table and dispatch must match");
    if (a.variant != 0) return cudaErrorInvalidValue;
    return launch_fused<R, 8, 8, 128>(a, sc, s);
  }
}

// The floors over the interiors of a call's patches (k = 0, tasks over
// [lo, hi + 1] as the update's).
template <typename R> cudaError_t run_floor(const AdvanceArgs& a, cudaStream_t s) {
  SolverConsts<R> sc{};
  sc.gamma = (R)a.gamma;
  sc.gm1 = sc.gamma - R(1);
  sc.p_floor = (R)a.p_floor;
  sc.rho_floor = (R)a.rho_floor;
  if (a.nblocksu == 0) return cudaSuccess;
  k_floor<R><<<a.nblocksu, kThreads, 0, s>>>(a.patches, a.tasksu, sc, a.d_floors);
  return cudaGetLastError();
}

// Solver constants in the arithmetic type, then the launches.
template <typename R> cudaError_t run_advance(const AdvanceArgs& a, cudaStream_t s) {
  SolverConsts<R> sc;
  sc.gamma = (R)a.gamma;
  sc.gm1 = sc.gamma - R(1);
  sc.igm1 = R(1) / sc.gm1;
  sc.eps_up = (R)a.eps_up;
  sc.limiter = a.limiter;
  sc.emf = a.emf;
  sc.p_floor = (R)a.p_floor;
  sc.rho_floor = (R)a.rho_floor;
  if (a.fused) return launch_fused_variant<R>(a, sc, s);
  return launch_advance<R>(a, (R*)a.scratch, (R*)a.stepc, sc, s);
}

}  // namespace MHD_ADVANCE_NS
}  // namespace mhd
