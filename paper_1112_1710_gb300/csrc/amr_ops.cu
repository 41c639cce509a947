// amr_ops.cu -- level operations of the subcycled AMR step (refinement ratio
// 2; Sec. 2.2 Prolongation, Restriction, flux synchronisation): prolongation
// into ghost zones, restriction, FP64 flux-register capture, deposit of the
// register differences into correction planes, and the correction itself.
// Built with --fmad=false; every expression follows one fixed evaluation
// order.  A fine patch is aligned to its coarse level: fine global index =
// 2 * coarse global index + {0, 1}.
#include <cuda_runtime.h>

#include <cstdint>

#include "amr.h"
#include "common.cuh"
#include "physics.cuh"

// Blocks per SM the FP32 prolongation is compiled for (its registers per
// thread: 80 at three blocks, with some spilling, the compiler's 112 at two).
#ifndef MHD_PROLONG_MINB
#define MHD_PROLONG_MINB 2
#endif

namespace mhd {

namespace {

__device__ __forceinline__ int64_t lin3(const DPatch& p, int i, int j, int k) {
  return (int64_t)i + (int64_t)j * p.s1 + (int64_t)k * p.s2;
}
__device__ __forceinline__ int64_t sof(const DPatch& p, int d) {
  return d == 0 ? (int64_t)1 : (d == 1 ? p.s1 : p.s2);
}
// is the axis-a face with array index ai a face of p's interior?
__device__ __forceinline__ bool own_face(const DPatch& p, const int* ai, int a) {
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int top = (e == a) ? p.g + p.n[e] : p.g + p.n[e] - 1;
    if (ai[e] < p.g || ai[e] > top) return false;
  }
  return true;
}
// does the axis-a face with array index ai exist in p's arrays?
__device__ __forceinline__ bool face_exists(const DPatch& p, const int* ai, int a) {
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int top = (e == a) ? p.N[e] : p.N[e] - 1;
    if (ai[e] < 0 || ai[e] > top) return false;
  }
  return true;
}
template <typename R> __device__ __forceinline__ R minmod(R a, R b) { return limiter<R>(1, a, b); }

// thermal energy E - |M|^2/(2 rho) - |Bc|^2/2 of cell x (Bc = face means)
template <typename R> __device__ __forceinline__ R thermal(const DPatch& p, int64_t x) {
  const R rho = ((const R*)p.U[0])[x];
  const R mx = ((const R*)p.U[1])[x], my = ((const R*)p.U[2])[x], mz = ((const R*)p.U[3])[x];
  R ke = R(0.5) * (mx * mx + my * my + mz * mz) / rho;
  R bx = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
  R by = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
  R bz = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
  R me = R(0.5) * (bx * bx + by * by + bz * bz);
  return ((const R*)p.U[4])[x] - ke - me;
}

// fine axis-a face at position pos (0 lower coarse face, 1 inner, 2 upper)
// and transverse sub-indices sub[] of the reconstruction in one coarse cell
template <typename R>
__device__ __forceinline__ R pface(int a, int pos, const int* sub, const R (&m)[3][2], const R (&qs)[3][2][3],
                                   const R (&lin)[3][3], const R (&c0)[3]) {
  const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
  if (pos == 1) {
    R sl = sub[lo_t] ? R(0.5) * lin[a][lo_t] : R(-0.5) * lin[a][lo_t];
    R sh = sub[hi_t] ? R(0.5) * lin[a][hi_t] : R(-0.5) * lin[a][hi_t];
    return c0[a] + sl + sh;
  }
  const int sd = pos == 2;
  R sl = sub[lo_t] ? qs[a][sd][lo_t] : -qs[a][sd][lo_t];
  R sh = sub[hi_t] ? qs[a][sd][hi_t] : -qs[a][sd][hi_t];
  return m[a][sd] + sl + sh;
}

__device__ __forceinline__ void box_cell(const int32_t* lo, const int32_t* ext, int e, int* c) {
  c[0] = lo[0] + e % ext[0];
  c[1] = lo[1] + (e / ext[0]) % ext[1];
  c[2] = lo[2] + e / (ext[0] * ext[1]);
}

// Two consecutive elements x, x + 1 of an array (x even where vec is set),
// each written if its flag is set; one vector store when both are.
template <typename R> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };
template <typename R>
__device__ __forceinline__ void st_pair(R* p, int64_t x, R v0, R v1, bool w0, bool w1, bool vec) {
  if (vec && w0 && w1) {
    typename Pair<R>::T v;
    v.x = v0;
    v.y = v1;
    *reinterpret_cast<typename Pair<R>::T*>(p + x) = v;
    return;
  }
  if (w0) p[x] = v0;
  if (w1) p[x + 1] = v1;
}
// Are all eight arrays of p aligned for pair stores at even indices?
template <typename R> __device__ __forceinline__ bool pair_aligned(const DPatch& p) {
  uintptr_t o = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) o |= (uintptr_t)p.U[q];
#pragma unroll
  for (int a = 0; a < 3; ++a) o |= (uintptr_t)p.B[a];
  return (o & (2 * sizeof(R) - 1)) == 0 && (p.s1 & 1) == 0 && (p.s2 & 1) == 0;
}

// ---------------------------------------------------------------- ghost copy
// Cell c of the top layer of a box along axis a (the item's element e runs
// over the two transverse axes, lower one fastest).
__device__ __forceinline__ void top_cell(const int32_t* lo, const int32_t* ext, int a, int e, int* c) {
  const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  const int u = t1 < t2 ? t1 : t2, v = t1 < t2 ? t2 : t1;
  c[a] = lo[a] + ext[a] - 1;
  c[u] = lo[u] + e % ext[u];
  c[v] = lo[v] + e / ext[u];
}

// One launch for all copies of a fill, one warp per task: a group of rows
// (x runs) of one copy box, the lanes along x (W = min(ext_x, 32) lanes per
// row, 32 / W rows side by side; boxes wider than 32 are cut into x chunks),
// kGhostRows such groups per task, their loads issued together, then their
// stores.  Each element writes its five cell values (inside the
// destination's arrays), its lower face along each axis, and on the box's
// top layer along an axis its upper face; no face of the destination's
// interior is written, nor one outside its face arrays.  A face that is the
// upper face of one box's top layer and the lower face of another's bottom
// layer takes the first box's value: the second skips it, from the
// rectangles of its bottom layer the host lists (the transverse extent it
// shares with a box whose top layer lies directly below it), so that no two
// threads write one element.
template <typename R> constexpr int kGhostRows = sizeof(R) == 4 ? 3 : 2;

__device__ __forceinline__ bool excluded(const DCopy& cp, const DExcl* __restrict__ X, const int* di, int a) {
  const int u = a == 0 ? 1 : 0, v = a == 2 ? 1 : 2;
  for (int r = cp.xr; r < cp.xr + cp.nx; ++r) {
    const DExcl x = X[r];
    if (x.axis == a && di[u] >= x.lo[0] && di[u] <= x.hi[0] && di[v] >= x.lo[1] && di[v] <= x.hi[1]) return true;
  }
  return false;
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 3) k_ghost2(const DPatch* __restrict__ P, const DCopy* __restrict__ C,
                                                        const DExcl* __restrict__ X,
                                                        const GhostTask* __restrict__ T, int ntasks) {
  constexpr int GR = kGhostRows<R>;
  const int wt = (int)blockIdx.x * (kThreads / 32) + (int)(threadIdx.x >> 5);
  if (wt >= ntasks) return;
  const int lane = (int)(threadIdx.x & 31);
  const GhostTask t = T[wt];
  const DCopy cp = C[t.copy];
  const DPatch& d = P[cp.dst];
  const DPatch& s = P[cp.src];
  const int W = cp.ext[0] < 32 ? cp.ext[0] : 32;
  int xr;
  const int rr = divmod24(lane, W, xr);
  const int RW = 32 / W;  // rows side by side
  const int xx = t.x0 + xr;
  const bool on = rr < RW && xx < cp.ext[0];
  const int nrows = cp.ext[1] * cp.ext[2];
  const int64_t ds1 = d.s1, ds2 = d.s2, ss1 = s.s1, ss2 = s.s2;
  const int g = d.g;
  // Per axis, with c the element's index along it: in the arrays (0 <= c <
  // N), on the arrays' extra face plane (c == N), inside the interior (g <=
  // c < g + n), on its upper face plane (c == g + n).  A lower face along a
  // exists if c_a is in the arrays or on the extra plane and the other two
  // are in the arrays; it is the interior's own if c_a is inside or on the
  // upper plane and the other two are inside.  The upper face of a cell is
  // the lower face of c_a + 1.
  const int i = cp.lo[0] + xx;
  const bool xin = i >= 0 && i < d.N[0], xN = i == d.N[0];
  const bool xint = i >= g && i < g + d.n[0], xtop = i == g + d.n[0];
  const bool xin1 = i >= -1 && i < d.N[0], xint1 = i >= g - 1 && i < g + d.n[0];  // for c_x + 1
  const bool xbot = xx == 0, xlast = xx == cp.ext[0] - 1;
  R u[GR][5], b[GR][3];
  int64_t xd[GR], xs[GR];
  unsigned w[GR];  // bit 0: the cell; bit 1 + a: the lower face along a; bit 4 + a: the upper face
  // loads first: a store would order every later load of a may-alias array
#pragma unroll
  for (int gg = 0; gg < GR; ++gg) {
    const int r = t.row0 + gg * RW + rr;
    w[gg] = 0u;
    xd[gg] = xs[gg] = 0;
    if (!on || r >= nrows) continue;
    int yy;
    const int zz = divmod24(r, cp.ext[1], yy);
    const int j = cp.lo[1] + yy, k = cp.lo[2] + zz;
    const bool yin = j >= 0 && j < d.N[1], yN = j == d.N[1];
    const bool zin = k >= 0 && k < d.N[2], zN = k == d.N[2];
    const bool yint = j >= g && j < g + d.n[1], ytop = j == g + d.n[1];
    const bool zint = k >= g && k < g + d.n[2], ztop = k == g + d.n[2];
    xd[gg] = (int64_t)i + (int64_t)j * ds1 + (int64_t)k * ds2;
    xs[gg] = (int64_t)(i + cp.off[0]) + (int64_t)(j + cp.off[1]) * ss1 + (int64_t)(k + cp.off[2]) * ss2;
    const bool ex[3] = {(xin || xN) && yin && zin, xin && (yin || yN) && zin, xin && yin && (zin || zN)};
    const bool own[3] = {(xint || xtop) && yint && zint, xint && (yint || ytop) && zint,
                         xint && yint && (zint || ztop)};
    const bool bot[3] = {xbot, yy == 0, zz == 0};
    if (xin && yin && zin) {
      w[gg] |= 1u;
#pragma unroll
      for (int q = 0; q < 5; ++q) u[gg][q] = ((const R*)s.U[q])[xs[gg]];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!ex[a] || own[a]) continue;
      if (bot[a] && cp.nx > 0) {
        const int di[3] = {i, j, k};
        if (excluded(cp, X, di, a)) continue;
      }
      w[gg] |= 2u << a;
      b[gg][a] = ((const R*)s.B[a])[xs[gg]];
    }
    // upper faces of the top layers
    if (xlast && xin1 && yin && zin && !(xint1 && yint && zint)) w[gg] |= 16u;
    if (yy == cp.ext[1] - 1 && xin && j >= -1 && j < d.N[1] && zin &&
        !(xint && j >= g - 1 && j < g + d.n[1] && zint))
      w[gg] |= 32u;
    if (zz == cp.ext[2] - 1 && xin && yin && k >= -1 && k < d.N[2] &&
        !(xint && yint && k >= g - 1 && k < g + d.n[2]))
      w[gg] |= 64u;
  }
#pragma unroll
  for (int gg = 0; gg < GR; ++gg) {
    if (w[gg] & 1u)
#pragma unroll
      for (int q = 0; q < 5; ++q) ((R*)d.U[q])[xd[gg]] = u[gg][q];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (w[gg] & (2u << a)) ((R*)d.B[a])[xd[gg]] = b[gg][a];
  }
  // the top layers' upper faces (a small share of the elements)
#pragma unroll
  for (int gg = 0; gg < GR; ++gg) {
    if (w[gg] & 16u) ((R*)d.B[0])[xd[gg] + 1] = ((const R*)s.B[0])[xs[gg] + 1];
    if (w[gg] & 32u) ((R*)d.B[1])[xd[gg] + ds1] = ((const R*)s.B[1])[xs[gg] + ss1];
    if (w[gg] & 64u) ((R*)d.B[2])[xd[gg] + ds2] = ((const R*)s.B[2])[xs[gg] + ss2];
  }
}

// ---------------------------------------------------------------- prolongation
template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? MHD_PROLONG_MINB : 1) k_prolong(const DPatch* __restrict__ PC,
                                                                        const DPatch* __restrict__ PF,
                                                                        const DBoxItem* __restrict__ items,
                                                                        const BlockTask* __restrict__ T,
                                                                        const int64_t* __restrict__ starts,
                                                                        int nitems, int packed) {
  int ii, e;
  if (!list_elem(T[blockIdx.x], starts, nitems, packed, ii, e)) return;
  const DBoxItem it = items[ii];
  int C3[3];
  box_cell(it.lo, it.ext, e, C3);
  const DPatch& pc = PC[it.a];
  const DPatch& pf = PF[it.b];
  const int ci[3] = {C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]};
  const int64_t c = lin3(pc, ci[0], ci[1], ci[2]);
  R uc[4], h[4][3], he[3];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R* Uq = (const R*)pc.U[q];
    uc[q] = Uq[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R a = uc[q] - Uq[c - sof(pc, d)];
      R b = Uq[c + sof(pc, d)] - uc[q];
      h[q][d] = R(0.25) * minmod(a, b);
    }
  }
  const R ec = thermal<R>(pc, c);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R a = ec - thermal<R>(pc, c - sof(pc, d));
    R b = thermal<R>(pc, c + sof(pc, d)) - ec;
    he[d] = R(0.25) * minmod(a, b);
  }
  R m[3][2], qs[3][2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R* Ba = (const R*)pc.B[a];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int64_t f = c + (sd ? sof(pc, a) : 0);
      m[a][sd] = Ba[f];
#pragma unroll
      for (int tt = 0; tt < 3; ++tt) {
        if (tt == a) {
          qs[a][sd][tt] = R(0);
          continue;
        }
        R lo = m[a][sd] - Ba[f - sof(pc, tt)];
        R hi = Ba[f + sof(pc, tt)] - m[a][sd];
        qs[a][sd][tt] = R(0.25) * minmod(lo, hi);
      }
    }
  }
  R lin[3][3], crs[3][3], sq[3], c0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int tt = 0; tt < 3; ++tt) {
      if (tt == a) {
        lin[a][tt] = R(0);
        crs[a][tt] = R(0);
        continue;
      }
      lin[a][tt] = qs[a][1][tt] + qs[a][0][tt];
      crs[a][tt] = qs[a][1][tt] - qs[a][0][tt];
    }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    sq[a] = R(-0.5) * (crs[b][a] + crs[cc][a]);
    c0[a] = R(0.5) * (m[a][0] + m[a][1]) - sq[a];
  }
  // The fine cells in x pairs (fa = 0, 1) for each (fb, fc), all unrolled so
  // that every index into the reconstruction is a compile-time constant; the
  // two values of a pair are stored together where the pair is aligned.
  const int f0x = 2 * C3[0] - pf.glo[0];
  const bool vec = ((f0x & 1) == 0) && pair_aligned<R>(pf);
  // per axis and sub-index: the fine index inside the interior, on its upper
  // face plane (a lower face of a fine cell is the patch's own when its
  // normal index is one of the two and the other two are inside)
  bool inI[3][2], onT[3][2];
#pragma unroll
  for (int e = 0; e < 3; ++e)
#pragma unroll
    for (int sb = 0; sb < 2; ++sb) {
      const int f = 2 * C3[e] + sb - pf.glo[e];
      inI[e][sb] = f >= pf.g && f < pf.g + pf.n[e];
      onT[e][sb] = f == pf.g + pf.n[e];
    }
#pragma unroll
  for (int fc = 0; fc < 2; ++fc)
#pragma unroll
    for (int fb = 0; fb < 2; ++fb) {
      const int fy = 2 * C3[1] + fb - pf.glo[1], fz = 2 * C3[2] + fc - pf.glo[2];
      const int64_t x = lin3(pf, f0x, fy, fz);
      R uf[2][4], en[2], lf[2][3];
#pragma unroll
      for (int fa = 0; fa < 2; ++fa) {
        const int sub[3] = {fa, fb, fc};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          R u = uc[q];
          u = u + (fa ? h[q][0] : -h[q][0]);
          u = u + (fb ? h[q][1] : -h[q][1]);
          u = u + (fc ? h[q][2] : -h[q][2]);
          uf[fa][q] = u;
        }
        R bc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lf[fa][a] = pface<R>(a, sub[a], sub, m, qs, lin, c0);
          const R f1 = pface<R>(a, sub[a] + 1, sub, m, qs, lin, c0);
          bc[a] = R(0.5) * (lf[fa][a] + f1);
        }
        R e = ec;
        e = e + (fa ? he[0] : -he[0]);
        e = e + (fb ? he[1] : -he[1]);
        e = e + (fc ? he[2] : -he[2]);
        const R kef = R(0.5) * (uf[fa][1] * uf[fa][1] + uf[fa][2] * uf[fa][2] + uf[fa][3] * uf[fa][3]) / uf[fa][0];
        const R mef = R(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
        en[fa] = e + kef + mef;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) st_pair<R>((R*)pf.U[q], x, uf[0][q], uf[1][q], true, true, vec);
      st_pair<R>((R*)pf.U[4], x, en[0], en[1], true, true, vec);
      // lower faces of both cells along each axis, never the patch's own
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bool own[2];
#pragma unroll
        for (int fa = 0; fa < 2; ++fa) {
          const int sub[3] = {fa, fb, fc};
          const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
          own[fa] = (inI[a][sub[a]] || onT[a][sub[a]]) && inI[b1][sub[b1]] && inI[b2][sub[b2]];
        }
        st_pair<R>((R*)pf.B[a], x, lf[0][a], lf[1][a], !own[0], !own[1], vec);
      }
      // upper faces of cells in the array's last layer along an axis
#pragma unroll
      for (int fa = 0; fa < 2; ++fa) {
        const int sub[3] = {fa, fb, fc};
        const int fi[3] = {f0x + fa, fy, fz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (fi[a] != pf.N[a] - 1) continue;
          int fu[3] = {fi[0], fi[1], fi[2]};
          fu[a] += 1;
          if (own_face(pf, fu, a)) continue;
          ((R*)pf.B[a])[x + fa + sof(pf, a)] = pface<R>(a, sub[a] + 1, sub, m, qs, lin, c0);
        }
      }
    }
}

// ---------------------------------------------------------------- restriction
template <typename R>
__global__ void __launch_bounds__(kThreads) k_restrict(const DPatch* __restrict__ PF, const DPatch* __restrict__ PC,
                                                       const DBoxItem* __restrict__ items,
                                                       const BlockTask* __restrict__ T,
                                                       const int64_t* __restrict__ starts, int nitems, int packed,
                                                       int pass) {
  // pass 0: every cell of an item box; pass 1: the top layer of an item box
  // along one axis (items: item x axis)
  int ii, e;
  if (!list_elem(T[blockIdx.x], starts, nitems, packed, ii, e)) return;
  const int bi = pass == 0 ? ii : ii / 3;
  const int ax = pass == 0 ? -1 : ii - 3 * bi;
  const DBoxItem it = items[bi];
  int C3[3];
  if (pass == 0) box_cell(it.lo, it.ext, e, C3);
  else top_cell(it.lo, it.ext, ax, e, C3);
  const DPatch& pf = PF[it.a];
  const DPatch& pc = PC[it.b];
  const int ca0[3] = {C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]};
  const bool inside = ca0[0] >= pc.g && ca0[0] < pc.g + pc.n[0] && ca0[1] >= pc.g && ca0[1] < pc.g + pc.n[1] &&
                      ca0[2] >= pc.g && ca0[2] < pc.g + pc.n[2];
  if (pass == 0 && inside) {
    const int64_t c = lin3(pc, ca0[0], ca0[1], ca0[2]);
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const R* Fq = (const R*)pf.U[q];
      R s = R(0);
      bool first = true;
      for (int fc = 0; fc < 2; ++fc)
        for (int fb = 0; fb < 2; ++fb)
          for (int fa = 0; fa < 2; ++fa) {
            R v = Fq[lin3(pf, 2 * C3[0] + fa - pf.glo[0], 2 * C3[1] + fb - pf.glo[1], 2 * C3[2] + fc - pf.glo[2])];
            s = first ? v : s + v;
            first = false;
          }
      ((R*)pc.U[q])[c] = R(0.125) * s;
    }
  }
  const int chi[3] = {it.lo[0] + it.ext[0] - 1, it.lo[1] + it.ext[1] - 1, it.lo[2] + it.ext[2] - 1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
    const int up = pass;
    if (up && (a != ax || C3[a] != chi[a])) continue;
    int cf[3] = {ca0[0], ca0[1], ca0[2]};
    cf[a] += up;
    if (!own_face(pc, cf, a)) continue;
    const R* Fa = (const R*)pf.B[a];
    R s = R(0);
    bool first = true;
    for (int j2 = 0; j2 < 2; ++j2)
      for (int j1 = 0; j1 < 2; ++j1) {
        int f[3];
        f[a] = 2 * (C3[a] + up);
        f[lo_t] = 2 * C3[lo_t] + j1;
        f[hi_t] = 2 * C3[hi_t] + j2;
        R v = Fa[lin3(pf, f[0] - pf.glo[0], f[1] - pf.glo[1], f[2] - pf.glo[2])];
        s = first ? v : s + v;
        first = false;
      }
    ((R*)pc.B[a])[lin3(pc, cf[0], cf[1], cf[2])] = R(0.25) * s;
  }
}

// ---------------------------------------------------------------- capture
// dst = (or +=) dt * F_q on the axis faces (5 planes) / dt * E_axis on edges
template <typename R>
__global__ void __launch_bounds__(kThreads) k_capture(const DPatch* __restrict__ P, const DCapture* __restrict__ C,
                                                      const BlockTask* __restrict__ T,
                                                      const int64_t* __restrict__ starts, int nitems, int packed,
                                                      const R* scr, const double* d_dt) {
  int ii, e;
  if (!list_elem(T[blockIdx.x], starts, nitems, packed, ii, e)) return;
  const DCapture cp = C[ii];
  const int64_t nv = (int64_t)cp.ext[0] * cp.ext[1] * cp.ext[2];
  int ai[3];
  box_cell(cp.lo, cp.ext, e, ai);
  const DPatch& p = P[cp.patch];
  const double dt = (*d_dt) * p.dt_scale;
  const int64_t x = lin3(p, ai[0], ai[1], ai[2]);
  if (cp.kind == 0) {
    // the five components of the face's flux group as whole vectors
    const R* F = scr + p.scr + (int64_t)(SC_F + cp.axis * 8) * p.snelem;
    R f[5];
    if constexpr (sizeof(R) == 4) {
      const float4 a = reinterpret_cast<const float4*>(F)[x];
      f[0] = a.x;
      f[1] = a.y;
      f[2] = a.z;
      f[3] = a.w;
      f[4] = reinterpret_cast<const float4*>(F + 4 * p.snelem)[x].x;
    } else {
      const double2 a = reinterpret_cast<const double2*>(F)[x];
      const double2 b = reinterpret_cast<const double2*>(F + 2 * p.snelem)[x];
      f[0] = a.x;
      f[1] = a.y;
      f[2] = b.x;
      f[3] = b.y;
      f[4] = *vgroup_at(F, p.snelem, x, 4);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double v = dt * (double)f[q];
      double* o = cp.dst + (int64_t)q * nv + e;
      *o = cp.mode ? *o + v : v;
    }
  } else {
    const R* Ed = scr + p.scr + (int64_t)(SC_ED + cp.axis) * p.snelem;
    const double v = dt * (double)Ed[x];
    double* o = cp.dst + e;
    *o = cp.mode ? *o + v : v;
  }
}

// ---------------------------------------------------------------- reflux
// Sets flag bit `bit` of element x of a coarse patch (flags are bytes packed
// four to a word; neighbouring elements of other threads share words); the
// thread that sets the element's first bit appends it to the call's list.
// The lanes of a warp that append take one run of the list with one atomic,
// in lane order, so that the list keeps the deposits' spatial order within a
// warp (neighbouring entries are neighbouring elements for the correction).
__device__ __forceinline__ void mark(unsigned int* flags, int64_t x, unsigned int bit, const RefluxList& L,
                                     int corr_idx) {
  const int sh = 8 * (int)(x & 3);
  const unsigned int old = atomicOr(flags + (x >> 2), bit << sh);
  const bool first = ((old >> sh) & 0xFFu) == 0u;
  const unsigned int act = __activemask();
  const unsigned int m = __ballot_sync(act, first);
  if (!m) return;
  const int lane = (int)(threadIdx.x & 31);
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(L.count, (unsigned long long)__popc(m));
  base = __shfl_sync(act, base, leader);
  if (first) {
    const unsigned long long i = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    if (i < L.capacity) L.entries[i] = ((unsigned long long)corr_idx << 40) | (unsigned long long)x;
  }
}

// After the correction: zeroes the plane elements the deposits wrote, so the
// correction planes are zero again between calls (only C/F elements are ever
// non-zero, and only during a call).
__global__ void __launch_bounds__(kThreads) k_unset(const DPatch* __restrict__ PC, const DDeposit* __restrict__ D,
                                                    const BlockTask* __restrict__ T) {
  const BlockTask t = T[blockIdx.x];
  const DDeposit dp = D[t.patch];
  const int e = t.start + threadIdx.x;
  if (e >= dp.ext[0] * dp.ext[1] * dp.ext[2]) return;
  int C3[3];
  box_cell(dp.lo, dp.ext, e, C3);
  const DPatch& pc = PC[dp.coarse];
  const int64_t c = lin3(pc, C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]);
  if (dp.kind == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) dp.corr[(int64_t)(dp.axis * 5 + q) * pc.nelem + c] = 0.0;
  } else {
    dp.corr[(int64_t)(15 + dp.axis) * pc.nelem + c] = 0.0;
  }
}

__global__ void __launch_bounds__(kThreads) k_deposit(const DPatch* __restrict__ PC,
                                                      const DDeposit* __restrict__ D,
                                                      const BlockTask* __restrict__ T, RefluxList L) {
  const BlockTask t = T[blockIdx.x];
  const DDeposit dp = D[t.patch];
  const int e = t.start + threadIdx.x;
  const int64_t cn = (int64_t)dp.ext[0] * dp.ext[1] * dp.ext[2];
  if (e >= cn) return;
  int C3[3];
  box_cell(dp.lo, dp.ext, e, C3);
  const DPatch& pc = PC[dp.coarse];
  const int64_t c = lin3(pc, C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]);
  const int64_t fn = (int64_t)dp.fext[0] * dp.fext[1] * dp.fext[2];
  if (dp.mode == 1) {
    // synchronisation of a face / edge shared by two patches of one level:
    // the other patch's register over the same box; dF = 0.5 (other - own)
    const int64_t fo = (int64_t)(C3[0] - dp.flo[0]) +
                       (int64_t)dp.fext[0] * ((C3[1] - dp.flo[1]) + (int64_t)dp.fext[1] * (C3[2] - dp.flo[2]));
    if (dp.kind == 0) {
#pragma unroll
      for (int q = 0; q < 5; ++q)
        dp.corr[(int64_t)(dp.axis * 5 + q) * pc.nelem + c] = 0.5 * (dp.fine[q * fn + fo] - dp.creg[q * cn + e]);
    } else {
      dp.corr[(int64_t)(15 + dp.axis) * pc.nelem + c] = 0.5 * (dp.fine[fo] - dp.creg[e]);
    }
  } else if (dp.kind == 0) {
    const int d = dp.axis;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
    for (int q = 0; q < 5; ++q) {
      double s = 0.0;
      bool first = true;
      for (int j2 = 0; j2 < 2; ++j2)
        for (int j1 = 0; j1 < 2; ++j1) {
          int f[3];
          f[d] = 2 * C3[d];
          f[lo_t] = 2 * C3[lo_t] + j1;
          f[hi_t] = 2 * C3[hi_t] + j2;
          const int64_t fo = (int64_t)(f[0] - dp.flo[0]) +
                             (int64_t)dp.fext[0] * ((f[1] - dp.flo[1]) + (int64_t)dp.fext[1] * (f[2] - dp.flo[2]));
          const double v = dp.fine[q * fn + fo];
          s = first ? v : s + v;
          first = false;
        }
      dp.corr[(int64_t)(d * 5 + q) * pc.nelem + c] = 0.25 * s - dp.creg[q * cn + e];
    }
  } else {
    const int a = dp.axis;
    double s = 0.0;
    for (int seg = 0; seg < 2; ++seg) {
      int f[3] = {2 * C3[0], 2 * C3[1], 2 * C3[2]};
      f[a] += seg;
      const int64_t fo = (int64_t)(f[0] - dp.flo[0]) +
                         (int64_t)dp.fext[0] * ((f[1] - dp.flo[1]) + (int64_t)dp.fext[1] * (f[2] - dp.flo[2]));
      s = seg ? s + dp.fine[fo] : dp.fine[fo];
    }
    dp.corr[(int64_t)(15 + a) * pc.nelem + c] = 0.5 * s - dp.creg[e];
  }
  // flag the elements whose correction reads this one: for a face along d the
  // cells above and below it; for an edge along a the faces that difference it
  const int ai[3] = {C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]};
  if (dp.kind == 0) {
    const int d = dp.axis;
    mark(dp.flags, c, 1u, L, dp.corr_idx);
    if (ai[d] > 0) mark(dp.flags, c - sof(pc, d), 1u, L, dp.corr_idx);
  } else {
    const int e2 = dp.axis;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (f == e2) continue;
      const int b = (f + 1) % 3, cc = (f + 2) % 3;
      const int sh = e2 == cc ? b : cc;  // the face x reads the edge at x and at x + s_sh
      mark(dp.flags, c, 2u << f, L, dp.corr_idx);
      if (ai[sh] > 0) mark(dp.flags, c - sof(pc, sh), 2u << f, L, dp.corr_idx);
    }
  }
}

// Applies the correction planes to the flagged elements of the coarse
// patches, one thread per entry of the call's list (the elements the deposits
// flagged, each once): the cell if it is an interior cell, the faces that are
// interior faces (region: interior grown by one on the upper side; flagged
// ghost elements are only cleared).  Each thread clears its element's flags.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_correct(const DPatch* __restrict__ PC, const DCorr* __restrict__ C,
                                                      RefluxList L) {
  const unsigned long long li = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  if (li >= *L.count || li >= L.capacity) return;
  const unsigned long long ent = L.entries[li];
  const DCorr cr = C[(int)(ent >> 40)];
  const DPatch& p = PC[cr.patch];
  const int64_t c = (int64_t)(ent & ((1ull << 40) - 1));
  const unsigned int fl = cr.flags[c];
  cr.flags[c] = 0;
  const int ai[3] = {(int)(c % p.s1), (int)((c / p.s1) % (p.s2 / p.s1)), (int)(c / p.s2)};
  if (ai[0] < p.g || ai[0] > p.g + p.n[0] || ai[1] < p.g || ai[1] > p.g + p.n[1] || ai[2] < p.g ||
      ai[2] > p.g + p.n[2])
    return;
  // Elements no deposit touched see only zero plane differences, and
  // u - 0/dx - 0/dx - 0/dx == u: they are not in the list, with the same
  // bits as applying the correction; so are zero differences below.
  if (!fl) return;
  const double* K = cr.base;
  const int64_t ne = p.nelem;
  const bool cell = (fl & 1u) && ai[0] < p.g + p.n[0] && ai[1] < p.g + p.n[1] && ai[2] < p.g + p.n[2];
  if (cell) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const double d0 = K[(0 * 5 + q) * ne + c + 1] - K[(0 * 5 + q) * ne + c];
      const double d1 = K[(1 * 5 + q) * ne + c + p.s1] - K[(1 * 5 + q) * ne + c];
      const double d2 = K[(2 * 5 + q) * ne + c + p.s2] - K[(2 * 5 + q) * ne + c];
      if (d0 == 0.0 && d1 == 0.0 && d2 == 0.0) continue;
      R* Uq = (R*)p.U[q];
      double u = (double)Uq[c];
      // FP64 state: the oracle's divisions; FP32 state (rounded to FP32 at the
      // end): multiplications by 1/dx, a tenth of the FP64 pipe work
      if (sizeof(R) == 8) u = u - d0 / p.dx[0] - d1 / p.dx[1] - d2 / p.dx[2];
      else u = u - d0 * p.rdx[0] - d1 * p.rdx[1] - d2 * p.rdx[2];
      Uq[c] = (R)u;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(fl & (2u << a)) || !own_face(p, ai, a)) continue;
    const int b = (a + 1) % 3, cc = (a + 2) % 3;
    const double dEc = K[(15 + cc) * ne + c + sof(p, b)] - K[(15 + cc) * ne + c];
    const double dEb = K[(15 + b) * ne + c + sof(p, cc)] - K[(15 + b) * ne + c];
    if (dEc == 0.0 && dEb == 0.0) continue;
    R* Ba = (R*)p.B[a];
    if (sizeof(R) == 8) Ba[c] = (R)((double)Ba[c] - (dEc / p.dx[b] - dEb / p.dx[cc]));
    else Ba[c] = (R)((double)Ba[c] - (dEc * p.rdx[b] - dEb * p.rdx[cc]));
  }
}

}  // namespace

int ghost_rows(int dtype) { return dtype == 0 ? kGhostRows<double> : kGhostRows<float>; }

cudaError_t ghost_fill2_launch(int dtype, const DPatch* patches, const DCopy* copies, const DExcl* excl,
                               const GhostTask* tasks, int ntasks, const KernelTimer* tm, cudaStream_t s) {
  if (ntasks == 0) return cudaSuccess;
  const int nb = (ntasks + kThreads / 32 - 1) / (kThreads / 32);
  if (dtype == 0)
    MHD_TIMED(tm, K_GHOST, s, (k_ghost2<double><<<nb, kThreads, 0, s>>>(patches, copies, excl, tasks, ntasks)));
  else
    MHD_TIMED(tm, K_GHOST, s, (k_ghost2<float><<<nb, kThreads, 0, s>>>(patches, copies, excl, tasks, ntasks)));
  return cudaGetLastError();
}

cudaError_t prolong_launch(int dtype, const DPatch* coarse, const DPatch* fine, const DBoxItem* items,
                           const PackedTasks& p, const KernelTimer* tm, cudaStream_t s) {
  if (p.nblocks == 0) return cudaSuccess;
  if (dtype == 0)
    MHD_TIMED(tm, K_PROLONG, s, (k_prolong<double><<<p.nblocks, kThreads, 0, s>>>(coarse, fine, items, p.tasks,
                                                                                  p.starts, p.nitems, p.packed)));
  else
    MHD_TIMED(tm, K_PROLONG, s, (k_prolong<float><<<p.nblocks, kThreads, 0, s>>>(coarse, fine, items, p.tasks,
                                                                                 p.starts, p.nitems, p.packed)));
  return cudaGetLastError();
}

cudaError_t restrict_launch(int dtype, const DPatch* fine, const DPatch* coarse, const DBoxItem* items,
                            const PackedTasks& p0, const PackedTasks& p1, const KernelTimer* tm, cudaStream_t s) {
  for (int pass = 0; pass < 2; ++pass) {
    const PackedTasks& p = pass ? p1 : p0;
    if (p.nblocks == 0) continue;
    if (dtype == 0)
      MHD_TIMED(tm, K_RESTRICT, s, (k_restrict<double><<<p.nblocks, kThreads, 0, s>>>(fine, coarse, items, p.tasks,
                                                                                      p.starts, p.nitems, p.packed, pass)));
    else
      MHD_TIMED(tm, K_RESTRICT, s, (k_restrict<float><<<p.nblocks, kThreads, 0, s>>>(fine, coarse, items, p.tasks,
                                                                                     p.starts, p.nitems, p.packed, pass)));
  }
  return cudaGetLastError();
}

cudaError_t capture_launch(int dtype, const DPatch* patches, const DCapture* caps, const PackedTasks& p,
                           const void* scratch, const double* d_dt, const KernelTimer* tm, cudaStream_t s) {
  if (p.nblocks == 0) return cudaSuccess;
  if (dtype == 0)
    MHD_TIMED(tm, K_CAPTURE, s, (k_capture<double><<<p.nblocks, kThreads, 0, s>>>(patches, caps, p.tasks, p.starts,
                                                                                  p.nitems, p.packed,
                                                                                  (const double*)scratch,
                                                                                  d_dt)));
  else
    MHD_TIMED(tm, K_CAPTURE, s, (k_capture<float><<<p.nblocks, kThreads, 0, s>>>(patches, caps, p.tasks, p.starts,
                                                                                 p.nitems, p.packed,
                                                                                 (const float*)scratch,
                                                                                 d_dt)));
  return cudaGetLastError();
}

cudaError_t reflux_launch(int dtype, const DPatch* coarse, const DCorr* corr, const RefluxList& list,
                          const DDeposit* deps, const BlockTask* dep_tasks, int ndep, const KernelTimer* tm,
                          cudaStream_t s) {
  if (ndep == 0) return cudaSuccess;  // no deposit: every correction is zero
  const int ncorr = (int)((list.capacity + kThreads - 1) / kThreads);
  MHD_TIMED(tm, K_REFLUX, s, (cudaMemsetAsync(list.count, 0, sizeof(unsigned long long), s),
                              k_deposit<<<ndep, kThreads, 0, s>>>(coarse, deps, dep_tasks, list)));
  if (ncorr) {
    if (dtype == 0)
      MHD_TIMED(tm, K_REFLUX, s, (k_correct<double><<<ncorr, kThreads, 0, s>>>(coarse, corr, list)));
    else
      MHD_TIMED(tm, K_REFLUX, s, (k_correct<float><<<ncorr, kThreads, 0, s>>>(coarse, corr, list)));
  }
  MHD_TIMED(tm, K_REFLUX, s, (k_unset<<<ndep, kThreads, 0, s>>>(coarse, deps, dep_tasks)));
  return cudaGetLastError();
}

}  // namespace mhd
