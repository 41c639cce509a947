// regrid.cu -- device work of regridding (Sec. 2.1): the error flags of the
// patches of a level, and the data transfer into a new iteration of a level
// (the O step of Sec. 2.2): copies of the previous iteration's cells and faces
// where old and new patches meet, and the prolongation of the rest of a new
// interior from the parent level, divergence-free at the seams.  Built with
// --fmad=false: the flag is a comparison of FP64 expressions that must take
// the oracle's decision bit for bit, and the FP64 transfer gives the oracle's
// bits.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "launch.h"
#include "physics.cuh"
#include "regrid.h"

namespace mhd {
namespace {

// Primitive rho and p of the cell at element x, in FP64 (an FP32 state is
// converted first), with the oracle's expression order.
template <typename R>
__device__ __forceinline__ void rho_p(const DPatch& p, int64_t x, double gm1, double& rho, double& pr) {
  double u[8];
#pragma unroll
  for (int q = 0; q < 5; ++q) u[q] = (double)((const R*)p.U[q])[x];
  u[5] = 0.5 * ((double)((const R*)p.B[0])[x] + (double)((const R*)p.B[0])[x + 1]);
  u[6] = 0.5 * ((double)((const R*)p.B[1])[x] + (double)((const R*)p.B[1])[x + p.s1]);
  u[7] = 0.5 * ((double)((const R*)p.B[2])[x] + (double)((const R*)p.B[2])[x + p.s2]);
  const double ir = 1.0 / u[0];
  const double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  const double ke = 0.5 * u[0] * (vx * vx + vy * vy + vz * vz);
  const double me = 0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  rho = u[0];
  pr = gm1 * (u[4] - ke - me);
}

// One thread per interior cell: flagged when, for q in {rho, p} and some
// axis d, |q(+d) - q(-d)| > theta (|q(+d)| + 2 |q| + |q(-d)|).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_flag(const DPatch* __restrict__ P, const BlockTask* __restrict__ T,
                                                   const int64_t* __restrict__ off, double gm1, double theta,
                                                   uint8_t* flags) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  const int e = t.start + threadIdx.x;
  const int nc = p.n[0] * p.n[1] * p.n[2];
  if (e >= nc) return;
  const int i = e % p.n[0], j = (e / p.n[0]) % p.n[1], k = e / (p.n[0] * p.n[1]);
  const int64_t x = (int64_t)(p.g + i) + (int64_t)(p.g + j) * p.s1 + (int64_t)(p.g + k) * p.s2;
  double r0, p0;
  rho_p<R>(p, x, gm1, r0, p0);
  int f = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t sd = d == 0 ? 1 : (d == 1 ? p.s1 : p.s2);
    double rm, pm, rp, pp;
    rho_p<R>(p, x - sd, gm1, rm, pm);
    rho_p<R>(p, x + sd, gm1, rp, pp);
    {
      const double num = fabs(rp - rm), den = fabs(rp) + 2.0 * fabs(r0) + fabs(rm);
      if (num > theta * den) f = 1;
    }
    {
      const double num = fabs(pp - pm), den = fabs(pp) + 2.0 * fabs(p0) + fabs(pm);
      if (num > theta * den) f = 1;
    }
  }
  flags[off[t.patch] + e] = (uint8_t)f;
}

__device__ __forceinline__ int64_t lin3r(const DPatch& p, int i, int j, int k) {
  return (int64_t)i + (int64_t)j * p.s1 + (int64_t)k * p.s2;
}
__device__ __forceinline__ int64_t sofr(const DPatch& p, int d) {
  return d == 0 ? (int64_t)1 : (d == 1 ? p.s1 : p.s2);
}
template <typename R> __device__ __forceinline__ R mm(R a, R b) { return limiter<R>(1, a, b); }
template <typename R> __device__ __forceinline__ R thermal_r(const DPatch& p, int64_t x) {
  const R rho = ((const R*)p.U[0])[x];
  const R mx = ((const R*)p.U[1])[x], my = ((const R*)p.U[2])[x], mz = ((const R*)p.U[3])[x];
  R ke = R(0.5) * (mx * mx + my * my + mz * mz) / rho;
  R bx = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
  R by = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
  R bz = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
  R me = R(0.5) * (bx * bx + by * by + bz * bz);
  return ((const R*)p.U[4])[x] - ke - me;
}

// One thread per element of a transfer item: the five cell values (kind -1)
// or one face value (kind a) from the old patch to the new one.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_transfer_copy(const DPatch* __restrict__ PO, const DPatch* __restrict__ PN,
                                                            const DTransfer* __restrict__ I,
                                                            const BlockTask* __restrict__ T) {
  const BlockTask t = T[blockIdx.x];
  const DTransfer it = I[t.patch];
  const int e = t.start + threadIdx.x;
  if (e >= it.ext[0] * it.ext[1] * it.ext[2]) return;
  const int g3[3] = {it.lo[0] + e % it.ext[0], it.lo[1] + (e / it.ext[0]) % it.ext[1],
                     it.lo[2] + e / (it.ext[0] * it.ext[1])};
  const DPatch& o = PO[it.src];
  const DPatch& n = PN[it.dst];
  const int64_t xs = lin3r(o, g3[0] - o.glo[0], g3[1] - o.glo[1], g3[2] - o.glo[2]);
  const int64_t xd = lin3r(n, g3[0] - n.glo[0], g3[1] - n.glo[1], g3[2] - n.glo[2]);
  if (it.kind < 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) ((R*)n.U[q])[xd] = ((const R*)o.U[q])[xs];
  } else {
    ((R*)n.B[it.kind])[xd] = ((const R*)o.B[it.kind])[xs];
  }
}

// phi = L^+ r on the eight children (Walsh functions of the cube; the S = 0
// part dropped), in the oracle's order.
template <typename R> __device__ __forceinline__ void cube_potential(const R (&r)[8], R (&phi)[8]) {
  R coef[8];
  coef[0] = R(0);
#pragma unroll
  for (int S = 1; S < 8; ++S) {
    R t = R(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int par = __popc(S & c) & 1;
      t = par ? t - r[c] : t + r[c];
    }
    const int w = __popc(S);
    coef[S] = (t * R(0.125)) / (R(2) * R(w));
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    R v = R(0);
#pragma unroll
    for (int S = 1; S < 8; ++S) {
      const int par = __popc(S & c) & 1;
      v = par ? v - coef[S] : v + coef[S];
    }
    phi[c] = v;
  }
}

// One thread per coarse cell of an item box: the prolongation into a new
// interior under the item's mask (bit 0: the children hold copied data, skip;
// bit 1 + 2 a + s: keep and read the four sub-faces on side s of axis a),
// with the seam correction of the inner faces and, with energy_mode 1, the
// conservative scaling of the children's thermal energy.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_prolong_new(const DPatch* __restrict__ PC, const DPatch* __restrict__ PF,
                                                          const DProlongNew* __restrict__ I,
                                                          const BlockTask* __restrict__ T, int energy_mode,
                                                          unsigned long long* nfall) {
  const BlockTask t = T[blockIdx.x];
  const DProlongNew it = I[t.patch];
  const int e = t.start + threadIdx.x;
  if (e >= it.ext[0] * it.ext[1] * it.ext[2]) return;
  const int C3[3] = {it.lo[0] + e % it.ext[0], it.lo[1] + (e / it.ext[0]) % it.ext[1],
                     it.lo[2] + e / (it.ext[0] * it.ext[1])};
  const int mk = it.mask[(C3[0] - it.mlo[0]) + it.mext[0] * ((C3[1] - it.mlo[1]) + it.mext[1] * (C3[2] - it.mlo[2]))];
  if (mk & 1) return;
  const DPatch& pc = PC[it.coarse];
  const DPatch& pf = PF[it.fine];
  const int64_t c = lin3r(pc, C3[0] - pc.glo[0], C3[1] - pc.glo[1], C3[2] - pc.glo[2]);
  R uc[4], h[4][3], he[3];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R* Uq = (const R*)pc.U[q];
    uc[q] = Uq[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R a = uc[q] - Uq[c - sofr(pc, d)];
      R b = Uq[c + sofr(pc, d)] - uc[q];
      h[q][d] = R(0.25) * mm(a, b);
    }
  }
  const R ec = thermal_r<R>(pc, c);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R a = ec - thermal_r<R>(pc, c - sofr(pc, d));
    R b = thermal_r<R>(pc, c + sofr(pc, d)) - ec;
    he[d] = R(0.25) * mm(a, b);
  }
  R m[3][2], qs[3][2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R* Ba = (const R*)pc.B[a];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int64_t f = c + (sd ? sofr(pc, a) : 0);
      m[a][sd] = Ba[f];
#pragma unroll
      for (int tt = 0; tt < 3; ++tt) {
        if (tt == a) {
          qs[a][sd][tt] = R(0);
          continue;
        }
        R lo = m[a][sd] - Ba[f - sofr(pc, tt)];
        R hi = Ba[f + sofr(pc, tt)] - m[a][sd];
        qs[a][sd][tt] = R(0.25) * mm(lo, hi);
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
  // fine faces fv[a][pos][s2][s1] (pos 0 lower coarse face, 1 inner, 2 upper)
  R fv[3][3][2][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
#pragma unroll
    for (int pos = 0; pos < 3; ++pos)
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          const bool keep = pos != 1 && ((mk >> (1 + 2 * a + (pos == 2))) & 1);
          R v;
          if (keep) {
            int g3[3];
            g3[a] = 2 * C3[a] + pos;
            g3[lo_t] = 2 * C3[lo_t] + s1;
            g3[hi_t] = 2 * C3[hi_t] + s2;
            v = ((const R*)pf.B[a])[lin3r(pf, g3[0] - pf.glo[0], g3[1] - pf.glo[1], g3[2] - pf.glo[2])];
          } else if (pos == 1) {
            R sl = s1 ? R(0.5) * lin[a][lo_t] : R(-0.5) * lin[a][lo_t];
            R sh = s2 ? R(0.5) * lin[a][hi_t] : R(-0.5) * lin[a][hi_t];
            v = c0[a] + sl + sh;
          } else {
            const int sd = pos == 2;
            R sl = s1 ? qs[a][sd][lo_t] : -qs[a][sd][lo_t];
            R sh = s2 ? qs[a][sd][hi_t] : -qs[a][sd][hi_t];
            v = m[a][sd] + sl + sh;
          }
          fv[a][pos][s2][s1] = v;
        }
  }
  if (mk >> 1) {
    R r[8], phi[8];
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      const int sub[3] = {c8 & 1, (c8 >> 1) & 1, (c8 >> 2) & 1};
      R dv = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
        const R up = fv[a][sub[a] + 1][sub[hi_t]][sub[lo_t]];
        const R dn = fv[a][sub[a]][sub[hi_t]][sub[lo_t]];
        dv = dv + (up - dn);
      }
      r[c8] = dv;
    }
    cube_potential(r, phi);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
      const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          const int lo8 = (s1 << lo_t) | (s2 << hi_t), hi8 = lo8 | (1 << a);
          fv[a][1][s2][s1] = fv[a][1][s2][s1] + (phi[hi8] - phi[lo8]);
        }
    }
  }
  // faces not kept
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
#pragma unroll
    for (int pos = 0; pos < 3; ++pos) {
      const bool keep = pos != 1 && ((mk >> (1 + 2 * a + (pos == 2))) & 1);
      if (keep) continue;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int s1 = 0; s1 < 2; ++s1) {
          int g3[3];
          g3[a] = 2 * C3[a] + pos;
          g3[lo_t] = 2 * C3[lo_t] + s1;
          g3[hi_t] = 2 * C3[hi_t] + s2;
          ((R*)pf.B[a])[lin3r(pf, g3[0] - pf.glo[0], g3[1] - pf.glo[1], g3[2] - pf.glo[2])] = fv[a][pos][s2][s1];
        }
    }
  }
  // the eight children
  R uf[8][4], ef[8], kef[8], mef[8];
#pragma unroll
  for (int c8 = 0; c8 < 8; ++c8) {
    const int fa = c8 & 1, fb = (c8 >> 1) & 1, fc = (c8 >> 2) & 1;
    const int sub[3] = {fa, fb, fc};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      R u = uc[q];
      u = u + (fa ? h[q][0] : -h[q][0]);
      u = u + (fb ? h[q][1] : -h[q][1]);
      u = u + (fc ? h[q][2] : -h[q][2]);
      uf[c8][q] = u;
    }
    R bc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
      const int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
      bc[a] = R(0.5) * (fv[a][sub[a]][sub[hi_t]][sub[lo_t]] + fv[a][sub[a] + 1][sub[hi_t]][sub[lo_t]]);
    }
    R en = ec;
    en = en + (fa ? he[0] : -he[0]);
    en = en + (fb ? he[1] : -he[1]);
    en = en + (fc ? he[2] : -he[2]);
    ef[c8] = en;
    kef[c8] = R(0.5) * (uf[c8][1] * uf[c8][1] + uf[c8][2] * uf[c8][2] + uf[c8][3] * uf[c8][3]) / uf[c8][0];
    mef[c8] = R(0.5) * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
  }
  R scale = R(0);
  bool cons = false;
  if (energy_mode == 1) {
    R sE = R(0), se = R(0);
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) {
      sE = sE + ((ef[c8] + kef[c8]) + mef[c8]);
      se = se + ef[c8];
    }
    const R delta = ((const R*)pc.U[4])[c] - R(0.125) * sE, ebar = R(0.125) * se;
    if (ebar + delta > R(0)) {
      cons = true;
      scale = delta / ebar;
    } else {
      atomicAdd(nfall, 1ull);
    }
  }
#pragma unroll
  for (int c8 = 0; c8 < 8; ++c8) {
    const int fa = c8 & 1, fb = (c8 >> 1) & 1, fc = (c8 >> 2) & 1;
    const int64_t x = lin3r(pf, 2 * C3[0] + fa - pf.glo[0], 2 * C3[1] + fb - pf.glo[1], 2 * C3[2] + fc - pf.glo[2]);
#pragma unroll
    for (int q = 0; q < 4; ++q) ((R*)pf.U[q])[x] = uf[c8][q];
    const R en = cons ? ef[c8] + ef[c8] * scale : ef[c8];
    ((R*)pf.U[4])[x] = (en + kef[c8]) + mef[c8];
  }
}

}  // namespace

cudaError_t flag_launch(int dtype, const DPatch* patches, const BlockTask* tasks, int nblocks, const int64_t* off,
                        double gamma, double theta, uint8_t* flags, cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  if (dtype == 0)
    k_flag<double><<<nblocks, kThreads, 0, s>>>(patches, tasks, off, gamma - 1.0, theta, flags);
  else
    k_flag<float><<<nblocks, kThreads, 0, s>>>(patches, tasks, off, gamma - 1.0, theta, flags);
  return cudaGetLastError();
}

}  // namespace mhd

namespace mhd {

cudaError_t transfer_copy_launch(int dtype, const DPatch* old, const DPatch* fresh, const DTransfer* items,
                                 const BlockTask* tasks, int nblocks, cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  if (dtype == 0)
    k_transfer_copy<double><<<nblocks, kThreads, 0, s>>>(old, fresh, items, tasks);
  else
    k_transfer_copy<float><<<nblocks, kThreads, 0, s>>>(old, fresh, items, tasks);
  return cudaGetLastError();
}

cudaError_t prolong_new_launch(int dtype, const DPatch* coarse, const DPatch* fine, const DProlongNew* items,
                               const BlockTask* tasks, int nblocks, int energy_mode, unsigned long long* nfall,
                               cudaStream_t s) {
  if (nblocks == 0) return cudaSuccess;
  if (dtype == 0)
    k_prolong_new<double><<<nblocks, kThreads, 0, s>>>(coarse, fine, items, tasks, energy_mode, nfall);
  else
    k_prolong_new<float><<<nblocks, kThreads, 0, s>>>(coarse, fine, items, tasks, energy_mode, nfall);
  return cudaGetLastError();
}

}  // namespace mhd
