// physics.cuh -- point functions of the ideal-MHD patch advance on the GPU,
// templated on the arithmetic type R (double or float).
//
// The scheme (the paper names only "the hyperbolic advance of each grid",
// Sec. 2.3, consuming n_ghost ghost layers per step):
//   primitive PLM reconstruction with a van Leer / minmod / MC limiter,
//   a conservative Hancock half-step predictor, a CT half-step predictor for
//   the face-normal field, the HLLD Riemann solver of Miyoshi & Kusano (2005,
//   JCP 208:315) and Gardiner & Stone (2005, JCP 205:509) edge EMFs.
// Every expression is written in one fixed evaluation order; the FP64
// translation unit is compiled with --fmad=false so that no multiply-add is
// contracted and results are reproducible bit for bit.
#pragma once

#include <cstdint>

namespace mhd {

// degen: relative threshold of the HLLD single-star degeneracy test.  It must
// sit well above the rounding of rho (S - u)(S - S_M) - Bn^2 in the arithmetic
// type: 1e-12 in FP64 (about 4500 ulp), 1e-5 in FP32 (about 80 ulp); an FP32
// test at 1e-12 never fires, and a denominator that is rounding noise then
// divides the transverse velocity and field.
template <typename R> struct Tr;
template <> struct Tr<double> {
  __device__ static __forceinline__ double abs(double x) { return fabs(x); }
  __device__ static __forceinline__ double sqrt_(double x) { return sqrt(x); }
  __device__ static __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  __device__ static __forceinline__ double degen() { return 1e-12; }
};
template <> struct Tr<float> {
  __device__ static __forceinline__ float abs(float x) { return fabsf(x); }
  __device__ static __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  __device__ static __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  __device__ static __forceinline__ float degen() { return 1e-5f; }
};

template <typename R> __device__ __forceinline__ R rmin(R a, R b) { return (a < b) ? a : b; }
template <typename R> __device__ __forceinline__ R rmax(R a, R b) { return (a > b) ? a : b; }

// Limited slope of the backward difference a and forward difference b;
// a*b <= 0 gives zero.
template <typename R> __device__ __forceinline__ R limiter(int lim, R a, R b) {
  R ab = a * b;
  if (!(ab > R(0))) return R(0);
  if (lim == 1) return (Tr<R>::abs(a) < Tr<R>::abs(b)) ? a : b;
  if (lim == 2) {
    R s = (a > R(0)) ? R(1) : R(-1);
    R m = rmin(rmin(R(2) * Tr<R>::abs(a), R(2) * Tr<R>::abs(b)), R(0.5) * Tr<R>::abs(a + b));
    return s * m;
  }
  return (ab + ab) / (a + b);
}

// conserved (rho, M, E, Bc) -> primitive (rho, v, p, Bc)
template <typename R> __device__ __forceinline__ void cons2prim(const R* u, R gm1, R* w) {
  R rho = u[0];
  R ir = R(1) / rho;
  R vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  R ke = R(0.5) * rho * (vx * vx + vy * vy + vz * vz);
  R me = R(0.5) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  w[0] = rho; w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = gm1 * (u[4] - ke - me);
  w[5] = u[5]; w[6] = u[6]; w[7] = u[7];
}

template <typename R> __device__ __forceinline__ void prim2cons(const R* w, R igm1, R* u) {
  R rho = w[0];
  R ke = R(0.5) * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
  R me = R(0.5) * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
  u[0] = rho;
  u[1] = rho * w[1]; u[2] = rho * w[2]; u[3] = rho * w[3];
  u[4] = w[4] * igm1 + ke + me;
  u[5] = w[5]; u[6] = w[6]; u[7] = w[7];
}

// Fast magnetosonic speed: c_f^2 = ((a^2+b^2) + sqrt((a^2+b^2)^2 - 4 a^2 b_n^2))/2.
template <typename R>
__device__ __forceinline__ R fast_speed(R rho, R p, R bn, R bt1, R bt2, R gamma) {
  R ir = R(1) / rho;
  R a2 = gamma * p * ir;
  R b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) * ir;
  R bn2 = bn * bn * ir;
  R s = a2 + b2;
  R d = s * s - R(4) * a2 * bn2;
  if (d < R(0)) d = R(0);
  return Tr<R>::sqrt_(R(0.5) * (s + Tr<R>::sqrt_(d)));
}

// Ideal-MHD flux along the normal of a rotated primitive state
// (rho, vn, vt1, vt2, p, -, bt1, bt2) with normal field bn; rotated output,
// f[5] (normal-B flux) is zero.
template <typename R> __device__ __forceinline__ void flux_rot(const R* r, R bn, R igm1, R* f) {
  R rho = r[0], vn = r[1], vt1 = r[2], vt2 = r[3], p = r[4];
  R bt1 = r[6], bt2 = r[7];
  R pm = R(0.5) * (bn * bn + bt1 * bt1 + bt2 * bt2);
  R pt = p + pm;
  R ke = R(0.5) * rho * (vn * vn + vt1 * vt1 + vt2 * vt2);
  R e = p * igm1 + ke + pm;
  R vb = vn * bn + vt1 * bt1 + vt2 * bt2;
  R mn_ = rho * vn;
  f[0] = mn_;
  f[1] = mn_ * vn + pt - bn * bn;
  f[2] = mn_ * vt1 - bn * bt1;
  f[3] = mn_ * vt2 - bn * bt2;
  f[4] = (e + pt) * vn - bn * vb;
  f[5] = R(0);
  f[6] = bt1 * vn - bn * vt1;
  f[7] = bt2 * vn - bn * vt2;
}

// rotation helpers: axis d -> (n, t1, t2) = (d, d+1, d+2) mod 3
template <typename R> __device__ __forceinline__ void rot_in(int d, const R* w, R* r) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  r[0] = w[0]; r[1] = w[1 + d]; r[2] = w[1 + t1]; r[3] = w[1 + t2];
  r[4] = w[4]; r[5] = w[5 + d]; r[6] = w[5 + t1]; r[7] = w[5 + t2];
}
template <typename R> __device__ __forceinline__ void rot_out(int d, const R* fr, R* f) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  f[0] = fr[0]; f[1 + d] = fr[1]; f[1 + t1] = fr[2]; f[1 + t2] = fr[3];
  f[4] = fr[4]; f[5 + d] = fr[5]; f[5 + t1] = fr[6]; f[5 + t2] = fr[7];
}

// Physical flux along axis d of an xyz primitive state (own B_d as normal).
template <typename R> __device__ __forceinline__ void flux_xyz(int d, const R* w, R igm1, R* f) {
  R r[8], fr[8];
  rot_in(d, w, r);
  flux_rot(r, r[5], igm1, fr);
  rot_out(d, fr, f);
}

// a / b, or a * ib with ib = 1 / b computed once for several quotients (the
// reciprocal form of the FP32 and the contracted FP64 builds; the parity
// build divides, as the oracle does)
template <bool FR, typename R> __device__ __forceinline__ R qdiv(R a, R b, R ib) {
  if constexpr (FR) return a * ib;
  else return a / b;
}
template <bool FR, typename R> __device__ __forceinline__ R recip(R b) {
  if constexpr (FR) return R(1) / b;
  else return R(0);
}

// HLLD flux (Miyoshi & Kusano 2005) between rotated primitive states L (lower
// side) and R_ (upper side) with interface normal field bn.  Wave speeds
// S_L = min(u_L,u_R) - max(cf), S_R = max(u_L,u_R) + max(cf); S_M, p_T* from
// MK05 eqs. (38), (41); star states eqs. (43)-(48) with a degenerate branch
// (|rho(S-u)(S-S_M) - Bn^2| <= degen max(rho(S-u)^2, Bn^2), degen 1e-12 in
// FP64 and 1e-5 in FP32, keeps the outer
// transverse v, B); Alfven speeds S* = S_M -/+ |Bn|/sqrt(rho*); double-star
// states eqs. (59)-(63); left-closed region selection.  f gets the rotated
// flux; *upw the upwind side of the contact (+1, -1, or 0 when
// |S_M| <= eps_up (S_R - S_L)).  FR: quotients with a common denominator
// multiply by its reciprocal, and |Bn|/sqrt(rho*) uses a reciprocal square
// root (8 divisions per face instead of 18), and the single-star field factor
// is written as 1 + rho (S - u)(S_M - u)/den, which is exactly 1 where
// S_M = u (a plain reciprocal would turn x/x into x (1/x), off by an ulp,
// and give a 2D problem a z-field of rounding noise).
template <typename R, bool FR = false>
__device__ __forceinline__ void hlld(const R* L, const R* Rr, R bn, R gamma, R igm1, R eps_up,
                                     R* f, R* upw) {
  R rl = L[0], ul = L[1], vl = L[2], wl_ = L[3], pl = L[4], byl = L[6], bzl = L[7];
  R rr = Rr[0], ur = Rr[1], vr = Rr[2], wr_ = Rr[3], pr = Rr[4], byr = Rr[6], bzr = Rr[7];

  R pml = R(0.5) * (bn * bn + byl * byl + bzl * bzl);
  R pmr = R(0.5) * (bn * bn + byr * byr + bzr * bzr);
  R ptl = pl + pml, ptr = pr + pmr;
  R el = pl * igm1 + R(0.5) * rl * (ul * ul + vl * vl + wl_ * wl_) + pml;
  R er = pr * igm1 + R(0.5) * rr * (ur * ur + vr * vr + wr_ * wr_) + pmr;

  R cfl = fast_speed(rl, pl, bn, byl, bzl, gamma);
  R cfr = fast_speed(rr, pr, bn, byr, bzr, gamma);
  R cmax = rmax(cfl, cfr);
  R sl = rmin(ul, ur) - cmax;
  R sr = rmax(ul, ur) + cmax;

  if (sl >= R(0)) {
    flux_rot(L, bn, igm1, f);
    *upw = R(1);
    return;
  }
  if (sr < R(0)) {
    flux_rot(Rr, bn, igm1, f);
    *upw = R(-1);
    return;
  }

  R sdl = sl - ul, sdr = sr - ur;
  R rsl = sdl * rl, rsr = sdr * rr;
  R dd = rsr - rsl;
  const R idd = recip<FR>(dd);
  R sm = qdiv<FR>((rsr * ur - rsl * ul) - (ptr - ptl), dd, idd);
  R pts = qdiv<FR>((rsr * ptl - rsl * ptr) + rsl * rsr * (ur - ul), dd, idd);
  R tie = eps_up * (sr - sl);
  *upw = (sm > tie) ? R(1) : ((sm < -tie) ? R(-1) : R(0));

  R sml = sl - sm, smr = sr - sm;
  const R isml = recip<FR>(sml), ismr = recip<FR>(smr);
  R rls = qdiv<FR>(rsl, sml, isml), rrs = qdiv<FR>(rsr, smr, ismr);
  R bn2 = bn * bn;
  R vls, wls, byls, bzls;
  R denl = rsl * sml - bn2;
  if (Tr<R>::abs(denl) <= Tr<R>::degen() * rmax(rsl * sdl, bn2)) {
    vls = vl; wls = wl_; byls = byl; bzls = bzl;
  } else {
    R fv, fb;
    if constexpr (FR) {
      // numerator of fb = den + rho (S - u)(S_M - u): fb = 1 + rho (S - u) t
      // with t = (S_M - u) / den, exactly 1 where S_M = u
      const R t = (sm - ul) * (R(1) / denl);
      fv = bn * t;
      fb = R(1) + rsl * t;
    } else {
      fv = bn * (sm - ul) / denl;
      fb = (rsl * sdl - bn2) / denl;
    }
    vls = vl - byl * fv; wls = wl_ - bzl * fv;
    byls = byl * fb; bzls = bzl * fb;
  }
  R vrs, wrs, byrs, bzrs;
  R denr = rsr * smr - bn2;
  if (Tr<R>::abs(denr) <= Tr<R>::degen() * rmax(rsr * sdr, bn2)) {
    vrs = vr; wrs = wr_; byrs = byr; bzrs = bzr;
  } else {
    R fv, fb;
    if constexpr (FR) {
      // numerator of fb = den + rho (S - u)(S_M - u): fb = 1 + rho (S - u) t
      // with t = (S_M - u) / den, exactly 1 where S_M = u
      const R t = (sm - ur) * (R(1) / denr);
      fv = bn * t;
      fb = R(1) + rsr * t;
    } else {
      fv = bn * (sm - ur) / denr;
      fb = (rsr * sdr - bn2) / denr;
    }
    vrs = vr - byr * fv; wrs = wr_ - bzr * fv;
    byrs = byr * fb; bzrs = bzr * fb;
  }
  R vbl = ul * bn + vl * byl + wl_ * bzl;
  R vbr = ur * bn + vr * byr + wr_ * bzr;
  R vbls = sm * bn + vls * byls + wls * bzls;
  R vbrs = sm * bn + vrs * byrs + wrs * bzrs;
  R els = qdiv<FR>(((sdl * el - ptl * ul) + pts * sm) + bn * (vbl - vbls), sml, isml);
  R ers = qdiv<FR>(((sdr * er - ptr * ur) + pts * sm) + bn * (vbr - vbrs), smr, ismr);

  R sqrl, sqrr, sls, srs;
  if constexpr (FR) {
    const R isl = Tr<R>::rsqrt_(rls), isr = Tr<R>::rsqrt_(rrs);
    sqrl = rls * isl;
    sqrr = rrs * isr;
    sls = sm - Tr<R>::abs(bn) * isl;
    srs = sm + Tr<R>::abs(bn) * isr;
  } else {
    sqrl = Tr<R>::sqrt_(rls);
    sqrr = Tr<R>::sqrt_(rrs);
    sls = sm - Tr<R>::abs(bn) / sqrl;
    srs = sm + Tr<R>::abs(bn) / sqrr;
  }

  R fo[8];
  if (sls >= R(0) || srs < R(0)) {
    // single-star region: F* = F_outer + S_outer (U* - U_outer)
    const bool left = (sls >= R(0));
    const R rho = left ? rl : rr, u = left ? ul : ur, v = left ? vl : vr, w = left ? wl_ : wr_;
    const R e = left ? el : er, by = left ? byl : byr, bz = left ? bzl : bzr;
    const R S = left ? sl : sr;
    const R rs = left ? rls : rrs, vs = left ? vls : vrs, ws = left ? wls : wrs;
    const R es = left ? els : ers, bys = left ? byls : byrs, bzs = left ? bzls : bzrs;
    flux_rot(left ? L : Rr, bn, igm1, fo);
    const R u0[8] = {rho, rho * u, rho * v, rho * w, e, bn, by, bz};
    const R us[8] = {rs, rs * sm, rs * vs, rs * ws, es, bn, bys, bzs};
#pragma unroll
    for (int q = 0; q < 8; ++q) f[q] = fo[q] + S * (us[q] - u0[q]);
    return;
  }

  R sgn = (bn >= R(0)) ? R(1) : R(-1);
  R ssum = sqrl + sqrr;
  const R iss = recip<FR>(ssum);
  R vss = qdiv<FR>((sqrl * vls + sqrr * vrs) + sgn * (byrs - byls), ssum, iss);
  R wss = qdiv<FR>((sqrl * wls + sqrr * wrs) + sgn * (bzrs - bzls), ssum, iss);
  R byss = qdiv<FR>((sqrl * byrs + sqrr * byls) + sgn * (sqrl * sqrr) * (vrs - vls), ssum, iss);
  R bzss = qdiv<FR>((sqrl * bzrs + sqrr * bzls) + sgn * (sqrl * sqrr) * (wrs - wls), ssum, iss);
  R vbss = sm * bn + vss * byss + wss * bzss;

  const bool left = (sm >= R(0));
  const R rho = left ? rl : rr, u = left ? ul : ur, v = left ? vl : vr, w = left ? wl_ : wr_;
  const R e = left ? el : er, by = left ? byl : byr, bz = left ? bzl : bzr;
  const R S = left ? sl : sr, Ss = left ? sls : srs;
  const R rs = left ? rls : rrs, vs = left ? vls : vrs, ws = left ? wls : wrs;
  const R es = left ? els : ers, bys = left ? byls : byrs, bzs = left ? bzls : bzrs;
  R ess;
  if (left) ess = els - sqrl * (vbls - vbss) * sgn;
  else ess = ers + sqrr * (vbrs - vbss) * sgn;
  flux_rot(left ? L : Rr, bn, igm1, fo);
  const R u0[8] = {rho, rho * u, rho * v, rho * w, e, bn, by, bz};
  const R us[8] = {rs, rs * sm, rs * vs, rs * ws, es, bn, bys, bzs};
  const R uss[8] = {rs, rs * sm, rs * vss, rs * wss, ess, bn, byss, bzss};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    R fs = fo[q] + S * (us[q] - u0[q]);
    f[q] = fs + Ss * (uss[q] - us[q]);
  }
}

}  // namespace mhd
