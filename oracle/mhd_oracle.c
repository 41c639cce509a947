/*
 * mhd_oracle.c -- plain, slow FP64 CPU oracle of the ghost-celled ideal-MHD
 * patch advance (MUSCL-Hancock + PLM + HLLD + constrained transport).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * library: only tests/, the smoke check and the bench's cpu_baseline /
 * reference leg load it.  It shares no code with the CUDA path.
 *
 * The paper (Carroll-Nellenback et al., "Efficient Parallelization for AMR MHD
 * Multiphysics Calculations") says only that each grid is advanced on its own
 * by a hyperbolic solver that consumes n_ghost ghost layers (Sec. 2.3) inside
 * the O/P/A/S/R life cycle of Sec. 2.2; it never states the solver.  The solver
 * below is the named published method:
 *   - primitive PLM reconstruction with a van Leer / minmod / MC limiter;
 *   - a Hancock half-step predictor in conservative form;
 *   - a CT half-step predictor for face-normal B (edge EMF = mean of the four
 *     cell-centred -v x B);
 *   - the HLLD Riemann solver of Miyoshi & Kusano (2005, JCP 208:315);
 *   - Gardiner & Stone (2005, JCP 205:509) upwinded edge EMFs (or the plain
 *     arithmetic mean of Balsara & Spicer 1999);
 *   - the conservative cell update and the CT face update.
 * Each step consumes exactly 2 ghost layers, so the extended-ghost rule of
 * Sec. 2.3 (width R * n_ghost) gives 4 ghost layers for R = 2.
 *
 * Every formula is written with explicit evaluation order (C's left-to-right
 * rule for equal precedence); the build uses -ffp-contract=off so no FMA is
 * formed.  The arrays are structure-of-arrays, x fastest, one shared set of
 * element strides for the five cell arrays and the three face arrays (face
 * arrays carry one extra entry along their normal).
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py against
 * closed forms and invariants (uniform-state HLLD flux, mirror symmetry,
 * stationary contact, conservation, div B, linear Alfven convergence,
 * symmetry of the Orszag-Tang vortex and of the blast, the Sec. 4 cell-update
 * count).  Absolute accuracy of the nonlinear problems has no printed value
 * in the paper and is unpinned beyond those invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* Marks the start of stage k of the advance (and of the other operations)
 * for the operation-counting build (opcount.cpp); a no-op here. */
#ifndef ORC_STAGE
#define ORC_STAGE(k) ((void)0)
#endif

typedef struct {
  int32_t n[3];    /* interior cells per axis                          */
  int32_t g;       /* ghost layers on every side                       */
  int64_t s[3];    /* element strides of every array, s[0] == 1        */
  double dx[3];    /* cell widths                                      */
  double *U[5];    /* rho, Mx, My, Mz, E at cell centres               */
  double *B[3];    /* Bx on x-faces, By on y-faces, Bz on z-faces       */
} orc_patch;

typedef struct {
  double gamma;
  double cfl;
  int32_t limiter;  /* 0 van Leer (harmonic), 1 minmod, 2 monotonised central */
  int32_t emf;      /* 0 Gardiner-Stone upwinded, 1 arithmetic mean          */
  double upwind_eps;/* |S_M| <= upwind_eps (S_R - S_L) counts as no upwind side */
  double p_floor;   /* > 0: pressure floor after the update (R33); 0: none    */
  double rho_floor; /* > 0: density floor after the update (R33); 0: none     */
} orc_params;

/* Cells raised to the pressure floor by the last orc_advance. */
static int64_t orc_floored = 0;
ORC_EXPORT int64_t orc_floor_count(void) { return orc_floored; }

/* Threads of the OpenMP loops over independent cells (timing of the oracle
 * on one core and on all; results do not depend on it).  n <= 0: all. */
#ifdef _OPENMP
#include <omp.h>
ORC_EXPORT void orc_set_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }
ORC_EXPORT int32_t orc_get_threads(void) { return omp_get_max_threads(); }
#else
ORC_EXPORT void orc_set_threads(int32_t n) { (void)n; }
ORC_EXPORT int32_t orc_get_threads(void) { return 1; }
#endif

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */
static double mn(double a, double b) { return (a < b) ? a : b; }
static double mx(double a, double b) { return (a > b) ? a : b; }

/* Slope limiter of the two one-sided differences a (backward), b (forward).
 * Tie-break: a*b <= 0 gives a zero slope. */
ORC_EXPORT double orc_limiter(int32_t lim, double a, double b) {
  double ab = a * b;
  if (!(ab > 0.0)) return 0.0;
  if (lim == 1) return (fabs(a) < fabs(b)) ? a : b;
  if (lim == 2) {
    double s = (a > 0.0) ? 1.0 : -1.0;
    double m = mn(mn(2.0 * fabs(a), 2.0 * fabs(b)), 0.5 * fabs(a + b));
    return s * m;
  }
  return (ab + ab) / (a + b);
}

/* conserved (rho, M, E, B) -> primitive (rho, v, p, B); B is cell-centred. */
static void cons2prim(const double *u, double gm1, double *w) {
  double rho = u[0];
  double ir = 1.0 / rho;
  double vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  double ke = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
  double me = 0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  w[0] = rho; w[1] = vx; w[2] = vy; w[3] = vz;
  w[4] = gm1 * (u[4] - ke - me);
  w[5] = u[5]; w[6] = u[6]; w[7] = u[7];
}

static void prim2cons(const double *w, double igm1, double *u) {
  double rho = w[0];
  double ke = 0.5 * rho * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
  double me = 0.5 * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
  u[0] = rho;
  u[1] = rho * w[1]; u[2] = rho * w[2]; u[3] = rho * w[3];
  u[4] = w[4] * igm1 + ke + me;
  u[5] = w[5]; u[6] = w[6]; u[7] = w[7];
}

/* Fast magnetosonic speed along a direction with normal field bn and the two
 * transverse components bt1, bt2:
 *   c_f^2 = ( (a^2+b^2) + sqrt((a^2+b^2)^2 - 4 a^2 b_n^2) ) / 2,
 *   a^2 = gamma p / rho, b^2 = |B|^2 / rho, b_n^2 = bn^2 / rho. */
ORC_EXPORT double orc_fast_speed(double rho, double p, double bn, double bt1,
                                 double bt2, double gamma) {
  double ir = 1.0 / rho;
  double a2 = gamma * p * ir;
  double b2 = (bn * bn + bt1 * bt1 + bt2 * bt2) * ir;
  double bn2 = bn * bn * ir;
  double s = a2 + b2;
  double d = s * s - 4.0 * a2 * bn2;
  if (d < 0.0) d = 0.0;
  return sqrt(0.5 * (s + sqrt(d)));
}

/* Rotate an xyz primitive state into (rho, vn, vt1, vt2, p, Bn, Bt1, Bt2)
 * with n = d, t1 = (d+1)%3, t2 = (d+2)%3. */
static void rot_in(int d, const double *w, double *r) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  r[0] = w[0]; r[1] = w[1 + d]; r[2] = w[1 + t1]; r[3] = w[1 + t2];
  r[4] = w[4]; r[5] = w[5 + d]; r[6] = w[5 + t1]; r[7] = w[5 + t2];
}
static void rot_out(int d, const double *fr, double *f) {
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  f[0] = fr[0]; f[1 + d] = fr[1]; f[1 + t1] = fr[2]; f[1 + t2] = fr[3];
  f[4] = fr[4]; f[5 + d] = fr[5]; f[5 + t1] = fr[6]; f[5 + t2] = fr[7];
}

/* Ideal-MHD flux along the normal of a rotated primitive state r whose normal
 * field is bn.  Output in rotated order; the normal-B flux is zero. */
static void flux_rot(const double *r, double bn, double igm1, double *f) {
  double rho = r[0], vn = r[1], vt1 = r[2], vt2 = r[3], p = r[4];
  double bt1 = r[6], bt2 = r[7];
  double pm = 0.5 * (bn * bn + bt1 * bt1 + bt2 * bt2);
  double pt = p + pm;
  double ke = 0.5 * rho * (vn * vn + vt1 * vt1 + vt2 * vt2);
  double e = p * igm1 + ke + pm;
  double vb = vn * bn + vt1 * bt1 + vt2 * bt2;
  double mn_ = rho * vn;
  f[0] = mn_;
  f[1] = mn_ * vn + pt - bn * bn;
  f[2] = mn_ * vt1 - bn * bt1;
  f[3] = mn_ * vt2 - bn * bt2;
  f[4] = (e + pt) * vn - bn * vb;
  f[5] = 0.0;
  f[6] = bt1 * vn - bn * vt1;
  f[7] = bt2 * vn - bn * vt2;
}

/* Physical flux along axis d of an xyz primitive state (its own B_d used as
 * the normal field).  Output in xyz order. */
ORC_EXPORT void orc_flux(int32_t d, const double *w, double gamma, double *f) {
  double r[8], fr[8];
  double igm1 = 1.0 / (gamma - 1.0);
  rot_in(d, w, r);
  flux_rot(r, r[5], igm1, fr);
  rot_out(d, fr, f);
}

/* The HLLD wave fan (Miyoshi & Kusano 2005) between rotated primitive states
 * L (lower side) and R (upper side) with interface normal field bn (the
 * states' own normal components are ignored):
 *   S_L = min(u_L,u_R) - max(cf_L,cf_R),  S_R = max(u_L,u_R) + max(cf_L,cf_R);
 *   contact speed S_M and star total pressure from MK05 eqs. (38) and (41);
 *   single-star states eqs. (43)-(48); Alfven speeds
 *   S_L* = S_M - |Bn|/sqrt(rho_L*), S_R* = S_M + |Bn|/sqrt(rho_R*);
 *   double-star states eqs. (59)-(63).
 * Degenerate single-star states (|rho(S-u)(S-S_M) - Bn^2| <=
 * 1e-12 max(rho (S-u)^2, Bn^2)) keep the outer transverse v and B; sgn(0)=+1.
 * All conserved states are in rotated order (rho, Mn, Mt1, Mt2, E, Bn, Bt1, Bt2). */
typedef struct {
  double sl, sls, sm, srs, sr;
  double fl[8], fr[8];
  double u0l[8], usl[8], ussl[8], ussr[8], usr[8], u0r[8];
} hlld_fan;

static void hlld_fan_solve(const double *L, const double *R, double bn, double gamma,
                           double igm1, hlld_fan *o) {
  double rl = L[0], ul = L[1], vl = L[2], wl_ = L[3], pl = L[4], byl = L[6], bzl = L[7];
  double rr = R[0], ur = R[1], vr = R[2], wr_ = R[3], pr = R[4], byr = R[6], bzr = R[7];

  double pml = 0.5 * (bn * bn + byl * byl + bzl * bzl);
  double pmr = 0.5 * (bn * bn + byr * byr + bzr * bzr);
  double ptl = pl + pml, ptr = pr + pmr;
  double el = pl * igm1 + 0.5 * rl * (ul * ul + vl * vl + wl_ * wl_) + pml;
  double er = pr * igm1 + 0.5 * rr * (ur * ur + vr * vr + wr_ * wr_) + pmr;

  double cfl = orc_fast_speed(rl, pl, bn, byl, bzl, gamma);
  double cfr = orc_fast_speed(rr, pr, bn, byr, bzr, gamma);
  double cmax = mx(cfl, cfr);
  double sl = mn(ul, ur) - cmax;
  double sr = mx(ul, ur) + cmax;
  flux_rot(L, bn, igm1, o->fl);
  flux_rot(R, bn, igm1, o->fr);

  double sdl = sl - ul, sdr = sr - ur;
  double rsl = sdl * rl, rsr = sdr * rr;
  double dd = rsr - rsl;
  double sm = ((rsr * ur - rsl * ul) - (ptr - ptl)) / dd;
  double pts = ((rsr * ptl - rsl * ptr) + rsl * rsr * (ur - ul)) / dd;

  /* single-star states */
  double sml = sl - sm, smr = sr - sm;
  double rls = rsl / sml, rrs = rsr / smr;
  double bn2 = bn * bn;
  double vls, wls, byls, bzls;
  double denl = rsl * sml - bn2;
  if (fabs(denl) <= 1e-12 * mx(rsl * sdl, bn2)) {
    vls = vl; wls = wl_; byls = byl; bzls = bzl;
  } else {
    double fv = bn * (sm - ul) / denl;
    double fb = (rsl * sdl - bn2) / denl;
    vls = vl - byl * fv; wls = wl_ - bzl * fv;
    byls = byl * fb; bzls = bzl * fb;
  }
  double vrs, wrs, byrs, bzrs;
  double denr = rsr * smr - bn2;
  if (fabs(denr) <= 1e-12 * mx(rsr * sdr, bn2)) {
    vrs = vr; wrs = wr_; byrs = byr; bzrs = bzr;
  } else {
    double fv = bn * (sm - ur) / denr;
    double fb = (rsr * sdr - bn2) / denr;
    vrs = vr - byr * fv; wrs = wr_ - bzr * fv;
    byrs = byr * fb; bzrs = bzr * fb;
  }
  double vbl = ul * bn + vl * byl + wl_ * bzl;
  double vbr = ur * bn + vr * byr + wr_ * bzr;
  double vbls = sm * bn + vls * byls + wls * bzls;
  double vbrs = sm * bn + vrs * byrs + wrs * bzrs;
  double els = (((sdl * el - ptl * ul) + pts * sm) + bn * (vbl - vbls)) / sml;
  double ers = (((sdr * er - ptr * ur) + pts * sm) + bn * (vbr - vbrs)) / smr;

  double sqrl = sqrt(rls), sqrr = sqrt(rrs);
  double sls = sm - fabs(bn) / sqrl;
  double srs = sm + fabs(bn) / sqrr;

  /* double-star states */
  double sgn = (bn >= 0.0) ? 1.0 : -1.0;
  double ssum = sqrl + sqrr;
  double vss = ((sqrl * vls + sqrr * vrs) + sgn * (byrs - byls)) / ssum;
  double wss = ((sqrl * wls + sqrr * wrs) + sgn * (bzrs - bzls)) / ssum;
  double byss = ((sqrl * byrs + sqrr * byls) + sgn * (sqrl * sqrr) * (vrs - vls)) / ssum;
  double bzss = ((sqrl * bzrs + sqrr * bzls) + sgn * (sqrl * sqrr) * (wrs - wls)) / ssum;
  double vbss = sm * bn + vss * byss + wss * bzss;
  double elss = els - sqrl * (vbls - vbss) * sgn;
  double erss = ers + sqrr * (vbrs - vbss) * sgn;

  o->sl = sl; o->sls = sls; o->sm = sm; o->srs = srs; o->sr = sr;
  double a0l[8] = {rl, rl * ul, rl * vl, rl * wl_, el, bn, byl, bzl};
  double a0r[8] = {rr, rr * ur, rr * vr, rr * wr_, er, bn, byr, bzr};
  double asl[8] = {rls, rls * sm, rls * vls, rls * wls, els, bn, byls, bzls};
  double asr[8] = {rrs, rrs * sm, rrs * vrs, rrs * wrs, ers, bn, byrs, bzrs};
  double assl[8] = {rls, rls * sm, rls * vss, rls * wss, elss, bn, byss, bzss};
  double assr[8] = {rrs, rrs * sm, rrs * vss, rrs * wss, erss, bn, byss, bzss};
  memcpy(o->u0l, a0l, sizeof a0l); memcpy(o->u0r, a0r, sizeof a0r);
  memcpy(o->usl, asl, sizeof asl); memcpy(o->usr, asr, sizeof asr);
  memcpy(o->ussl, assl, sizeof assl); memcpy(o->ussr, assr, sizeof assr);
}

/* HLLD flux along axis d between xyz primitive states wl (lower side) and wr
 * (upper side) with interface normal field bn.  Region selection is
 * left-closed: 0<=S_L -> F_L; S_L<0<=S_L* -> F_L* = F_L + S_L (U_L* - U_L);
 * S_L*<0<=S_M -> F_L** = F_L* + S_L* (U_L** - U_L*); S_M<0<=S_R* -> F_R**;
 * S_R*<0<=S_R -> F_R*; S_R<0 -> F_R.
 * *upw receives the upwind side of the contact used by the EMF upwinding:
 * +1 if S_L >= 0 or S_M > eps_up (S_R - S_L), -1 if S_R < 0 or
 * S_M < -eps_up (S_R - S_L), 0 otherwise.  In every star region the mass flux
 * is rho* S_M, so this is the sign of the mass flux with rounding-level
 * contact speeds counted as zero. */
ORC_EXPORT void orc_hlld(int32_t d, const double *wl, const double *wr, double bn,
                         double gamma, double eps_up, double *fout, double *upw) {
  double igm1 = 1.0 / (gamma - 1.0);
  double L[8], R[8], f[8];
  hlld_fan o;
  rot_in(d, wl, L);
  rot_in(d, wr, R);
  hlld_fan_solve(L, R, bn, gamma, igm1, &o);
  if (o.sl >= 0.0) {
    memcpy(f, o.fl, sizeof f);
    *upw = 1.0;
  } else if (o.sr < 0.0) {
    memcpy(f, o.fr, sizeof f);
    *upw = -1.0;
  } else {
    double tie = eps_up * (o.sr - o.sl);
    *upw = (o.sm > tie) ? 1.0 : ((o.sm < -tie) ? -1.0 : 0.0);
    for (int q = 0; q < 8; ++q) {
      if (o.sls >= 0.0) {
        f[q] = o.fl[q] + o.sl * (o.usl[q] - o.u0l[q]);
      } else if (o.sm >= 0.0) {
        double fs = o.fl[q] + o.sl * (o.usl[q] - o.u0l[q]);
        f[q] = fs + o.sls * (o.ussl[q] - o.usl[q]);
      } else if (o.srs >= 0.0) {
        double fs = o.fr[q] + o.sr * (o.usr[q] - o.u0r[q]);
        f[q] = fs + o.srs * (o.ussr[q] - o.usr[q]);
      } else {
        f[q] = o.fr[q] + o.sr * (o.usr[q] - o.u0r[q]);
      }
    }
  }
  rot_out(d, f, fout);
}

/* Debug view of the fan for the tests: speeds[5] = S_L, S_L*, S_M, S_R*, S_R;
 * states[6*8] = U_L, U_L*, U_L**, U_R**, U_R*, U_R; fluxes[2*8] = F_L, F_R
 * (all rotated along axis d). */
ORC_EXPORT void orc_hlld_fan(int32_t d, const double *wl, const double *wr, double bn,
                             double gamma, double *speeds, double *states, double *fluxes) {
  double igm1 = 1.0 / (gamma - 1.0);
  double L[8], R[8];
  hlld_fan o;
  rot_in(d, wl, L);
  rot_in(d, wr, R);
  hlld_fan_solve(L, R, bn, gamma, igm1, &o);
  speeds[0] = o.sl; speeds[1] = o.sls; speeds[2] = o.sm; speeds[3] = o.srs; speeds[4] = o.sr;
  memcpy(states + 0, o.u0l, 8 * sizeof(double));
  memcpy(states + 8, o.usl, 8 * sizeof(double));
  memcpy(states + 16, o.ussl, 8 * sizeof(double));
  memcpy(states + 24, o.ussr, 8 * sizeof(double));
  memcpy(states + 32, o.usr, 8 * sizeof(double));
  memcpy(states + 40, o.u0r, 8 * sizeof(double));
  memcpy(fluxes, o.fl, 8 * sizeof(double));
  memcpy(fluxes + 8, o.fr, 8 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* patch helpers                                                        */
/* ------------------------------------------------------------------ */
static int64_t ix(const orc_patch *P, int i, int j, int k) {
  return (int64_t)i * P->s[0] + (int64_t)j * P->s[1] + (int64_t)k * P->s[2];
}
static int64_t nelem(const orc_patch *P) {
  int nz = P->n[2] + 2 * P->g;
  return P->s[2] * (int64_t)(nz + 1);
}
static double *tmp(const orc_patch *P) {
  return (double *)calloc((size_t)nelem(P), sizeof(double));
}

/* primitive state of cell (i,j,k); Bc = mean of the two face values */
static void cell_prim(const orc_patch *P, int i, int j, int k, double gm1, double *w) {
  int64_t c = ix(P, i, j, k);
  double u[8];
  for (int q = 0; q < 5; ++q) u[q] = P->U[q][c];
  u[5] = 0.5 * (P->B[0][c] + P->B[0][c + P->s[0]]);
  u[6] = 0.5 * (P->B[1][c] + P->B[1][c + P->s[1]]);
  u[7] = 0.5 * (P->B[2][c] + P->B[2][c + P->s[2]]);
  cons2prim(u, gm1, w);
}

/* ------------------------------------------------------------------ */
/* periodic ghost fill (single patch covering a periodic domain)        */
/* ------------------------------------------------------------------ */
ORC_EXPORT void orc_copy(const orc_patch *Ps, const int32_t *sglo, const orc_patch *Pd,
                         const int32_t *dglo, const int32_t *lo, const int32_t *hi,
                         const int32_t *off, int32_t pass);

/* Periodic ghost fill of one patch that covers its periodic domain: every
 * periodic image of the interior (offsets of up to ceil((g+1)/n) periods
 * along each axis) that overlaps the ghost-extended box grown by one cell is
 * copied with the rule of orc_copy (cells and lower faces in pass 0, upper
 * faces in pass 1; the patch's own interior faces are never written). */
ORC_EXPORT void orc_fill_periodic(const orc_patch *P) {
  const int g = P->g;
  const int32_t glo[3] = {0, 0, 0};
  int r[3];
  for (int d = 0; d < 3; ++d) r[d] = (g + P->n[d]) / P->n[d];
  for (int pass = 0; pass < 2; ++pass)
    for (int oz = -r[2]; oz <= r[2]; ++oz)
      for (int oy = -r[1]; oy <= r[1]; ++oy)
        for (int ox = -r[0]; ox <= r[0]; ++ox) {
          int o[3] = {ox, oy, oz};
          if (!ox && !oy && !oz) continue;
          int32_t lo[3], hi[3], off[3];
          int empty = 0;
          for (int d = 0; d < 3; ++d) {
            int a = o[d] * P->n[d], b = a + P->n[d] - 1;
            lo[d] = a > -g - 1 ? a : -g - 1;
            hi[d] = b < P->n[d] + g ? b : P->n[d] + g;
            off[d] = -o[d] * P->n[d];
            if (lo[d] > hi[d]) empty = 1;
          }
          if (empty) continue;
          orc_copy(P, glo, P, glo, lo, hi, off, pass);
        }
}

/* ------------------------------------------------------------------ */
/* CFL time step                                                        */
/* ------------------------------------------------------------------ */
/* dt = cfl * min over interior cells, min over axes d, of
 *      dx_d / (|v_d| + c_f,d). */
ORC_EXPORT double orc_cfl_dt(const orc_patch *P, const orc_params *prm) {
  const int g = P->g;
  const double gm1 = prm->gamma - 1.0;
  double m = INFINITY;
  ORC_STAGE(8);
#pragma omp parallel for collapse(2) reduction(min : m)
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) {
        double w[8];
        cell_prim(P, i, j, k, gm1, w);
        for (int d = 0; d < 3; ++d) {
          int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          double cf = orc_fast_speed(w[0], w[4], w[5 + d], w[5 + t1], w[5 + t2], prm->gamma);
          double t = P->dx[d] / (fabs(w[1 + d]) + cf);
          m = mn(m, t);
        }
      }
  return prm->cfl * m;
}

/* ------------------------------------------------------------------ */
/* flux-register capture                                                */
/* ------------------------------------------------------------------ */
/* One capture item: the fluxes dt*F (components rho, Mx, My, Mz, E) on the
 * axis-d faces whose array indices lie in [lo, hi] (face index along d,
 * cell indices across) are written (mode 0) or added (mode 1) to dst, laid
 * out x fastest over the box, component slowest. */
typedef struct {
  int32_t d;
  int32_t lo[3], hi[3];
  int32_t mode;
  double *dst;
} orc_capture;

/* One EMF capture item: dt*E_a on the axis-a edges whose array indices lie in
 * [lo, hi] are written or added to dst (x fastest). */
typedef struct {
  int32_t a;
  int32_t lo[3], hi[3];
  int32_t mode;
  double *dst;
} orc_ecapture;

/* ------------------------------------------------------------------ */
/* floors (reading R33)                                                  */
/* ------------------------------------------------------------------ */
/* One cell (i, j, k) under the floors of prm: a density below rho_floor is
 * set to rho_floor with M kept and the pressure reset to p_floor (E =
 * p_floor / (gamma - 1) + |M|^2 / (2 rho_floor) + |Bc|^2 / 2); otherwise a
 * pressure below p_floor gets E += (p_floor - p) / (gamma - 1).  Bc is the
 * mean of the cell's two faces.  Returns 1 if the cell was changed. */
static int floor_cell(const orc_patch *P, int i, int j, int k, const orc_params *prm) {
  const double gm1 = prm->gamma - 1.0;
  int64_t c = ix(P, i, j, k);
  double w[8];
  cell_prim(P, i, j, k, gm1, w);
  if (prm->rho_floor > 0.0 && !(w[0] >= prm->rho_floor)) {
    double mx = P->U[1][c], my = P->U[2][c], mz = P->U[3][c];
    double ke = 0.5 * (mx * mx + my * my + mz * mz) / prm->rho_floor;
    double me = 0.5 * (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]);
    P->U[0][c] = prm->rho_floor;
    P->U[4][c] = (prm->p_floor / gm1 + ke) + me;
    return 1;
  }
  if (prm->p_floor > 0.0 && w[4] < prm->p_floor) {
    double add = (prm->p_floor - w[4]) / gm1;
    P->U[4][c] = P->U[4][c] + add;
    return 1;
  }
  return 0;
}

/* The floors applied to every interior cell of P (after refluxing, which
 * changes cells outside any advance).  Returns the number of changed cells. */
ORC_EXPORT int64_t orc_floor(const orc_patch *P, const orc_params *prm) {
  const int g = P->g;
  int64_t n = 0;
  if (!(prm->p_floor > 0.0 || prm->rho_floor > 0.0)) return 0;
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) n += floor_cell(P, i, j, k, prm);
  return n;
}

/* ------------------------------------------------------------------ */
/* the patch advance                                                    */
/* ------------------------------------------------------------------ */
/* One step of length dt of the cells in the update box = interior grown by k
 * layers (Sec. 2.3 extended ghosts; requires k + 2 <= g), together with the
 * face fields on that box.  Data must be valid on the interior grown by k+2.
 * Returns the number of updated cells with rho <= 0 or p <= 0 (or NaN), or -1
 * on bad arguments.  cap/ecap capture dt*F and dt*E for flux registers. */
ORC_EXPORT int64_t orc_advance(const orc_patch *P, const orc_params *prm, double dt,
                               int32_t kgrow, const orc_capture *cap, int32_t ncap,
                               const orc_ecapture *ecap, int32_t necap) {
  const int g = P->g;
  if (kgrow < 0 || kgrow + 2 > g) return -1;
  const double gamma = prm->gamma;
  const double gm1 = gamma - 1.0;
  const double igm1 = 1.0 / gm1;
  const int lim = prm->limiter;
  const int64_t *s = P->s;
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = g - kgrow;
    hi[d] = g + P->n[d] - 1 + kgrow;
  }
  double hdt = 0.5 * dt;
  double hdtdx[3], dtdx[3];
  for (int d = 0; d < 3; ++d) {
    hdtdx[d] = hdt / P->dx[d];
    dtdx[d] = dt / P->dx[d];
  }


  ORC_STAGE(1);
  /* ---- stage 1: primitives and cell-centred E^n = -v x Bc on UB+2 ---- */
  double *W[8], *En[3];
  for (int q = 0; q < 8; ++q) W[q] = tmp(P);
  for (int a = 0; a < 3; ++a) En[a] = tmp(P);
#pragma omp parallel for collapse(2)
  for (int k = lo[2] - 2; k <= hi[2] + 2; ++k)
    for (int j = lo[1] - 2; j <= hi[1] + 2; ++j)
      for (int i = lo[0] - 2; i <= hi[0] + 2; ++i) {
        double w[8];
        int64_t c = ix(P, i, j, k);
        cell_prim(P, i, j, k, gm1, w);
        /* the floors (R33) also bound the primitives the step reads, ghost
         * cells included (a prolonged ghost next to a copied face can have
         * a pressure below them) */
        if (prm->rho_floor > 0.0 && !(w[0] >= prm->rho_floor)) w[0] = prm->rho_floor;
        if (prm->p_floor > 0.0 && !(w[4] >= prm->p_floor)) w[4] = prm->p_floor;
        for (int q = 0; q < 8; ++q) W[q][c] = w[q];
        for (int a = 0; a < 3; ++a) {
          int b = (a + 1) % 3, cc = (a + 2) % 3;
          En[a][c] = w[1 + cc] * w[5 + b] - w[1 + b] * w[5 + cc];
        }
      }


  ORC_STAGE(2);
  /* ---- stage 2: slopes, face values, Hancock predictor on UB+1 ---- */
  /* Wf[(d*2+side)*8+q]: side 0 = lower face of the cell, 1 = upper face */
  double *Wf[48], *Er[3];
  for (int q = 0; q < 48; ++q) Wf[q] = tmp(P);
  for (int a = 0; a < 3; ++a) Er[a] = tmp(P);
#pragma omp parallel for collapse(2)
  for (int k = lo[2] - 1; k <= hi[2] + 1; ++k)
    for (int j = lo[1] - 1; j <= hi[1] + 1; ++j)
      for (int i = lo[0] - 1; i <= hi[0] + 1; ++i) {
        int64_t c = ix(P, i, j, k);
        double w[8], dw[3][8], fw[3][2][8];
        for (int q = 0; q < 8; ++q) w[q] = W[q][c];
        for (int d = 0; d < 3; ++d)
          for (int q = 0; q < 8; ++q) {
            double a = w[q] - W[q][c - s[d]];
            double b = W[q][c + s[d]] - w[q];
            dw[d][q] = orc_limiter(lim, a, b);
          }
        /* face values and the first positivity rule */
        int bad = 0;
        for (int d = 0; d < 3; ++d)
          for (int q = 0; q < 8; ++q) {
            fw[d][0][q] = w[q] - 0.5 * dw[d][q];
            fw[d][1][q] = w[q] + 0.5 * dw[d][q];
          }
        for (int d = 0; d < 3; ++d)
          for (int sd = 0; sd < 2; ++sd)
            if (!(fw[d][sd][0] > 0.0) || !(fw[d][sd][4] > 0.0)) bad = 1;
        if (bad)
          for (int d = 0; d < 3; ++d)
            for (int sd = 0; sd < 2; ++sd)
              for (int q = 0; q < 8; ++q) fw[d][sd][q] = w[q];
        /* Hancock increment dU = -(dt/2) sum_d (F_d(W_{d+}) - F_d(W_{d-}))/dx_d */
        double du[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          double fp[8], fm[8];
          orc_flux(d, fw[d][1], gamma, fp);
          orc_flux(d, fw[d][0], gamma, fm);
          for (int q = 0; q < 8; ++q) du[q] = du[q] - hdtdx[d] * (fp[q] - fm[q]);
        }
        /* predicted face states and the second positivity rule */
        double pw[3][2][8];
        int bad2 = 0;
        for (int d = 0; d < 3; ++d)
          for (int sd = 0; sd < 2; ++sd) {
            double u[8];
            prim2cons(fw[d][sd], igm1, u);
            for (int q = 0; q < 8; ++q) u[q] = u[q] + du[q];
            cons2prim(u, gm1, pw[d][sd]);
            if (!(pw[d][sd][0] > 0.0) || !(pw[d][sd][4] > 0.0)) bad2 = 1;
          }
        if (bad2) {
          for (int d = 0; d < 3; ++d)
            for (int sd = 0; sd < 2; ++sd)
              for (int q = 0; q < 8; ++q) pw[d][sd][q] = w[q];
          for (int q = 0; q < 8; ++q) du[q] = 0.0;
        }
        for (int d = 0; d < 3; ++d)
          for (int sd = 0; sd < 2; ++sd)
            for (int q = 0; q < 8; ++q) Wf[(d * 2 + sd) * 8 + q][c] = pw[d][sd][q];
        /* reference cell EMF from U^{n+1/2} = U^n + dU */
        double uh[8], uc[8];
        prim2cons(w, igm1, uc);
        for (int q = 0; q < 8; ++q) uh[q] = uc[q] + du[q];
        double ir = 1.0 / uh[0];
        double v[3] = {uh[1] * ir, uh[2] * ir, uh[3] * ir};
        for (int a = 0; a < 3; ++a) {
          int b = (a + 1) % 3, cc = (a + 2) % 3;
          Er[a][c] = v[cc] * uh[5 + b] - v[b] * uh[5 + cc];
        }
      }


  ORC_STAGE(3);
  /* ---- stage 3: edge E^n = mean of the four neighbouring cell values ---- */
  /* Ee[a] at cell index c is the axis-a edge at the lower b and lower c corner */
  double *Ee[3];
  for (int a = 0; a < 3; ++a) Ee[a] = tmp(P);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    int elo[3], ehi[3];
    for (int d = 0; d < 3; ++d) { elo[d] = lo[d] - 1; ehi[d] = hi[d] + 2; }
    elo[a] = lo[a] - 1; ehi[a] = hi[a] + 1;
#pragma omp parallel for collapse(2)
    for (int k = elo[2]; k <= ehi[2]; ++k)
      for (int j = elo[1]; j <= ehi[1]; ++j)
        for (int i = elo[0]; i <= ehi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          double e00 = En[a][c - s[b] - s[cc]];
          double e10 = En[a][c - s[cc]];
          double e01 = En[a][c - s[b]];
          double e11 = En[a][c];
          Ee[a][c] = 0.25 * (e00 + e10 + e01 + e11);
        }
  }


  ORC_STAGE(4);
  /* ---- stage 4: face-normal B at n+1/2 (CT half step) ---- */
  double *Bh[3];
  for (int a = 0; a < 3; ++a) Bh[a] = tmp(P);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    int flo[3], fhi[3];
    for (int d = 0; d < 3; ++d) { flo[d] = lo[d] - 1; fhi[d] = hi[d] + 1; }
    flo[a] = lo[a]; fhi[a] = hi[a] + 1;
#pragma omp parallel for collapse(2)
    for (int k = flo[2]; k <= fhi[2]; ++k)
      for (int j = flo[1]; j <= fhi[1]; ++j)
        for (int i = flo[0]; i <= fhi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          double dEc = Ee[cc][c + s[b]] - Ee[cc][c];
          double dEb = Ee[b][c + s[cc]] - Ee[b][c];
          Bh[a][c] = P->B[a][c] - (hdtdx[b] * dEc - hdtdx[cc] * dEb);
        }
  }


  ORC_STAGE(5);
  /* ---- stage 5: HLLD fluxes on the faces ---- */
  double *F[3][8], *Up[3];
  for (int d = 0; d < 3; ++d) {
    for (int q = 0; q < 8; ++q) F[d][q] = tmp(P);
    Up[d] = tmp(P);
  }
  for (int d = 0; d < 3; ++d) {
    int flo[3], fhi[3];
    for (int e = 0; e < 3; ++e) { flo[e] = lo[e] - 1; fhi[e] = hi[e] + 1; }
    flo[d] = lo[d]; fhi[d] = hi[d] + 1;
#pragma omp parallel for collapse(2)
    for (int k = flo[2]; k <= fhi[2]; ++k)
      for (int j = flo[1]; j <= fhi[1]; ++j)
        for (int i = flo[0]; i <= fhi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          double wl[8], wr[8], f[8], up;
          for (int q = 0; q < 8; ++q) {
            wl[q] = Wf[(d * 2 + 1) * 8 + q][c - s[d]];
            wr[q] = Wf[(d * 2 + 0) * 8 + q][c];
          }
          orc_hlld(d, wl, wr, Bh[d][c], gamma, prm->upwind_eps, f, &up);
          for (int q = 0; q < 8; ++q) F[d][q][c] = f[q];
          Up[d][c] = up;
        }
  }


  ORC_STAGE(6);
  /* ---- stage 6: edge EMFs on the edges of the update box ---- */
  double *Ed[3];
  for (int a = 0; a < 3; ++a) Ed[a] = tmp(P);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    int elo[3], ehi[3];
    for (int d = 0; d < 3; ++d) { elo[d] = lo[d]; ehi[d] = hi[d] + 1; }
    ehi[a] = hi[a];
#pragma omp parallel for collapse(2)
    for (int k = elo[2]; k <= ehi[2]; ++k)
      for (int j = elo[1]; j <= ehi[1]; ++j)
        for (int i = elo[0]; i <= ehi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          /* face EMFs: E_a = -F_b[B_c] on b-faces, +F_c[B_b] on c-faces */
          double eb_lo = -F[b][5 + cc][c - s[cc]];
          double eb_hi = -F[b][5 + cc][c];
          double ec_lo = F[cc][5 + b][c - s[b]];
          double ec_hi = F[cc][5 + b][c];
          double avg = 0.25 * (eb_lo + eb_hi + ec_lo + ec_hi);
          if (prm->emf == 1) {
            Ed[a][c] = avg;
            continue;
          }
          double r00 = Er[a][c - s[b] - s[cc]];
          double r10 = Er[a][c - s[cc]];
          double r01 = Er[a][c - s[b]];
          double r11 = Er[a][c];
          double mb_lo = Up[b][c - s[cc]];
          double mb_hi = Up[b][c];
          double mc_lo = Up[cc][c - s[b]];
          double mc_hi = Up[cc][c];
          double dc14, dc34, db14, db34;
          /* derivative along c at c-1/4, upwinded by the b-face contact side at row c */
          if (mb_hi > 0.0) dc14 = r01 - ec_lo;
          else if (mb_hi < 0.0) dc14 = r11 - ec_hi;
          else dc14 = 0.5 * ((r01 - ec_lo) + (r11 - ec_hi));
          /* along c at c-3/4, upwinded by the b-face contact side at row c-1 */
          if (mb_lo > 0.0) dc34 = ec_lo - r00;
          else if (mb_lo < 0.0) dc34 = ec_hi - r10;
          else dc34 = 0.5 * ((ec_lo - r00) + (ec_hi - r10));
          /* along b at b-1/4, upwinded by the c-face contact side at column b */
          if (mc_hi > 0.0) db14 = r10 - eb_lo;
          else if (mc_hi < 0.0) db14 = r11 - eb_hi;
          else db14 = 0.5 * ((r10 - eb_lo) + (r11 - eb_hi));
          /* along b at b-3/4, upwinded by the c-face contact side at column b-1 */
          if (mc_lo > 0.0) db34 = eb_lo - r00;
          else if (mc_lo < 0.0) db34 = eb_hi - r01;
          else db34 = 0.5 * ((eb_lo - r00) + (eb_hi - r01));
          Ed[a][c] = avg + 0.25 * (dc34 - dc14 + db34 - db14);
        }
  }

  /* ---- flux-register capture (before the state is overwritten) ---- */
  for (int t = 0; t < ncap; ++t) {
    const orc_capture *C = &cap[t];
    int nx = C->hi[0] - C->lo[0] + 1, ny = C->hi[1] - C->lo[1] + 1, nz = C->hi[2] - C->lo[2] + 1;
    int64_t nb = (int64_t)nx * ny * nz;
    for (int k = C->lo[2]; k <= C->hi[2]; ++k)
      for (int j = C->lo[1]; j <= C->hi[1]; ++j)
        for (int i = C->lo[0]; i <= C->hi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          int64_t o = (int64_t)(i - C->lo[0]) + (int64_t)nx * ((j - C->lo[1]) + (int64_t)ny * (k - C->lo[2]));
          for (int q = 0; q < 5; ++q) {
            double v = dt * F[C->d][q][c];
            if (C->mode == 0) C->dst[q * nb + o] = v;
            else C->dst[q * nb + o] = C->dst[q * nb + o] + v;
          }
        }
  }
  for (int t = 0; t < necap; ++t) {
    const orc_ecapture *C = &ecap[t];
    int nx = C->hi[0] - C->lo[0] + 1, ny = C->hi[1] - C->lo[1] + 1;
    for (int k = C->lo[2]; k <= C->hi[2]; ++k)
      for (int j = C->lo[1]; j <= C->hi[1]; ++j)
        for (int i = C->lo[0]; i <= C->hi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          int64_t o = (int64_t)(i - C->lo[0]) + (int64_t)nx * ((j - C->lo[1]) + (int64_t)ny * (k - C->lo[2]));
          double v = dt * Ed[C->a][c];
          if (C->mode == 0) C->dst[o] = v;
          else C->dst[o] = C->dst[o] + v;
        }
  }


  ORC_STAGE(7);
  /* ---- stage 7: conservative cell update and CT face update ---- */
  int64_t nneg = 0;
#pragma omp parallel for collapse(2) reduction(+ : nneg)
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int64_t c = ix(P, i, j, k);
        for (int q = 0; q < 5; ++q) {
          double u = P->U[q][c];
          u = u - dtdx[0] * (F[0][q][c + s[0]] - F[0][q][c])
                - dtdx[1] * (F[1][q][c + s[1]] - F[1][q][c])
                - dtdx[2] * (F[2][q][c + s[2]] - F[2][q][c]);
          P->U[q][c] = u;
        }
      }
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    int flo[3], fhi[3];
    for (int d = 0; d < 3; ++d) { flo[d] = lo[d]; fhi[d] = hi[d]; }
    fhi[a] = hi[a] + 1;
#pragma omp parallel for collapse(2)
    for (int k = flo[2]; k <= fhi[2]; ++k)
      for (int j = flo[1]; j <= fhi[1]; ++j)
        for (int i = flo[0]; i <= fhi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          double dEc = Ed[cc][c + s[b]] - Ed[cc][c];
          double dEb = Ed[b][c + s[cc]] - Ed[b][c];
          P->B[a][c] = P->B[a][c] - (dtdx[b] * dEc - dtdx[cc] * dEb);
        }
  }
  /* floors (reading R33; off when p_floor and rho_floor are 0) */
  int64_t nfl = 0;
  if (prm->p_floor > 0.0 || prm->rho_floor > 0.0) {
#pragma omp parallel for collapse(2) reduction(+ : nfl)
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) nfl += floor_cell(P, i, j, k, prm);
  }
  orc_floored = nfl;
  /* positivity of the new state (status only) */
#pragma omp parallel for collapse(2) reduction(+ : nneg)
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        double w[8];
        cell_prim(P, i, j, k, gm1, w);
        if (!(w[0] > 0.0) || !(w[4] > 0.0)) nneg += 1;
      }

  for (int q = 0; q < 8; ++q) free(W[q]);
  for (int q = 0; q < 48; ++q) free(Wf[q]);
  for (int a = 0; a < 3; ++a) {
    free(En[a]); free(Er[a]); free(Ee[a]); free(Bh[a]); free(Ed[a]);
  }
  for (int d = 0; d < 3; ++d) {
    for (int q = 0; q < 8; ++q) free(F[d][q]);
    free(Up[d]);
  }
  return nneg;
}

/* ------------------------------------------------------------------ */
/* error flagging for regridding (Sec. 2.1)                             */
/* ------------------------------------------------------------------ */
/* The paper leaves the refinement criterion to the application.  Reading:
 * an interior cell is flagged when the normalised central difference of the
 * density or of the pressure along some axis exceeds theta,
 *   eta = |q(+d) - q(-d)| / (|q(+d)| + 2 |q| + |q(-d)|) > theta,
 * q in {rho, p} (p from the cell-centred field), d in {x, y, z}; eta lies in
 * [0, 1].  flags: one byte per interior cell, x fastest (1 = flagged).
 * Needs one valid ghost layer.  Returns the number of flagged cells. */
ORC_EXPORT int64_t orc_flag(const orc_patch *P, const orc_params *prm, double theta, uint8_t *flags) {
  const int g = P->g;
  const double gm1 = prm->gamma - 1.0;
  int64_t count = 0;
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) {
        double w[8], wm[8], wp[8];
        cell_prim(P, i, j, k, gm1, w);
        int f = 0;
        for (int d = 0; d < 3; ++d) {
          int im = i - (d == 0), jm = j - (d == 1), km = k - (d == 2);
          int ip = i + (d == 0), jp = j + (d == 1), kp = k + (d == 2);
          cell_prim(P, im, jm, km, gm1, wm);
          cell_prim(P, ip, jp, kp, gm1, wp);
          for (int t = 0; t < 2; ++t) {
            int q = t ? 4 : 0;
            double num = fabs(wp[q] - wm[q]);
            double den = fabs(wp[q]) + 2.0 * fabs(w[q]) + fabs(wm[q]);
            if (num > theta * den) f = 1;
          }
        }
        int64_t o = (int64_t)(i - g) + (int64_t)P->n[0] * ((j - g) + (int64_t)P->n[1] * (k - g));
        flags[o] = (uint8_t)f;
        count += f;
      }
  return count;
}

/* ------------------------------------------------------------------ */
/* conservation sums                                                    */
/* ------------------------------------------------------------------ */
/* out[q] = sum over interior cells of U_q * dV (q < 5) and, for q = 5..7,
 * the sum over the lower faces of the interior cells of B_{q-5} * dV,
 * accumulated serially in k, j, i order. */
ORC_EXPORT void orc_sums(const orc_patch *P, double *out) {
  const int g = P->g;
  double dv = P->dx[0] * P->dx[1] * P->dx[2];
  for (int q = 0; q < 8; ++q) out[q] = 0.0;
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) {
        int64_t c = ix(P, i, j, k);
        for (int q = 0; q < 5; ++q) out[q] += P->U[q][c] * dv;
        for (int a = 0; a < 3; ++a) out[5 + a] += P->B[a][c] * dv;
      }
}

/* max over interior cells of |div B| * min(dx) / max|B_face| (relative). */
ORC_EXPORT double orc_divb_max(const orc_patch *P) {
  const int g = P->g;
  double m = 0.0;
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) {
        int64_t c = ix(P, i, j, k);
        double dvb = (P->B[0][c + P->s[0]] - P->B[0][c]) / P->dx[0]
                   + (P->B[1][c + P->s[1]] - P->B[1][c]) / P->dx[1]
                   + (P->B[2][c + P->s[2]] - P->B[2][c]) / P->dx[2];
        m = mx(m, fabs(dvb));
      }
  return m;
}

/* ================================================================== */
/* AMR level operations (Sec. 2.2: Prolongation, Restriction, flux      */
/* synchronisation), refinement ratio R = 2.  A fine patch is aligned   */
/* to its coarse level (even lower index, even extent); fine global     */
/* index = 2 * coarse global index + {0, 1}.                            */
/* ================================================================== */

/* global -> array index of a patch whose interior starts at global lo */
static int gidx(int global, int lo, int g) { return global - lo + g; }

static double minmod2(double a, double b) { return orc_limiter(1, a, b); }

/* thermal energy E - |M|^2/(2 rho) - |Bc|^2/2 of cell c (Bc = face means) */
static double thermal(const orc_patch *P, int64_t c) {
  double rho = P->U[0][c];
  double ke = 0.5 * (P->U[1][c] * P->U[1][c] + P->U[2][c] * P->U[2][c] + P->U[3][c] * P->U[3][c]) / rho;
  double bx = 0.5 * (P->B[0][c] + P->B[0][c + P->s[0]]);
  double by = 0.5 * (P->B[1][c] + P->B[1][c + P->s[1]]);
  double bz = 0.5 * (P->B[2][c] + P->B[2][c + P->s[2]]);
  double me = 0.5 * (bx * bx + by * by + bz * bz);
  return P->U[4][c] - ke - me;
}

/* fine axis-a face at position pos (0 lower coarse face, 1 inner, 2 upper)
 * and transverse sub-indices sub[] of the reconstruction in one coarse cell */
static double pface(int a, int pos, const int *sub, double m[3][2], double qs[3][2][3],
                    double lin[3][3], const double *c0) {
  int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
  if (pos == 1) {
    double sl = sub[lo_t] ? 0.5 * lin[a][lo_t] : -0.5 * lin[a][lo_t];
    double sh = sub[hi_t] ? 0.5 * lin[a][hi_t] : -0.5 * lin[a][hi_t];
    return c0[a] + sl + sh;
  }
  int sd = pos == 2;
  double sl = sub[lo_t] ? qs[a][sd][lo_t] : -qs[a][sd][lo_t];
  double sh = sub[hi_t] ? qs[a][sd][hi_t] : -qs[a][sd][hi_t];
  return m[a][sd] + sl + sh;
}


/* Prolongation of the coarse cells of box [clo, chi] (coarse global index)
 * of coarse patch Pc (interior starting at global cglo) into fine patch Pf
 * (interior starting at fglo): for each coarse cell, the 8 fine cells and
 * the lower faces of those fine cells (plus the extra upper face where a fine
 * cell is the last of its array), skipping the fine patch's own interior
 * faces.  Density and momentum: U_f = U_c + (+-h_x) + (+-h_y) + (+-h_z), h_d =
 * 0.25 * minmod of the coarse one-sided differences (conservative limited
 * linear).  Total energy: the thermal energy e = E - |M|^2/(2 rho) - |Bc|^2/2
 * is prolonged the same way (so e_f >= e_c / 4 > 0) and E_f = (e_f +
 * |M_f|^2/(2 rho_f)) + |Bc_f|^2/2, Bc_f the mean of the fine cell's two faces
 * of the reconstruction below; prolonging E itself left negative pressure in
 * low-beta ghost cells.
 * Faces: divergence-free reconstruction inside the coarse cell (Balsara
 * 2001 for R = 2): each coarse face gives its mean and its minmod transverse
 * quarter-slopes; the quadratic field Bx = a0 + ax x + ay y + az z + axx x^2 +
 * axy xy + axz xz (and cyclic) matching those traces with div B = 0
 * identically yields the inner faces.  Fine units: the coarse cell is
 * [-1, 1]^3, fine cells have unit width. */
ORC_EXPORT void orc_prolong(const orc_patch *Pc, const int32_t *cglo, const orc_patch *Pf,
                            const int32_t *fglo, const int32_t *clo, const int32_t *chi) {
  const int gc = Pc->g, gf = Pf->g;
  const int64_t *sc = Pc->s, *sf = Pf->s;
  int Nf[3];
  for (int d = 0; d < 3; ++d) Nf[d] = Pf->n[d] + 2 * gf;
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int ci[3] = {gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc)};
        int64_t c = ix(Pc, ci[0], ci[1], ci[2]);
        /* cells */
        double uc[4], h[4][3], ec, he[3];
        for (int q = 0; q < 4; ++q) {
          uc[q] = Pc->U[q][c];
          for (int d = 0; d < 3; ++d) {
            double a = uc[q] - Pc->U[q][c - sc[d]];
            double b = Pc->U[q][c + sc[d]] - uc[q];
            h[q][d] = 0.25 * minmod2(a, b);
          }
        }
        ec = thermal(Pc, c);
        for (int d = 0; d < 3; ++d) {
          double a = ec - thermal(Pc, c - sc[d]);
          double b = thermal(Pc, c + sc[d]) - ec;
          he[d] = 0.25 * minmod2(a, b);
        }
        /* faces: mean and transverse quarter-slopes of the six coarse faces */
        double m[3][2], qs[3][2][3];  /* qs[normal][side][transverse axis] */
        for (int a = 0; a < 3; ++a)
          for (int sd = 0; sd < 2; ++sd) {
            int64_t f = c + (sd ? sc[a] : 0);
            m[a][sd] = Pc->B[a][f];
            for (int t = 0; t < 3; ++t) {
              if (t == a) { qs[a][sd][t] = 0.0; continue; }
              double lo = m[a][sd] - Pc->B[a][f - sc[t]];
              double hi = Pc->B[a][f + sc[t]] - m[a][sd];
              qs[a][sd][t] = 0.25 * minmod2(lo, hi);
            }
          }
        /* polynomial coefficients: lin[a][t] = coefficient of x_t in B_a
         * (t != a), crs[a][t] = coefficient of x_a x_t in B_a */
        double lin[3][3], crs[3][3], sq[3], c0[3];
        for (int a = 0; a < 3; ++a)
          for (int t = 0; t < 3; ++t) {
            if (t == a) { lin[a][t] = 0.0; crs[a][t] = 0.0; continue; }
            lin[a][t] = qs[a][1][t] + qs[a][0][t];
            crs[a][t] = qs[a][1][t] - qs[a][0][t];
          }
        for (int a = 0; a < 3; ++a) {
          int b = (a + 1) % 3, cc = (a + 2) % 3;
          sq[a] = -0.5 * (crs[b][a] + crs[cc][a]);
          c0[a] = 0.5 * (m[a][0] + m[a][1]) - sq[a];
        }
        /* the 8 fine cells */
        for (int fc = 0; fc < 2; ++fc)
          for (int fb = 0; fb < 2; ++fb)
            for (int fa = 0; fa < 2; ++fa) {
              int sub[3] = {fa, fb, fc};
              int fi[3];
              for (int d = 0; d < 3; ++d) fi[d] = gidx(2 * (d == 0 ? I : d == 1 ? J : K) + sub[d], fglo[d], gf);
              int64_t x = ix(Pf, fi[0], fi[1], fi[2]);
              double uf[4];
              for (int q = 0; q < 4; ++q) {
                double u = uc[q];
                u = u + (fa ? h[q][0] : -h[q][0]);
                u = u + (fb ? h[q][1] : -h[q][1]);
                u = u + (fc ? h[q][2] : -h[q][2]);
                uf[q] = u;
                Pf->U[q][x] = u;
              }
              /* face-averaged field of the reconstruction (a function of the
               * coarse data only, so every patch that prolongs this cell gets
               * the same energy) */
              double bc[3];
              for (int a = 0; a < 3; ++a) {
                double f0 = pface(a, sub[a], sub, m, qs, lin, c0);
                double f1 = pface(a, sub[a] + 1, sub, m, qs, lin, c0);
                bc[a] = 0.5 * (f0 + f1);
              }
              double e = ec;
              e = e + (fa ? he[0] : -he[0]);
              e = e + (fb ? he[1] : -he[1]);
              e = e + (fc ? he[2] : -he[2]);
              double kef = 0.5 * (uf[1] * uf[1] + uf[2] * uf[2] + uf[3] * uf[3]) / uf[0];
              double mef = 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
              Pf->U[4][x] = e + kef + mef;
              for (int a = 0; a < 3; ++a) {
                int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
                int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
                /* lower face of this fine cell along a, and (if last) the upper */
                for (int up = 0; up < 2; ++up) {
                  int fidx[3] = {fi[0], fi[1], fi[2]};
                  if (up) {
                    if (fi[a] != Nf[a] - 1) continue;
                    fidx[a] += 1;
                  }
                  int own = 1;
                  for (int e = 0; e < 3; ++e) {
                    int top = (e == a) ? gf + Pf->n[e] : gf + Pf->n[e] - 1;
                    if (fidx[e] < gf || fidx[e] > top) own = 0;
                  }
                  if (own) continue;
                  int pos = sub[a] + up; /* 0 lower coarse face, 1 inner, 2 upper */
                  double v;
                  if (pos == 1) {
                    double sl = sub[lo_t] ? 0.5 * lin[a][lo_t] : -0.5 * lin[a][lo_t];
                    double sh = sub[hi_t] ? 0.5 * lin[a][hi_t] : -0.5 * lin[a][hi_t];
                    v = c0[a] + sl + sh;
                  } else {
                    int sd = pos == 2;
                    double sl = sub[lo_t] ? qs[a][sd][lo_t] : -qs[a][sd][lo_t];
                    double sh = sub[hi_t] ? qs[a][sd][hi_t] : -qs[a][sd][hi_t];
                    v = m[a][sd] + sl + sh;
                  }
                  Pf->B[a][ix(Pf, fidx[0], fidx[1], fidx[2])] = v;
                }
              }
            }
      }
}

/* ================================================================== */
/* Data transfer into a new iteration of a level (regridding, Sec. 2.1; */
/* the O step of Sec. 2.2): a new fine patch takes the previous         */
/* iteration's data where the two meet and is prolonged from its        */
/* parent level elsewhere.                                              */
/* ================================================================== */

/* Copy of one box from an old patch Ps to a new patch Pd of the same level
 * (global indices, both patches' own arrays): kind -1 copies the five cell
 * arrays over the cells of [lo, hi]; kind a (0..2) copies the axis-a face
 * array over the faces of [lo, hi] (index along a = face index). */
ORC_EXPORT void orc_transfer_copy(const orc_patch *Ps, const int32_t *sglo, const orc_patch *Pd,
                                  const int32_t *dglo, int32_t kind, const int32_t *lo, const int32_t *hi) {
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int64_t xs = ix(Ps, gidx(i, sglo[0], Ps->g), gidx(j, sglo[1], Ps->g), gidx(k, sglo[2], Ps->g));
        int64_t xd = ix(Pd, gidx(i, dglo[0], Pd->g), gidx(j, dglo[1], Pd->g), gidx(k, dglo[2], Pd->g));
        if (kind < 0)
          for (int q = 0; q < 5; ++q) Pd->U[q][xd] = Ps->U[q][xs];
        else
          Pd->B[kind][xd] = Ps->B[kind][xs];
      }
}

/* The potential phi = L^+ r on the eight fine cells of a coarse cell (cell c
 * = fa + 2 fb + 4 fc), L the graph Laplacian of the cube (two cells joined by
 * each inner face): through the cube's Walsh functions chi_S(c) = (-1)^|S & c|,
 * eigenvalue 2 |S| for S != 0; the S = 0 part (the coarse cell's net flux,
 * zero up to rounding) is dropped. */
static void cube_potential(const double *r, double *phi) {
  double coef[8];
  coef[0] = 0.0;
  for (int S = 1; S < 8; ++S) {
    double t = 0.0;
    for (int c = 0; c < 8; ++c) {
      int par = __builtin_popcount(S & c) & 1;
      t = par ? t - r[c] : t + r[c];
    }
    int w = __builtin_popcount(S);
    coef[S] = (t * 0.125) / (2.0 * w);
  }
  for (int c = 0; c < 8; ++c) {
    double v = 0.0;
    for (int S = 1; S < 8; ++S) {
      int par = __builtin_popcount(S & c) & 1;
      v = par ? v - coef[S] : v + coef[S];
    }
    phi[c] = v;
  }
}

/* Prolongation of the coarse cells of box [clo, chi] (coarse global index)
 * of Pc into the interior of a new fine patch Pf (cells and every face of
 * the fine cells, the fine patch's own boundary faces included), cell by
 * cell under mask[] (one byte per coarse cell of the box [mlo, mlo + mext),
 * x fastest):
 *   bit 0: the coarse cell's children already hold the previous iteration's
 *          data (copied): nothing is written;
 *   bit 1 + 2 a + s: the four fine sub-faces on side s of axis a already hold
 *          the previous iteration's values: they are kept and read, not
 *          written.
 * Cells: density and momentum limited-linear as orc_prolong; energy with
 * energy_mode 0 as orc_prolong (thermal energy limited-linear, R22), with
 * energy_mode 1 conservatively: the thermal part of the eight children is
 * scaled by (1 + delta / ebar), delta = E_c - mean of the children's total
 * energies, ebar = mean thermal energy, so that the children's energies
 * average to E_c while every thermal energy keeps its sign (unchanged when
 * ebar + delta <= 0; such cells are counted).  Faces: the divergence-free
 * reconstruction of orc_prolong (Balsara 2001) on the coarse faces that are
 * not kept and inside the coarse cell; where some sub-faces are kept, the
 * twelve inner faces are then changed by the least-squares correction that
 * makes every child's divergence zero again (Toth & Roe 2002 fix the inner
 * faces of a refined cell from its boundary sub-faces; here the smallest
 * change of Balsara's values does): delta_f = phi(upper child) - phi(lower
 * child), phi = L^+ r, r the children's divergences (cube_potential).
 * Equal cell widths along the three axes.  Returns the count of energy
 * fallbacks. */
ORC_EXPORT int64_t orc_prolong_new(const orc_patch *Pc, const int32_t *cglo, const orc_patch *Pf,
                                   const int32_t *fglo, const int32_t *clo, const int32_t *chi,
                                   const uint8_t *mask, const int32_t *mlo, const int32_t *mext,
                                   int32_t energy_mode) {
  const int gc = Pc->g, gf = Pf->g;
  const int64_t *sc = Pc->s;
  int64_t nfall = 0;
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int C3[3] = {I, J, K};
        int mk = mask[(I - mlo[0]) + mext[0] * ((J - mlo[1]) + mext[1] * (K - mlo[2]))];
        if (mk & 1) continue;
        int ci[3] = {gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc)};
        int64_t c = ix(Pc, ci[0], ci[1], ci[2]);
        double uc[4], h[4][3], ec, he[3];
        for (int q = 0; q < 4; ++q) {
          uc[q] = Pc->U[q][c];
          for (int d = 0; d < 3; ++d) {
            double a = uc[q] - Pc->U[q][c - sc[d]];
            double b = Pc->U[q][c + sc[d]] - uc[q];
            h[q][d] = 0.25 * minmod2(a, b);
          }
        }
        ec = thermal(Pc, c);
        for (int d = 0; d < 3; ++d) {
          double a = ec - thermal(Pc, c - sc[d]);
          double b = thermal(Pc, c + sc[d]) - ec;
          he[d] = 0.25 * minmod2(a, b);
        }
        double m[3][2], qs[3][2][3];
        for (int a = 0; a < 3; ++a)
          for (int sd = 0; sd < 2; ++sd) {
            int64_t f = c + (sd ? sc[a] : 0);
            m[a][sd] = Pc->B[a][f];
            for (int t = 0; t < 3; ++t) {
              if (t == a) { qs[a][sd][t] = 0.0; continue; }
              double lo = m[a][sd] - Pc->B[a][f - sc[t]];
              double hi = Pc->B[a][f + sc[t]] - m[a][sd];
              qs[a][sd][t] = 0.25 * minmod2(lo, hi);
            }
          }
        double lin[3][3], crs[3][3], sq[3], c0[3];
        for (int a = 0; a < 3; ++a)
          for (int t = 0; t < 3; ++t) {
            if (t == a) { lin[a][t] = 0.0; crs[a][t] = 0.0; continue; }
            lin[a][t] = qs[a][1][t] + qs[a][0][t];
            crs[a][t] = qs[a][1][t] - qs[a][0][t];
          }
        for (int a = 0; a < 3; ++a) {
          int b = (a + 1) % 3, cc = (a + 2) % 3;
          sq[a] = -0.5 * (crs[b][a] + crs[cc][a]);
          c0[a] = 0.5 * (m[a][0] + m[a][1]) - sq[a];
        }
        /* fine faces of this coarse cell: fb_[a][pos][s2][s1] with pos 0
         * lower coarse face, 1 inner, 2 upper; s1 / s2 the sub-index along
         * the lower / higher transverse axis */
        double fv[3][3][2][2];
        int64_t fx[3][3][2][2];
        for (int a = 0; a < 3; ++a) {
          int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
          int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
          for (int pos = 0; pos < 3; ++pos)
            for (int s2 = 0; s2 < 2; ++s2)
              for (int s1 = 0; s1 < 2; ++s1) {
                int g3[3];
                g3[a] = 2 * C3[a] + pos;
                g3[lo_t] = 2 * C3[lo_t] + s1;
                g3[hi_t] = 2 * C3[hi_t] + s2;
                int64_t x = ix(Pf, gidx(g3[0], fglo[0], gf), gidx(g3[1], fglo[1], gf), gidx(g3[2], fglo[2], gf));
                fx[a][pos][s2][s1] = x;
                int keep = pos != 1 && ((mk >> (1 + 2 * a + (pos == 2))) & 1);
                double v;
                if (keep) {
                  v = Pf->B[a][x];
                } else if (pos == 1) {
                  double sl = s1 ? 0.5 * lin[a][lo_t] : -0.5 * lin[a][lo_t];
                  double sh = s2 ? 0.5 * lin[a][hi_t] : -0.5 * lin[a][hi_t];
                  v = c0[a] + sl + sh;
                } else {
                  int sd = pos == 2;
                  double sl = s1 ? qs[a][sd][lo_t] : -qs[a][sd][lo_t];
                  double sh = s2 ? qs[a][sd][hi_t] : -qs[a][sd][hi_t];
                  v = m[a][sd] + sl + sh;
                }
                fv[a][pos][s2][s1] = v;
              }
        }
        if (mk >> 1) {
          /* the children's divergences with the kept sub-faces, then the
           * smallest change of the inner faces that zeroes them */
          double r[8], phi[8];
          for (int cc8 = 0; cc8 < 8; ++cc8) {
            int sub[3] = {cc8 & 1, (cc8 >> 1) & 1, (cc8 >> 2) & 1};
            double dv = 0.0;
            for (int a = 0; a < 3; ++a) {
              int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
              int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
              double up = fv[a][sub[a] + 1][sub[hi_t]][sub[lo_t]];
              double dn = fv[a][sub[a]][sub[hi_t]][sub[lo_t]];
              dv = dv + (up - dn);
            }
            r[cc8] = dv;
          }
          cube_potential(r, phi);
          for (int a = 0; a < 3; ++a) {
            int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
            int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
            for (int s2 = 0; s2 < 2; ++s2)
              for (int s1 = 0; s1 < 2; ++s1) {
                int lo8 = 0, hi8;
                lo8 |= (s1 << lo_t) | (s2 << hi_t);
                hi8 = lo8 | (1 << a);
                fv[a][1][s2][s1] = fv[a][1][s2][s1] + (phi[hi8] - phi[lo8]);
              }
          }
        }
        /* write the faces that are not kept */
        for (int a = 0; a < 3; ++a)
          for (int pos = 0; pos < 3; ++pos) {
            int keep = pos != 1 && ((mk >> (1 + 2 * a + (pos == 2))) & 1);
            if (keep) continue;
            for (int s2 = 0; s2 < 2; ++s2)
              for (int s1 = 0; s1 < 2; ++s1) Pf->B[a][fx[a][pos][s2][s1]] = fv[a][pos][s2][s1];
          }
        /* the eight children */
        double uf[8][4], ef[8], kef[8], mef[8];
        int64_t xf[8];
        for (int cc8 = 0; cc8 < 8; ++cc8) {
          int fa = cc8 & 1, fb = (cc8 >> 1) & 1, fc = (cc8 >> 2) & 1;
          int sub[3] = {fa, fb, fc};
          xf[cc8] = ix(Pf, gidx(2 * I + fa, fglo[0], gf), gidx(2 * J + fb, fglo[1], gf), gidx(2 * K + fc, fglo[2], gf));
          for (int q = 0; q < 4; ++q) {
            double u = uc[q];
            u = u + (fa ? h[q][0] : -h[q][0]);
            u = u + (fb ? h[q][1] : -h[q][1]);
            u = u + (fc ? h[q][2] : -h[q][2]);
            uf[cc8][q] = u;
          }
          double bc[3];
          for (int a = 0; a < 3; ++a) {
            int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
            int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
            bc[a] = 0.5 * (fv[a][sub[a]][sub[hi_t]][sub[lo_t]] + fv[a][sub[a] + 1][sub[hi_t]][sub[lo_t]]);
          }
          double e = ec;
          e = e + (fa ? he[0] : -he[0]);
          e = e + (fb ? he[1] : -he[1]);
          e = e + (fc ? he[2] : -he[2]);
          ef[cc8] = e;
          kef[cc8] = 0.5 * (uf[cc8][1] * uf[cc8][1] + uf[cc8][2] * uf[cc8][2] + uf[cc8][3] * uf[cc8][3]) / uf[cc8][0];
          mef[cc8] = 0.5 * (bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]);
        }
        double scale = 0.0;
        int cons = 0;
        if (energy_mode == 1) {
          double sE = 0.0, se = 0.0;
          for (int cc8 = 0; cc8 < 8; ++cc8) {
            sE = sE + ((ef[cc8] + kef[cc8]) + mef[cc8]);
            se = se + ef[cc8];
          }
          double delta = Pc->U[4][c] - 0.125 * sE, ebar = 0.125 * se;
          if (ebar + delta > 0.0) {
            cons = 1;
            scale = delta / ebar;
          } else {
            nfall += 1;
          }
        }
        for (int cc8 = 0; cc8 < 8; ++cc8) {
          for (int q = 0; q < 4; ++q) Pf->U[q][xf[cc8]] = uf[cc8][q];
          double e = cons ? ef[cc8] + ef[cc8] * scale : ef[cc8];
          Pf->U[4][xf[cc8]] = (e + kef[cc8]) + mef[cc8];
        }
      }
  return nfall;
}

/* Restriction of fine patch Pf onto coarse patch Pc for the coarse cells of
 * box [clo, chi] (the coarsened fine interior clipped to Pc's interior grown
 * by one cell): every box cell inside Pc's interior = 0.125 * (sum of its 8
 * fine cells, x fastest); every face of a box cell that is a face of Pc's
 * interior (normal index in [lo, hi+1], others in [lo, hi]) = 0.25 * (sum of
 * its 4 fine sub-faces, lower transverse axis fastest).  Pass 0 writes the
 * cells and the lower faces, pass 1 the upper faces of the box's top layer,
 * so a coarse face shared by two coarse patches, or by two fine patches,
 * receives the same value everywhere. */
static int own_face_c(const orc_patch *P, const int *ai, int a) {
  for (int e = 0; e < 3; ++e) {
    int top = (e == a) ? P->g + P->n[e] : P->g + P->n[e] - 1;
    if (ai[e] < P->g || ai[e] > top) return 0;
  }
  return 1;
}

ORC_EXPORT void orc_restrict(const orc_patch *Pf, const int32_t *fglo, const orc_patch *Pc,
                             const int32_t *cglo, const int32_t *clo, const int32_t *chi,
                             int32_t pass) {
  const int gc = Pc->g, gf = Pf->g;
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int C3[3] = {I, J, K};
        int ca0[3] = {gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc)};
        int inside = 1;
        for (int e = 0; e < 3; ++e)
          if (ca0[e] < gc || ca0[e] > gc + Pc->n[e] - 1) inside = 0;
        int64_t c = ix(Pc, ca0[0], ca0[1], ca0[2]);
        for (int q = 0; q < 5 && pass == 0 && inside; ++q) {
          double s = 0.0;
          int first = 1;
          for (int fc = 0; fc < 2; ++fc)
            for (int fb = 0; fb < 2; ++fb)
              for (int fa = 0; fa < 2; ++fa) {
                double v = Pf->U[q][ix(Pf, gidx(2 * I + fa, fglo[0], gf), gidx(2 * J + fb, fglo[1], gf),
                                        gidx(2 * K + fc, fglo[2], gf))];
                s = first ? v : s + v;
                first = 0;
              }
          Pc->U[q][c] = 0.125 * s;
        }
        for (int a = 0; a < 3; ++a) {
          int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
          int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
          for (int up = 0; up < 2; ++up) {
            if (up != pass) continue;
            if (up && C3[a] != chi[a]) continue;
            int cf[3] = {ca0[0], ca0[1], ca0[2]};
            cf[a] += up;
            if (!own_face_c(Pc, cf, a)) continue;
            double s = 0.0;
            int first = 1;
            for (int j2 = 0; j2 < 2; ++j2)
              for (int j1 = 0; j1 < 2; ++j1) {
                int f[3];
                f[a] = 2 * (C3[a] + up);
                f[lo_t] = 2 * C3[lo_t] + j1;
                f[hi_t] = 2 * C3[hi_t] + j2;
                double v = Pf->B[a][ix(Pf, gidx(f[0], fglo[0], gf), gidx(f[1], fglo[1], gf), gidx(f[2], fglo[2], gf))];
                s = first ? v : s + v;
                first = 0;
              }
            int ca[3] = {gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc)};
            ca[a] += up;
            Pc->B[a][ix(Pc, ca[0], ca[1], ca[2])] = 0.25 * s;
          }
        }
      }
}

/* Flux-register deposit of coarse faces: for each axis-d face of the coarse
 * box [clo, chi] (face index = index of its upper cell), the correction
 * dF_q = 0.25 * (sum of the 4 fine sub-face registers, lower transverse axis
 * fastest) - (coarse register), written into the correction planes corr[d*5+q]
 * (laid out with the coarse patch's strides).  fine: 5 planes over the fine
 * box [flo, fhi] (x fastest); coarse: 5 planes over [clo, chi]. */
ORC_EXPORT void orc_deposit_faces(const orc_patch *Pc, const int32_t *cglo, double *const *corr,
                                  int32_t d, const int32_t *clo, const int32_t *chi,
                                  const double *fine, const int32_t *flo, const int32_t *fhi,
                                  const double *coarse) {
  const int gc = Pc->g;
  int fe[3], ce[3];
  for (int e = 0; e < 3; ++e) { fe[e] = fhi[e] - flo[e] + 1; ce[e] = chi[e] - clo[e] + 1; }
  int64_t fn = (int64_t)fe[0] * fe[1] * fe[2], cn = (int64_t)ce[0] * ce[1] * ce[2];
  int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  int lo_t = t1 < t2 ? t1 : t2, hi_t = t1 < t2 ? t2 : t1;
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int C3[3] = {I, J, K};
        int64_t co = (int64_t)(I - clo[0]) + (int64_t)ce[0] * ((J - clo[1]) + (int64_t)ce[1] * (K - clo[2]));
        int64_t c = ix(Pc, gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc));
        for (int q = 0; q < 5; ++q) {
          double s = 0.0;
          int first = 1;
          for (int j2 = 0; j2 < 2; ++j2)
            for (int j1 = 0; j1 < 2; ++j1) {
              int f[3];
              f[d] = 2 * C3[d];
              f[lo_t] = 2 * C3[lo_t] + j1;
              f[hi_t] = 2 * C3[hi_t] + j2;
              int64_t fo = (int64_t)(f[0] - flo[0]) + (int64_t)fe[0] * ((f[1] - flo[1]) + (int64_t)fe[1] * (f[2] - flo[2]));
              double v = fine[q * fn + fo];
              s = first ? v : s + v;
              first = 0;
            }
          corr[d * 5 + q][c] = 0.25 * s - coarse[q * cn + co];
        }
      }
}

/* EMF deposit of coarse axis-a edges of box [clo, chi] (an edge is stored at
 * the cell whose lower corner lines it lies on): dE = 0.5 * (sum of the two
 * fine segments) - (coarse register), into corr[15 + a]. */
ORC_EXPORT void orc_deposit_edges(const orc_patch *Pc, const int32_t *cglo, double *const *corr,
                                  int32_t a, const int32_t *clo, const int32_t *chi,
                                  const double *fine, const int32_t *flo, const int32_t *fhi,
                                  const double *coarse) {
  const int gc = Pc->g;
  int fe[3], ce[3];
  for (int e = 0; e < 3; ++e) { fe[e] = fhi[e] - flo[e] + 1; ce[e] = chi[e] - clo[e] + 1; }
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int C3[3] = {I, J, K};
        int64_t co = (int64_t)(I - clo[0]) + (int64_t)ce[0] * ((J - clo[1]) + (int64_t)ce[1] * (K - clo[2]));
        int64_t c = ix(Pc, gidx(I, cglo[0], gc), gidx(J, cglo[1], gc), gidx(K, cglo[2], gc));
        double s = 0.0;
        for (int seg = 0; seg < 2; ++seg) {
          int f[3] = {2 * C3[0], 2 * C3[1], 2 * C3[2]};
          f[a] += seg;
          int64_t fo = (int64_t)(f[0] - flo[0]) + (int64_t)fe[0] * ((f[1] - flo[1]) + (int64_t)fe[1] * (f[2] - flo[2]));
          s = seg ? s + fine[fo] : fine[fo];
        }
        corr[15 + a][c] = 0.5 * s - coarse[co];
      }
}

/* Synchronisation of fluxes on faces shared by two patches of one level
 * (Sec. 2.2 S step; R14): each of the two patches registered dt * F on the
 * shared faces of box [clo, chi] (its level's global index, x fastest, 5
 * planes) during its advance.  When the two registers differ (the patches
 * computed the face from different data), both are corrected to their mean:
 * the patch with register `own` gets dF_q = 0.5 * (other - own) in corr[5 d
 * + q] at those faces, so that orc_correct leaves its cells as if it had
 * used the mean flux.  Called once for each of the two patches (own and
 * other swapped); where the registers agree the correction is exactly 0. */
ORC_EXPORT void orc_sync_faces(const orc_patch *P, const int32_t *glo, double *const *corr, int32_t d,
                               const int32_t *clo, const int32_t *chi, const double *other,
                               const double *own) {
  const int g = P->g;
  int ce[3];
  for (int e = 0; e < 3; ++e) ce[e] = chi[e] - clo[e] + 1;
  int64_t cn = (int64_t)ce[0] * ce[1] * ce[2];
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int64_t o = (int64_t)(I - clo[0]) + (int64_t)ce[0] * ((J - clo[1]) + (int64_t)ce[1] * (K - clo[2]));
        int64_t c = ix(P, gidx(I, glo[0], g), gidx(J, glo[1], g), gidx(K, glo[2], g));
        for (int q = 0; q < 5; ++q) corr[d * 5 + q][c] = 0.5 * (other[q * cn + o] - own[q * cn + o]);
      }
}

/* The same for the EMFs dt * E_a registered on shared axis-a edges of box
 * [clo, chi]: dE = 0.5 * (other - own) into corr[15 + a]. */
ORC_EXPORT void orc_sync_edges(const orc_patch *P, const int32_t *glo, double *const *corr, int32_t a,
                               const int32_t *clo, const int32_t *chi, const double *other,
                               const double *own) {
  const int g = P->g;
  int ce[3];
  for (int e = 0; e < 3; ++e) ce[e] = chi[e] - clo[e] + 1;
  for (int K = clo[2]; K <= chi[2]; ++K)
    for (int J = clo[1]; J <= chi[1]; ++J)
      for (int I = clo[0]; I <= chi[0]; ++I) {
        int64_t o = (int64_t)(I - clo[0]) + (int64_t)ce[0] * ((J - clo[1]) + (int64_t)ce[1] * (K - clo[2]));
        int64_t c = ix(P, gidx(I, glo[0], g), gidx(J, glo[1], g), gidx(K, glo[2], g));
        corr[15 + a][c] = 0.5 * (other[o] - own[o]);
      }
}

/* Applies the correction planes to every interior cell and every interior
 * face of coarse patch P:
 *   U_q -= (dF_x(+x) - dF_x)/dx - ... (x, y, z in order),
 *   B_a -= ((dE_c(+b) - dE_c)/dx_b - (dE_b(+c) - dE_b)/dx_c)
 * (planes are zero away from coarse-fine boundaries). */
ORC_EXPORT void orc_correct(const orc_patch *P, double *const *corr) {
  const int g = P->g;
  const int64_t *s = P->s;
  for (int k = g; k < g + P->n[2]; ++k)
    for (int j = g; j < g + P->n[1]; ++j)
      for (int i = g; i < g + P->n[0]; ++i) {
        int64_t c = ix(P, i, j, k);
        for (int q = 0; q < 5; ++q) {
          double u = P->U[q][c];
          u = u - (corr[0 * 5 + q][c + s[0]] - corr[0 * 5 + q][c]) / P->dx[0]
                - (corr[1 * 5 + q][c + s[1]] - corr[1 * 5 + q][c]) / P->dx[1]
                - (corr[2 * 5 + q][c + s[2]] - corr[2 * 5 + q][c]) / P->dx[2];
          P->U[q][c] = u;
        }
      }
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    int hi[3] = {g + P->n[0] - 1, g + P->n[1] - 1, g + P->n[2] - 1};
    hi[a] += 1;
    for (int k = g; k <= hi[2]; ++k)
      for (int j = g; j <= hi[1]; ++j)
        for (int i = g; i <= hi[0]; ++i) {
          int64_t c = ix(P, i, j, k);
          double dEc = corr[15 + cc][c + s[b]] - corr[15 + cc][c];
          double dEb = corr[15 + b][c + s[cc]] - corr[15 + b][c];
          P->B[a][c] = P->B[a][c] - (dEc / P->dx[b] - dEb / P->dx[cc]);
        }
  }
}

/* Ghost copy (Sec. 2.2 "update ghost cells"), two passes over all copies of
 * a fill.  Box [lo, hi] (destination global index) is a source interior
 * image clipped to the destination's ghost-extended box grown by one cell:
 * the box cells inside the destination's arrays take the values of Ps at
 * global index + off, and so does every face of a box cell that exists in
 * the destination's face arrays (the extra cell layer supplies the faces on
 * the array's outer planes): pass 0 writes cells and lower faces, pass 1 the
 * upper faces of the box's top layer along each axis.  No pass writes a face
 * of Pd's interior (normal index in [g, g+n], others in [g, g+n-1]).
 * Within one pass the copies of a fill write disjoint elements; a face that
 * is the top face of one box and the bottom face of another gets the pass-1
 * value (both sources hold the same face). */
static int dst_own_face(const orc_patch *Pd, const int *di, int a) {
  for (int e = 0; e < 3; ++e) {
    int top = (e == a) ? Pd->g + Pd->n[e] : Pd->g + Pd->n[e] - 1;
    if (di[e] < Pd->g || di[e] > top) return 0;
  }
  return 1;
}

/* does the axis-a face with array index di exist in P's face arrays? */
static int face_exists(const orc_patch *P, const int *di, int a) {
  for (int e = 0; e < 3; ++e) {
    int N = P->n[e] + 2 * P->g;
    int top = (e == a) ? N : N - 1;
    if (di[e] < 0 || di[e] > top) return 0;
  }
  return 1;
}

ORC_EXPORT void orc_copy(const orc_patch *Ps, const int32_t *sglo, const orc_patch *Pd,
                         const int32_t *dglo, const int32_t *lo, const int32_t *hi,
                         const int32_t *off, int32_t pass) {
  const int gs = Ps->g, gd = Pd->g;
  int Nd[3];
  for (int d = 0; d < 3; ++d) Nd[d] = Pd->n[d] + 2 * gd;
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int gl[3] = {i, j, k};
        int di[3] = {gidx(i, dglo[0], gd), gidx(j, dglo[1], gd), gidx(k, dglo[2], gd)};
        int si[3] = {gidx(i + off[0], sglo[0], gs), gidx(j + off[1], sglo[1], gs), gidx(k + off[2], sglo[2], gs)};
        int64_t xd = ix(Pd, di[0], di[1], di[2]), xs = ix(Ps, si[0], si[1], si[2]);
        int cell_in = 1;
        for (int e = 0; e < 3; ++e)
          if (di[e] < 0 || di[e] > Nd[e] - 1) cell_in = 0;
        if (pass == 0) {
          if (cell_in)
            for (int q = 0; q < 5; ++q) Pd->U[q][xd] = Ps->U[q][xs];
          for (int a = 0; a < 3; ++a)
            if (face_exists(Pd, di, a) && !dst_own_face(Pd, di, a)) Pd->B[a][xd] = Ps->B[a][xs];
        } else {
          for (int a = 0; a < 3; ++a) {
            if (gl[a] != hi[a]) continue;
            int du[3] = {di[0], di[1], di[2]};
            du[a] += 1;
            if (!face_exists(Pd, du, a) || dst_own_face(Pd, du, a)) continue;
            Pd->B[a][xd + Pd->s[a]] = Ps->B[a][xs + Ps->s[a]];
          }
        }
      }
}
