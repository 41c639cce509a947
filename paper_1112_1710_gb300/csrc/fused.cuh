// fused.cuh -- the whole patch advance (A of the paper's Sec. 2.2 life cycle)
// as one persistent kernel over a work queue, with every intermediate in
// shared memory.  Included by advance.cuh inside its per-build namespace.
//
// A work item is an x-y tile of BX x BY cells of a patch's update box UB and a
// chunk [z0, z1) of its planes.  The tile marches along z; for the front plane
// zf each iteration runs five phases separated by block barriers:
//   A  primitives W and cell E^n = -v x Bc on plane zf        (tile + 2 halo)
//   B  slopes, Hancock predictor, predicted face states and the reference
//      cell EMF on plane zf-1 (tile + 1 halo); edge averages of E^n at
//      z-index zf (x- and y-edges) and on plane zf-1 (z-edges)
//   C  CT half step of the face-normal field and HLLD on the x- and y-faces of
//      plane zf-1 and on the z-faces at z-index zf-1
//   D  edge EMFs at z-index zf-1 (x-, y-edges) and on plane zf-1 (z-edges)
//   E  conservative and CT update of plane zf-2 (and its lower z-faces)
// so the pipeline is two planes deep, and ring buffers of two (three for W)
// planes carry what the next iteration still needs.  Every element is
// computed with the expressions of the staged kernels in the same order, so
// the FP64 parity build of this kernel gives the staged (and the oracle's)
// bits.  Tiles overlap by their halos and recompute them; the stored state is
// read from the patch arrays and the new state written to an output copy,
// because neighbouring tiles still read old values (k_commit copies it back).
#pragma once

template <int BX, int BY> struct FusedLayout {
  static constexpr int P2 = BX + 4, Q2 = BY + 4;  // tile + 2 halo (cells)
  static constexpr int P1 = BX + 2, Q1 = BY + 2;  // tile + 1 halo (cells, faces)
  static constexpr int PE = BX + 3, QE = BY + 3;  // edge averages
  static constexpr int PT = BX + 1, QT = BY + 1;  // edge EMFs of the update
  static constexpr int G2 = P2 * Q2, G1 = P1 * Q1, GE = PE * QE, GT = PT * QT;
  // offsets in elements
  static constexpr int W = 0;                  // [3 slots][8][G2]
  static constexpr int EN = W + 3 * 8 * G2;    // [2][3][G2]
  static constexpr int WFXY = EN + 2 * 3 * G2;  // [32][G1]: (d*2+side)*8+q, d = 0, 1
  static constexpr int WFZB = WFXY + 32 * G1;   // [8][G1]: z, lower side
  static constexpr int WFZT = WFZB + 8 * G1;    // [2][8][G1]: z, upper side
  static constexpr int ER = WFZT + 2 * 8 * G1;  // [2][3][G1]
  static constexpr int EEXY = ER + 2 * 3 * G1;  // [2][2][GE]
  static constexpr int EEZ = EEXY + 2 * 2 * GE;  // [GE]
  static constexpr int FXY = EEZ + GE;           // [2][2][8][G1]
  static constexpr int FZ = FXY + 2 * 2 * 8 * G1;  // [2][8][G1]
  static constexpr int EDXY = FZ + 2 * 8 * G1;   // [2][2][GT]
  static constexpr int EDZ = EDXY + 2 * 2 * GT;  // [2][GT]
  static constexpr int TOTAL = EDZ + 2 * GT;
};

__device__ __forceinline__ int slot2(int z) { return z & 1; }
__device__ __forceinline__ int slot3(int z) { return z % 3; }

// Phase A: primitives and cell E^n on plane z over the tile + 2 halo.
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_prim(const DPatch& p, R* sm, int X0, int Y0, int TX, int TY, int z,
                                           const SolverConsts<R>& sc, int* status) {
  using L = FusedLayout<BX, BY>;
  R* W = sm + L::W + slot3(z) * 8 * L::G2;
  R* En = sm + L::EN + slot2(z) * 3 * L::G2;
  const int w2 = TX + 4, n = w2 * (TY + 4);
  bool bad = false;
  for (int r = threadIdx.x; r < n; r += NT) {
    int lx;
    const int ly = divmod24(r, w2, lx);
    const int64_t x = (int64_t)(X0 - 2 + lx) + (int64_t)(Y0 - 2 + ly) * p.s1 + (int64_t)z * p.s2;
    R u[8];
#pragma unroll
    for (int q = 0; q < 5; ++q) u[q] = ((const R*)p.U[q])[x];
    u[5] = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
    u[6] = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + p.s1]);
    u[7] = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + p.s2]);
    R w[8];
    cons2prim(u, sc.gm1, w);
    if (sc.rho_floor > R(0) && !(w[0] >= sc.rho_floor)) w[0] = sc.rho_floor;
    if (sc.p_floor > R(0) && !(w[4] >= sc.p_floor)) w[4] = sc.p_floor;
    const int s = ly * L::P2 + lx;
#pragma unroll
    for (int q = 0; q < 8; ++q) W[q * L::G2 + s] = w[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, cc = (a + 2) % 3;
      En[a * L::G2 + s] = w[1 + cc] * w[5 + b] - w[1 + b] * w[5 + cc];
    }
    if (!(w[0] > R(0)) || !(w[4] > R(0))) bad = true;
  }
  if (bad) raise_status(status, -4);
}

// Phase B (1): slopes, Hancock predictor and predicted face states of plane z.
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_pred(R* sm, int TX, int TY, int z, const SolverConsts<R>& sc,
                                           const StepDt<R>& st) {
  using L = FusedLayout<BX, BY>;
  const R* Wm = sm + L::W + slot3(z - 1) * 8 * L::G2;
  const R* W0 = sm + L::W + slot3(z) * 8 * L::G2;
  const R* Wp = sm + L::W + slot3(z + 1) * 8 * L::G2;
  R* WFXY = sm + L::WFXY;
  R* WFZB = sm + L::WFZB;
  R* WFZT = sm + L::WFZT + slot2(z) * 8 * L::G1;
  R* ER = sm + L::ER + slot2(z) * 3 * L::G1;
  const int w1 = TX + 2, n = w1 * (TY + 2);
  for (int r = threadIdx.x; r < n; r += NT) {
    int hx;
    const int hy = divmod24(r, w1, hx);
    const int s2 = (hy + 1) * L::P2 + hx + 1;  // the cell in the 2-halo grid
    const int s1 = hy * L::P1 + hx;
    R w[8], dw[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = W0[q * L::G2 + s2];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      {
        R a = w[q] - W0[q * L::G2 + s2 - 1];
        R b = W0[q * L::G2 + s2 + 1] - w[q];
        dw[0][q] = limiter(sc.limiter, a, b);
      }
      {
        R a = w[q] - W0[q * L::G2 + s2 - L::P2];
        R b = W0[q * L::G2 + s2 + L::P2] - w[q];
        dw[1][q] = limiter(sc.limiter, a, b);
      }
      {
        R a = w[q] - Wm[q * L::G2 + s2];
        R b = Wp[q * L::G2 + s2] - w[q];
        dw[2][q] = limiter(sc.limiter, a, b);
      }
    }
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R rm = w[0] - R(0.5) * dw[d][0], rp = w[0] + R(0.5) * dw[d][0];
      R pm = w[4] - R(0.5) * dw[d][4], pp = w[4] + R(0.5) * dw[d][4];
      if (!(rm > R(0)) || !(rp > R(0)) || !(pm > R(0)) || !(pp > R(0))) bad = true;
    }
    R du[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) du[q] = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R fwm[8], fwp[8], fm[8], fp[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        fwm[q] = bad ? w[q] : w[q] - R(0.5) * dw[d][q];
        fwp[q] = bad ? w[q] : w[q] + R(0.5) * dw[d][q];
      }
      flux_xyz(d, fwp, sc.igm1, fp);
      flux_xyz(d, fwm, sc.igm1, fm);
#pragma unroll
      for (int q = 0; q < 8; ++q) du[q] = du[q] - st.hdtdx[d] * (fp[q] - fm[q]);
    }
    // predicted face states, stored as computed; the second positivity rule
    // replaces all six by W (and du by 0) if any is non-positive
    bool bad2 = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        R fw[8], u[8], pw[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          fw[q] = bad ? w[q] : (sd ? w[q] + R(0.5) * dw[d][q] : w[q] - R(0.5) * dw[d][q]);
        prim2cons(fw, sc.igm1, u);
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = u[q] + du[q];
        cons2prim(u, sc.gm1, pw);
        if (!(pw[0] > R(0)) || !(pw[4] > R(0))) bad2 = true;
        R* dst = d < 2 ? WFXY + (d * 2 + sd) * 8 * L::G1 : (sd ? WFZT : WFZB);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q * L::G1 + s1] = pw[q];
      }
    }
    if (bad2) {
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        R* dst = f < 4 ? WFXY + f * 8 * L::G1 : (f == 5 ? WFZT : WFZB);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q * L::G1 + s1] = w[q];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) du[q] = R(0);
    }
    R uc[8], uh[8];
    prim2cons(w, sc.igm1, uc);
#pragma unroll
    for (int q = 0; q < 8; ++q) uh[q] = uc[q] + du[q];
    R ir = R(1) / uh[0];
    R v[3] = {uh[1] * ir, uh[2] * ir, uh[3] * ir};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, cc = (a + 2) % 3;
      ER[a * L::G1 + s1] = v[cc] * uh[5 + b] - v[b] * uh[5 + cc];
    }
  }
}

// Phase B (2): edge averages of E^n.  x- and y-edges at z-index ze (from the
// cell planes ze-1 and ze), z-edges on plane zz (when zz >= 0).
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_edges(R* sm, int TX, int TY, int ze, bool do_xy, int zz, bool do_z) {
  using L = FusedLayout<BX, BY>;
  const int we = TX + 3, n = we * (TY + 3);
  const R* Em = sm + L::EN + slot2(ze - 1) * 3 * L::G2;
  const R* E0 = sm + L::EN + slot2(ze) * 3 * L::G2;
  const R* Ez = sm + L::EN + slot2(zz) * 3 * L::G2 + 2 * L::G2;
  R* EXY = sm + L::EEXY + slot2(ze) * 2 * L::GE;
  R* EZ = sm + L::EEZ;
  for (int r = threadIdx.x; r < n; r += NT) {
    int ex;
    const int ey = divmod24(r, we, ex);
    const int s = (ey + 1) * L::P2 + ex + 1;  // cell (i, j) of the edge in the 2-halo grid
    const int se = ey * L::PE + ex;
    if (do_xy) {
      {  // x-edge: cells (j-1, k-1), (j, k-1), (j-1, k), (j, k)
        R e00 = Em[0 * L::G2 + s - L::P2];
        R e10 = Em[0 * L::G2 + s];
        R e01 = E0[0 * L::G2 + s - L::P2];
        R e11 = E0[0 * L::G2 + s];
        EXY[0 * L::GE + se] = R(0.25) * (e00 + e10 + e01 + e11);
      }
      {  // y-edge: cells (i-1, k-1), (i-1, k), (i, k-1), (i, k)
        R e00 = Em[1 * L::G2 + s - 1];
        R e10 = E0[1 * L::G2 + s - 1];
        R e01 = Em[1 * L::G2 + s];
        R e11 = E0[1 * L::G2 + s];
        EXY[1 * L::GE + se] = R(0.25) * (e00 + e10 + e01 + e11);
      }
    }
    if (do_z) {  // z-edge: cells (i-1, j-1), (i, j-1), (i-1, j), (i, j)
      R e00 = Ez[s - L::P2 - 1];
      R e10 = Ez[s - L::P2];
      R e01 = Ez[s - 1];
      R e11 = Ez[s];
      EZ[se] = R(0.25) * (e00 + e10 + e01 + e11);
    }
  }
}

// HLLD flux of one face from its two predicted states, rotated to and from
// the face-normal frame; slot 5+d of the result carries the contact side.
template <typename R, int d>
__device__ __forceinline__ void face_flux(const R* wl, const R* wr, R bh, const SolverConsts<R>& sc, R* f) {
  R L[8], Rr[8], fr[8], upw;
  rot_in(d, wl, L);
  rot_in(d, wr, Rr);
  hlld<R, kFastRecip>(L, Rr, bh, sc.gamma, sc.igm1, sc.eps_up, fr, &upw);
  rot_out(d, fr, f);
  f[5 + d] = upw;
}

// Phase C: fluxes of plane zc (x-, y-faces) and of the z-faces at z-index zc.
// With fst set (patches whose fluxes feed flux registers) the hydrodynamic
// flux components of the faces this item owns are also stored in the staged
// scratch layout, where the capture kernel reads them.
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_flux(const DPatch& p, R* sm, int X0, int Y0, int TX, int TY, int zc,
                                           bool do_xy, bool do_z, const SolverConsts<R>& sc,
                                           const StepDt<R>& st, R* fst, bool own_z, bool own_ztop, bool xlast,
                                           bool ylast) {
  using L = FusedLayout<BX, BY>;
  const R* WFXY = sm + L::WFXY;
  const R* WFZB = sm + L::WFZB;
  const R* WFZT = sm + L::WFZT + slot2(zc - 1) * 8 * L::G1;
  const R* EX0 = sm + L::EEXY + slot2(zc) * 2 * L::GE;      // x-edges at z-index zc
  const R* EY0 = EX0 + L::GE;                                // y-edges at z-index zc
  const R* EX1 = sm + L::EEXY + slot2(zc + 1) * 2 * L::GE;  // z-index zc+1
  const R* EY1 = EX1 + L::GE;
  const R* EZ = sm + L::EEZ;
  R* FX = sm + L::FXY + slot2(zc) * 16 * L::G1;
  R* FY = FX + 8 * L::G1;
  R* FZ = sm + L::FZ + slot2(zc) * 8 * L::G1;
  const int w1 = TX + 2, n1 = w1 * (TY + 2);
  const int nx = do_xy ? n1 : 0, ny = do_xy ? n1 : 0, nz = do_z ? n1 : 0;
  const int ntot = nx + ny + nz;
  for (int r = threadIdx.x; r < ntot; r += NT) {
    int dir = 0, e = r;
    if (e >= nx) {
      e -= nx;
      dir = 1;
      if (e >= ny) {
        e -= ny;
        dir = 2;
      }
    }
    int hx;
    const int hy = divmod24(e, w1, hx);
    const int s1 = hy * L::P1 + hx;
    const int se = hy * L::PE + hx;
    const int64_t x = (int64_t)(X0 - 1 + hx) + (int64_t)(Y0 - 1 + hy) * p.s1 + (int64_t)zc * p.s2;
    R wl[8], wr[8], f[8];
    if (dir == 0) {  // x-face at (i, j): cells i-1 | i
      if (hx == 0) continue;
      R dEc = EZ[se + L::PE] - EZ[se];
      R dEb = EY1[se] - EY0[se];
      R bh = ((const R*)p.B[0])[x] - (st.hdtdx[1] * dEc - st.hdtdx[2] * dEb);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        wl[q] = WFXY[(1 * 8 + q) * L::G1 + s1 - 1];
        wr[q] = WFXY[(0 * 8 + q) * L::G1 + s1];
      }
      face_flux<R, 0>(wl, wr, bh, sc, f);
#pragma unroll
      for (int q = 0; q < 8; ++q) FX[q * L::G1 + s1] = f[q];
      if (fst && own_z && hy >= 1 && hy <= TY && (hx <= TX || xlast)) {
#pragma unroll
        for (int q = 0; q < 5; ++q) *vgroup_at(fst + (int64_t)(SC_F + 0 * 8) * p.snelem, p.snelem, x, q) = f[q];
      }
    } else if (dir == 1) {  // y-face: cells j-1 | j
      if (hy == 0) continue;
      R dEc = EX1[se] - EX0[se];
      R dEb = EZ[se + 1] - EZ[se];
      R bh = ((const R*)p.B[1])[x] - (st.hdtdx[2] * dEc - st.hdtdx[0] * dEb);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        wl[q] = WFXY[(3 * 8 + q) * L::G1 + s1 - L::P1];
        wr[q] = WFXY[(2 * 8 + q) * L::G1 + s1];
      }
      face_flux<R, 1>(wl, wr, bh, sc, f);
#pragma unroll
      for (int q = 0; q < 8; ++q) FY[q * L::G1 + s1] = f[q];
      if (fst && own_z && hx >= 1 && hx <= TX && (hy <= TY || ylast)) {
#pragma unroll
        for (int q = 0; q < 5; ++q) *vgroup_at(fst + (int64_t)(SC_F + 1 * 8) * p.snelem, p.snelem, x, q) = f[q];
      }
    } else {  // z-face at z-index zc: cells zc-1 | zc
      R dEc = EY0[se + 1] - EY0[se];
      R dEb = EX0[se + L::PE] - EX0[se];
      R bh = ((const R*)p.B[2])[x] - (st.hdtdx[0] * dEc - st.hdtdx[1] * dEb);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        wl[q] = WFZT[q * L::G1 + s1];
        wr[q] = WFZB[q * L::G1 + s1];
      }
      face_flux<R, 2>(wl, wr, bh, sc, f);
#pragma unroll
      for (int q = 0; q < 8; ++q) FZ[q * L::G1 + s1] = f[q];
      if (fst && (own_z || own_ztop) && hx >= 1 && hx <= TX && hy >= 1 && hy <= TY) {
#pragma unroll
        for (int q = 0; q < 5; ++q) *vgroup_at(fst + (int64_t)(SC_F + 2 * 8) * p.snelem, p.snelem, x, q) = f[q];
      }
    }
  }
}

// Phase D: edge EMFs at z-index ze (x-, y-edges) and on plane ze (z-edges).
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_emf(const DPatch& p, R* sm, int X0, int Y0, int TX, int TY, int ze,
                                          bool do_xy, bool do_z, const SolverConsts<R>& sc, R* fst,
                                          bool own_xy, bool xlast, bool ylast) {
  using L = FusedLayout<BX, BY>;
  const R* FXm = sm + L::FXY + slot2(ze - 1) * 16 * L::G1;  // plane ze-1
  const R* FYm = FXm + 8 * L::G1;
  const R* FX0 = sm + L::FXY + slot2(ze) * 16 * L::G1;  // plane ze
  const R* FY0 = FX0 + 8 * L::G1;
  const R* FZ0 = sm + L::FZ + slot2(ze) * 8 * L::G1;  // z-faces at z-index ze
  const R* ERm = sm + L::ER + slot2(ze - 1) * 3 * L::G1;
  const R* ER0 = sm + L::ER + slot2(ze) * 3 * L::G1;
  R* EDXY = sm + L::EDXY + slot2(ze) * 2 * L::GT;
  R* EDZ = sm + L::EDZ + slot2(ze) * L::GT;
  const int wt = TX + 1, n = wt * (TY + 1);
  for (int r = threadIdx.x; r < n; r += NT) {
    int tx;
    const int ty = divmod24(r, wt, tx);
    const int s = (ty + 1) * L::P1 + tx + 1;  // cell (i, j) in the 1-halo grid
    const int st_ = ty * L::PT + tx;
    const int64_t x = (int64_t)(X0 + tx) + (int64_t)(Y0 + ty) * p.s1 + (int64_t)ze * p.s2;
    const bool ox = tx < TX || xlast, oy = ty < TY || ylast;
    if (do_xy && tx < TX) {  // x-edge (a = 0; b = y, c = z)
      R v = edge_emf_value(-FYm[7 * L::G1 + s], -FY0[7 * L::G1 + s], FZ0[6 * L::G1 + s - L::P1],
                           FZ0[6 * L::G1 + s], ERm[0 * L::G1 + s - L::P1], ERm[0 * L::G1 + s],
                           ER0[0 * L::G1 + s - L::P1], ER0[0 * L::G1 + s], FYm[6 * L::G1 + s],
                           FY0[6 * L::G1 + s], FZ0[7 * L::G1 + s - L::P1], FZ0[7 * L::G1 + s], sc.emf);
      EDXY[0 * L::GT + st_] = v;
      if (fst && own_xy && oy) fst[(int64_t)(SC_ED + 0) * p.snelem + x] = v;
    }
    if (do_xy && ty < TY) {  // y-edge (a = 1; b = z, c = x)
      R v = edge_emf_value(-FZ0[5 * L::G1 + s - 1], -FZ0[5 * L::G1 + s], FXm[7 * L::G1 + s],
                           FX0[7 * L::G1 + s], ERm[1 * L::G1 + s - 1], ER0[1 * L::G1 + s - 1],
                           ERm[1 * L::G1 + s], ER0[1 * L::G1 + s], FZ0[7 * L::G1 + s - 1], FZ0[7 * L::G1 + s],
                           FXm[5 * L::G1 + s], FX0[5 * L::G1 + s], sc.emf);
      EDXY[1 * L::GT + st_] = v;
      if (fst && own_xy && ox) fst[(int64_t)(SC_ED + 1) * p.snelem + x] = v;
    }
    if (do_z) {  // z-edge (a = 2; b = x, c = y)
      R v = edge_emf_value(-FX0[6 * L::G1 + s - L::P1], -FX0[6 * L::G1 + s], FY0[5 * L::G1 + s - 1],
                           FY0[5 * L::G1 + s], ER0[2 * L::G1 + s - L::P1 - 1], ER0[2 * L::G1 + s - L::P1],
                           ER0[2 * L::G1 + s - 1], ER0[2 * L::G1 + s], FX0[5 * L::G1 + s - L::P1],
                           FX0[5 * L::G1 + s], FY0[6 * L::G1 + s - 1], FY0[6 * L::G1 + s], sc.emf);
      EDZ[st_] = v;
      if (fst && ox && oy) fst[(int64_t)(SC_ED + 2) * p.snelem + x] = v;
    }
  }
}

// Phase E: update of the cells and the x-, y-faces of plane zu and of the
// z-faces at z-index zu (and at zu+1 when top is set), into the output copy.
template <typename R, int BX, int BY, int NT>
__device__ __forceinline__ void fused_update(const DPatch& p, R* sm, R* out, int X0, int Y0, int TX, int TY,
                                             int zu, bool cells, bool top, bool xlast, bool ylast,
                                             const StepDt<R>& st) {
  using L = FusedLayout<BX, BY>;
  const R* FX = sm + L::FXY + slot2(zu) * 16 * L::G1;
  const R* FY = FX + 8 * L::G1;
  const R* FZ0 = sm + L::FZ + slot2(zu) * 8 * L::G1;
  const R* FZ1 = sm + L::FZ + slot2(zu + 1) * 8 * L::G1;
  const R* EX0 = sm + L::EDXY + slot2(zu) * 2 * L::GT;  // x-edge EMFs at z-index zu
  const R* EY0 = EX0 + L::GT;
  const R* EX1 = sm + L::EDXY + slot2(zu + 1) * 2 * L::GT;  // z-index zu+1
  const R* EY1 = EX1 + L::GT;
  const R* EZ = sm + L::EDZ + slot2(zu) * L::GT;  // z-edge EMFs on plane zu
  const int wt = TX + 1, n = wt * (TY + 1);
  for (int r = threadIdx.x; r < n; r += NT) {
    int tx;
    const int ty = divmod24(r, wt, tx);
    const bool in_x = tx < TX, in_y = ty < TY;
    const int s1 = (ty + 1) * L::P1 + tx + 1;
    const int st_ = ty * L::PT + tx;
    const int64_t x = (int64_t)(X0 + tx) + (int64_t)(Y0 + ty) * p.s1 + (int64_t)zu * p.s2;
    // all loads first (the output copy may alias the state for the compiler)
    const bool do_c = cells && in_x && in_y, do_x = cells && in_y && (in_x || xlast),
               do_y = cells && in_x && (in_y || ylast), do_z = cells && in_x && in_y, do_t = top && in_x && in_y;
    R un[5], bx = R(0), by = R(0), bz = R(0), bt = R(0);
    if (do_c) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        R u = ((const R*)p.U[q])[x];
        un[q] = u - st.dtdx[0] * (FX[q * L::G1 + s1 + 1] - FX[q * L::G1 + s1]) -
                st.dtdx[1] * (FY[q * L::G1 + s1 + L::P1] - FY[q * L::G1 + s1]) -
                st.dtdx[2] * (FZ1[q * L::G1 + s1] - FZ0[q * L::G1 + s1]);
      }
    }
    if (do_x) {  // x-face (a = 0; b = y, c = z)
      R dEc = EZ[st_ + L::PT] - EZ[st_];
      R dEb = EY1[st_] - EY0[st_];
      bx = ((const R*)p.B[0])[x] - (st.dtdx[1] * dEc - st.dtdx[2] * dEb);
    }
    if (do_y) {  // y-face (a = 1; b = z, c = x)
      R dEc = EX1[st_] - EX0[st_];
      R dEb = EZ[st_ + 1] - EZ[st_];
      by = ((const R*)p.B[1])[x] - (st.dtdx[2] * dEc - st.dtdx[0] * dEb);
    }
    if (do_z) {  // z-face (a = 2; b = x, c = y)
      R dEc = EY0[st_ + 1] - EY0[st_];
      R dEb = EX0[st_ + L::PT] - EX0[st_];
      bz = ((const R*)p.B[2])[x] - (st.dtdx[0] * dEc - st.dtdx[1] * dEb);
    }
    if (do_t) {  // the top z-face of the last chunk
      R dEc = EY1[st_ + 1] - EY1[st_];
      R dEb = EX1[st_ + L::PT] - EX1[st_];
      bt = ((const R*)p.B[2])[x + p.s2] - (st.dtdx[0] * dEc - st.dtdx[1] * dEb);
    }
    if (do_c)
#pragma unroll
      for (int q = 0; q < 5; ++q) out[(int64_t)q * p.snelem + x] = un[q];
    if (do_x) out[5 * p.snelem + x] = bx;
    if (do_y) out[6 * p.snelem + x] = by;
    if (do_z) out[7 * p.snelem + x] = bz;
    if (do_t) out[7 * p.snelem + x + p.s2] = bt;
  }
}

// The persistent kernel: CTAs take (patch, tile, z-chunk) items off a counter
// until the queue is empty.  `out` is the arena; each patch's output copy
// (8 arrays with the patch's strides) starts at its `scr` offset.
template <typename R, int BX, int BY, int NT>
__global__ void __launch_bounds__(NT, 1) k_fused(const DPatch* __restrict__ P, const FusedItem* __restrict__ items,
                                                 int nitems, int* counter, R* arena, const R* __restrict__ K,
                                                 SolverConsts<R> sc, int* status) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  R* sm = (R*)fused_smem;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const FusedItem w = items[it];
    const DPatch& p = P[w.patch];
    const StepDt<R> st(K, w.patch);
    R* out = arena + p.scr;
    const int uhx = p.g + p.n[0] - 1 + p.k, uhy = p.g + p.n[1] - 1 + p.k, uhz = p.g + p.n[2] - 1 + p.k;
    const int X0 = w.x0, Y0 = w.y0, Zs = w.z0, Ze = w.z1;
    const int TX = min(BX, uhx + 1 - X0), TY = min(BY, uhy + 1 - Y0);
    const bool xlast = X0 + TX == uhx + 1, ylast = Y0 + TY == uhy + 1, zlast = Ze == uhz + 1;
    R* fst = (p.flags & 1) ? out : nullptr;
    for (int zf = Zs - 2; zf <= Ze + 1; ++zf) {
      fused_prim<R, BX, BY, NT>(p, sm, X0, Y0, TX, TY, zf, sc, status);
      __syncthreads();
      if (zf >= Zs) fused_pred<R, BX, BY, NT>(sm, TX, TY, zf - 1, sc, st);
      fused_edges<R, BX, BY, NT>(sm, TX, TY, zf, zf >= Zs - 1, zf - 1, zf >= Zs && zf <= Ze + 1);
      __syncthreads();
      if (zf >= Zs)
        fused_flux<R, BX, BY, NT>(p, sm, X0, Y0, TX, TY, zf - 1, true, zf - 1 >= Zs, sc, st, fst,
                                  zf - 1 >= Zs && zf - 1 < Ze, zlast && zf - 1 == Ze, xlast, ylast);
      __syncthreads();
      if (zf - 1 >= Zs)
        fused_emf<R, BX, BY, NT>(p, sm, X0, Y0, TX, TY, zf - 1, true, zf - 1 <= Ze - 1, sc, fst,
                                 zf - 1 < Ze || zlast, xlast, ylast);
      __syncthreads();
      if (zf - 2 >= Zs)
        fused_update<R, BX, BY, NT>(p, sm, out, X0, Y0, TX, TY, zf - 2, true, zlast && zf - 2 == Ze - 1, xlast,
                                    ylast, st);
    }
    __syncthreads();
  }
}

// Copies the new state of the update box (cells and the faces the advance
// writes) from the output copies back into the patch arrays.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_commit(const DPatch* __restrict__ P, const BlockTask* __restrict__ T,
                                                     const R* __restrict__ arena) {
  const BlockTask t = T[blockIdx.x];
  const DPatch& p = P[t.patch];
  const int ex = p.n[0] + 2 * p.k + 1, ey = p.n[1] + 2 * p.k + 1, ez = p.n[2] + 2 * p.k + 1;
  const int e = t.start + threadIdx.x;
  if (e >= ex * ey * ez) return;
  int r0, r1;
  const int q0 = divmod24(e, ex, r0);
  const int q1 = divmod24(q0, ey, r1);
  const int lo = p.g - p.k;
  const int id[3] = {lo + r0, lo + r1, lo + q1};
  const bool inner[3] = {r0 < ex - 1, r1 < ey - 1, q1 < ez - 1};
  const int64_t x = (int64_t)id[0] + (int64_t)id[1] * p.s1 + (int64_t)id[2] * p.s2;
  const R* out = arena + p.scr;
  const bool cell = inner[0] && inner[1] && inner[2];
  R v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool ok = q < 5 ? cell : inner[(q - 4) % 3] && inner[(q - 3) % 3];
    if (ok) v[q] = out[(int64_t)q * p.snelem + x];
  }
  if (cell)
#pragma unroll
    for (int q = 0; q < 5; ++q) ((R*)p.U[q])[x] = v[q];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (inner[(a + 1) % 3] && inner[(a + 2) % 3]) ((R*)p.B[a])[x] = v[5 + a];
}
