// pf.cuh -- the primitive, predictor and Riemann-solver passes of the patch
// advance (A of the paper's Sec. 2.2 life cycle) fused into one kernel, with
// the predicted face states kept on chip; the staged k_update then finishes
// the step from the fluxes this kernel stores.  Included by advance.cuh
// inside its per-build namespace.
//
// A work item is an x-y tile of tx x ty cells (at most TX x TY, the host
// splits each patch's UB+1 region into tiles of near-equal extents) and a
// chunk [z0, z1) of its planes.  A block has one thread per tile cell and one
// per cell of the tile's lower x column and lower y row (the left neighbours
// whose upper face states the tile's lowest faces need); the shared-memory
// arrays are laid out for the largest tile.  Marching along z,
// for each plane zc:
//   1. the primitives W and cell EMFs E^n of plane zc + 1 over the tile grown
//      by two cells below and one above (the stencil of the predictor and of
//      the edge averages) go into rings of three planes in shared memory;
//   2. every thread runs the predictor of its cell on plane zc (limited
//      slopes, Hancock increment, six predicted face states) and leaves the
//      states the tile's faces read in shared memory: the lower x, y and z
//      states of tile cells, the upper x states of the tile and the left
//      column and the upper y states of the tile and the lower row; the
//      tile's upper z states stay in registers until the plane's faces are
//      done and then replace the previous plane's in shared memory;
//   3. the block's threads take the tile's lower x, y and z faces of plane zc
//      (the faces of one axis in runs of whole warps): the CT half-step
//      normal field from edge averages of E^n, the HLLD flux, stored in the
//      staged layout (vector groups) for k_update and the captures.
// The predictor and the Riemann solver thus never hold registers at the same
// time, which keeps the kernel at two to four blocks per SM in FP32 (by tile
// shape).  Each element is
// computed with the staged kernels' expressions in the same order (the FP64
// parity build of this kernel gives the staged, and so the oracle's, bits).
// Tiles overlap only in the predictor of their lower column and row.
#pragma once

template <int TX, int TY> struct PfLayout {
  static constexpr int NC = TX * TY;             // tile cells
  static constexpr int NT = NC + TX + TY;        // threads
  static constexpr int PX = TX + 3, PY = TY + 3; // W / E^n region: x0-2 .. x0+TX
  static constexpr int G = PX * PY;
  static constexpr int NXU = (TX + 1) * TY;      // upper x states: cells x0-1 .. x0+TX-1
  static constexpr int NYU = TX * (TY + 1);      // upper y states: rows y0-1 .. y0+TY-1
  // offsets in elements
  static constexpr int W = 0;                    // [3][8][G]
  static constexpr int EN = W + 3 * 8 * G;       // [3][3][G]
  static constexpr int XU = EN + 3 * 3 * G;      // [7][NXU]
  static constexpr int YU = XU + 7 * NXU;        // [7][NYU]
  static constexpr int LO = YU + 7 * NYU;        // [3][7][NC] lower x, y, z states (tile cell order)
  static constexpr int ZU = LO + 3 * 7 * NC;     // [7][NC] upper z states of the previous plane (same)
  static constexpr int TOTAL = ZU + 7 * NC;
};

// The predictor of one cell from the W ring: the six predicted face states
// in their faces' rotated frames (7 values each), and the Hancock increment
// (zero after the second positivity rule's fallback) for the reference EMF.
template <typename R, int TX, int TY>
__device__ __forceinline__ void pf_predict(const R* __restrict__ sm, int s, int zc, const SolverConsts<R>& sc,
                                           const StepDt<R>& st, R (&fs)[6][7], R (&duk)[8], R (&w)[8]) {
  using L = PfLayout<TX, TY>;
  const R* W0 = sm + L::W + (zc % 3) * 8 * L::G;
  const R* Wm = sm + L::W + ((zc + 2) % 3) * 8 * L::G;
  const R* Wp = sm + L::W + ((zc + 1) % 3) * 8 * L::G;
  R dw[3][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) w[q] = W0[q * L::G + s];
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      R wm, wp;
      if (d == 0) {
        wm = W0[q * L::G + s - 1];
        wp = W0[q * L::G + s + 1];
      } else if (d == 1) {
        wm = W0[q * L::G + s - L::PX];
        wp = W0[q * L::G + s + L::PX];
      } else {
        wm = Wm[q * L::G + s];
        wp = Wp[q * L::G + s];
      }
      dw[d][q] = limiter(sc.limiter, w[q] - wm, wp - w[q]);
    }
    if (face_rule1(w, dw[d])) bad = true;
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
  bool bad2 = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      R fw[8], u[8], pw[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) fw[q] = bad ? w[q] : (sd ? w[q] + R(0.5) * dw[d][q] : w[q] - R(0.5) * dw[d][q]);
      prim2cons(fw, sc.igm1, u);
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = u[q] + du[q];
      cons2prim(u, sc.gm1, pw);
      if (!(pw[0] > R(0)) || !(pw[4] > R(0))) bad2 = true;
      R* o = fs[2 * d + sd];
      o[0] = pw[0]; o[1] = pw[1 + d]; o[2] = pw[1 + t1]; o[3] = pw[1 + t2];
      o[4] = pw[4]; o[5] = pw[5 + t1]; o[6] = pw[5 + t2];
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) duk[q] = du[q];
  if (bad2) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        R* o = fs[2 * d + sd];
        o[0] = w[0]; o[1] = w[1 + d]; o[2] = w[1 + t1]; o[3] = w[1 + t2];
        o[4] = w[4]; o[5] = w[5 + t1]; o[6] = w[5 + t2];
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) duk[q] = R(0);
  }
}

// E^n average at the axis-a edge stored at ring position s of plane z (the
// four cells around it, the staged expression and order).
template <typename R, int TX, int TY, int a>
__device__ __forceinline__ R pf_edge(const R* __restrict__ sm, int s, int z) {
  using L = PfLayout<TX, TY>;
  constexpr int b = (a + 1) % 3, cc = (a + 2) % 3;
  // ring offsets along x, y (in the plane) and the plane for z
  const R* E0 = sm + L::EN + (z % 3) * 3 * L::G + a * L::G;
  const R* Em = sm + L::EN + ((z + 2) % 3) * 3 * L::G + a * L::G;  // plane z - 1
  const int so[3] = {1, L::PX, 0};
  // positions of x - sb - sc, x - sc, x - sb, x (the z axis changes plane)
  R e00, e10, e01, e11;
  if (b != 2 && cc != 2) {
    e00 = E0[s - so[b] - so[cc]];
    e10 = E0[s - so[cc]];
    e01 = E0[s - so[b]];
    e11 = E0[s];
  } else if (b == 2) {  // sb is the z stride
    e00 = Em[s - so[cc]];
    e10 = E0[s - so[cc]];
    e01 = Em[s];
    e11 = E0[s];
  } else {  // cc == 2
    e00 = Em[s - so[b]];
    e10 = Em[s];
    e01 = E0[s - so[b]];
    e11 = E0[s];
  }
  return R(0.25) * (e00 + e10 + e01 + e11);
}

// The flux of the axis-d lower face of tile cell c (position fx, fy on plane
// zc, element x): the CT half-step normal field from edge averages of E^n,
// the left state from the upper states of the cell below along d and the
// right state from the cell's own lower state, then HLLD.
template <typename R, int TX, int TY, int d>
__device__ __forceinline__ void pf_face(const R* __restrict__ sm, const DPatch& p, const StepDt<R>& st,
                                        const SolverConsts<R>& sc, R* scr, int64_t x, int fx, int fy, int zc,
                                        int x0, int y0, int c) {
  using L = PfLayout<TX, TY>;
  constexpr int b = (d + 1) % 3, cc = (d + 2) % 3;
  const int s = (fy - (y0 - 2)) * L::PX + (fx - (x0 - 2));
  R dEc, dEb;
  if (d == 0) {
    dEc = pf_edge<R, TX, TY, 2>(sm, s + L::PX, zc) - pf_edge<R, TX, TY, 2>(sm, s, zc);
    dEb = pf_edge<R, TX, TY, 1>(sm, s, zc + 1) - pf_edge<R, TX, TY, 1>(sm, s, zc);
  } else if (d == 1) {
    dEc = pf_edge<R, TX, TY, 0>(sm, s, zc + 1) - pf_edge<R, TX, TY, 0>(sm, s, zc);
    dEb = pf_edge<R, TX, TY, 2>(sm, s + 1, zc) - pf_edge<R, TX, TY, 2>(sm, s, zc);
  } else {
    dEc = pf_edge<R, TX, TY, 1>(sm, s + 1, zc) - pf_edge<R, TX, TY, 1>(sm, s, zc);
    dEb = pf_edge<R, TX, TY, 0>(sm, s + L::PX, zc) - pf_edge<R, TX, TY, 0>(sm, s, zc);
  }
  const R bh = ((const R*)p.B[d])[x] - (st.hdtdx[b] * dEc - st.hdtdx[cc] * dEb);
  const R* left;
  int lstride;
  if (d == 0) {
    left = sm + L::XU + (fx - x0) + (fy - y0) * (TX + 1);   // cell fx - 1 in XU
    lstride = L::NXU;
  } else if (d == 1) {
    left = sm + L::YU + (fy - y0) * TX + (fx - x0);         // row fy - 1 in YU
    lstride = L::NYU;
  } else {
    left = sm + L::ZU + c;                                  // plane zc - 1
    lstride = L::NC;
  }
  const R* right = sm + L::LO + d * 7 * L::NC + c;
  R Lf[8], Rf[8];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    Lf[q < 5 ? q : q + 1] = left[q * lstride];
    Rf[q < 5 ? q : q + 1] = right[q * L::NC];
  }
  Lf[5] = R(0);
  Rf[5] = R(0);
  R fr[8], f[8], upw;
  hlld<R, kFastRecip>(Lf, Rf, bh, sc.gamma, sc.igm1, sc.eps_up, fr, &upw);
  rot_out(d, fr, f);
  f[5 + d] = upw;
  VecIO<R>::store8(arr(scr, p, SC_F + d * 8), p.snelem, x, f);
}

template <typename R, int TX, int TY, int MINB>
__global__ void __launch_bounds__(PfLayout<TX, TY>::NT, MINB)
    k_pf(const DPatch* __restrict__ P, const FusedItem* __restrict__ items, R* scr, const R* __restrict__ K,
         SolverConsts<R> sc, int* status) {
  using L = PfLayout<TX, TY>;
  extern __shared__ __align__(16) unsigned char pf_smem[];
  R* sm = reinterpret_cast<R*>(pf_smem);
  const FusedItem it = items[blockIdx.x];
  const DPatch& p = P[it.patch];
  const StepDt<R> st(K, it.patch);
  const int x0 = it.x0, y0 = it.y0, z0 = it.z0, z1 = it.z1, tx = it.tx, ty = it.ty;
  const int nc = tx * ty;                   // tile cells
  const int lo = p.g - p.k;                 // update box
  const int hix = p.g + p.n[0] - 1 + p.k, hiy = p.g + p.n[1] - 1 + p.k, hiz = p.g + p.n[2] - 1 + p.k;
  // this thread's predictor cell: tile, lower row (y0 - 1), left column
  // (x0 - 1) or none
  const int t = threadIdx.x;
  int cx = x0 - 2, cy = y0 - 2;
  const bool tile = t < nc;
  if (tile) {
    cx = x0 + t % tx;
    cy = y0 + t / tx;
  } else if (t < nc + tx) {
    cx = x0 + (t - nc);
    cy = y0 - 1;
  } else if (t < nc + tx + ty) {
    cx = x0 - 1;
    cy = y0 + (t - nc - tx);
  }
  // inside UB+1: the predictor is defined there
  const bool act = t < nc + tx + ty && cx >= lo - 1 && cx <= hix + 1 && cy >= lo - 1 && cy <= hiy + 1;
  const int s = (cy - (y0 - 2)) * L::PX + (cx - (x0 - 2));
  const int zstart = z0 - 1 >= lo - 1 ? z0 - 1 : z0;
  const int64_t s1 = p.s1, s2 = p.s2;
  // fills the W / E^n ring slot of plane zl over x0-2 .. x0+tx, y0-2 ..
  // y0+ty, clipped to UB+2
  auto load_plane = [&](int zl) {
    R* W = sm + L::W + (zl % 3) * 8 * L::G;
    R* En = sm + L::EN + (zl % 3) * 3 * L::G;
    bool bad = false;
    const int rx = tx + 3;
    for (int rr = t; rr < rx * (ty + 3); rr += L::NT) {
      const int lx = rr % rx, ly = rr / rx;
      const int r = ly * L::PX + lx;
      const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
      if (gx < lo - 2 || gx > hix + 2 || gy < lo - 2 || gy > hiy + 2 || zl < lo - 2 || zl > hiz + 2) continue;
      const int64_t x = (int64_t)gx + (int64_t)gy * s1 + (int64_t)zl * s2;
      R u[8];
#pragma unroll
      for (int q = 0; q < 5; ++q) u[q] = ((const R*)p.U[q])[x];
      u[5] = R(0.5) * (((const R*)p.B[0])[x] + ((const R*)p.B[0])[x + 1]);
      u[6] = R(0.5) * (((const R*)p.B[1])[x] + ((const R*)p.B[1])[x + s1]);
      u[7] = R(0.5) * (((const R*)p.B[2])[x] + ((const R*)p.B[2])[x + s2]);
      R w[8];
      cons2prim(u, sc.gm1, w);
      if (sc.rho_floor > R(0) && !(w[0] >= sc.rho_floor)) w[0] = sc.rho_floor;
      if (sc.p_floor > R(0) && !(w[4] >= sc.p_floor)) w[4] = sc.p_floor;
#pragma unroll
      for (int q = 0; q < 8; ++q) W[q * L::G + r] = w[q];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, cc = (a + 2) % 3;
        En[a * L::G + r] = w[1 + cc] * w[5 + b] - w[1 + b] * w[5 + cc];
      }
      if (!(w[0] > R(0)) || !(w[4] > R(0))) bad = true;
    }
    if (bad) raise_status(status, -4);
  };
  load_plane(zstart - 1);
  load_plane(zstart);
  R zup[7];                                  // this tile cell's upper z state on plane zc
#pragma unroll
  for (int q = 0; q < 7; ++q) zup[q] = R(0);
  for (int zc = zstart; zc < z1; ++zc) {
    load_plane(zc + 1);
    __syncthreads();
    // 2. predictor of this thread's cell on plane zc
    if (act) {
      R fs[6][7], duk[8], w[8];
      pf_predict<R, TX, TY>(sm, s, zc, sc, st, fs, duk, w);
      if (tile) {
        const int c = t;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int q = 0; q < 7; ++q) sm[L::LO + (d * 7 + q) * L::NC + c] = fs[2 * d][q];
#pragma unroll
        for (int q = 0; q < 7; ++q) zup[q] = fs[5][q];
        if (sc.emf != 1 && zc >= z0) {
          // reference cell EMF from U^{n+1/2}, read by the upwinded EMF average
          const int64_t x = (int64_t)cx + (int64_t)cy * s1 + (int64_t)zc * s2;
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
      }
      // upper x state: tile cells and the left column; upper y state: tile
      // cells and the lower row
      if (cx < x0 + TX && cy >= y0) {
        const int ix = (cy - y0) * (TX + 1) + (cx - (x0 - 1));
#pragma unroll
        for (int q = 0; q < 7; ++q) sm[L::XU + q * L::NXU + ix] = fs[1][q];
      }
      if (cy < y0 + TY && cx >= x0) {
        const int iy = (cy - (y0 - 1)) * TX + (cx - x0);
#pragma unroll
        for (int q = 0; q < 7; ++q) sm[L::YU + q * L::NYU + iy] = fs[3][q];
      }
    }
    __syncthreads();
    // 3. the tile's lower faces on plane zc, axis-major, each axis's run
    // padded to whole warps (warp-uniform axis)
    if (zc >= z0) {
      const int ncp = (nc + 31) & ~31;
      for (int task = t; task < 3 * ncp; task += L::NT) {
        const int d = task / ncp, c = task - d * ncp;
        if (c >= nc) continue;
        const int fx = x0 + c % tx, fy = y0 + c / tx;
        if (fx > hix + 1 || fy > hiy + 1) continue;
        if ((d == 0 ? fx : d == 1 ? fy : zc) < lo) continue;
        if (d == 2 && zc <= zstart) continue;   // no upper z state of plane zc - 1
        const int64_t x = (int64_t)fx + (int64_t)fy * s1 + (int64_t)zc * s2;
        if (d == 0)
          pf_face<R, TX, TY, 0>(sm, p, st, sc, scr, x, fx, fy, zc, x0, y0, c);
        else if (d == 1)
          pf_face<R, TX, TY, 1>(sm, p, st, sc, scr, x, fx, fy, zc, x0, y0, c);
        else
          pf_face<R, TX, TY, 2>(sm, p, st, sc, scr, x, fx, fy, zc, x0, y0, c);
      }
    }
    // the next plane's load and predictor overwrite the ring slot and the
    // states this plane's faces read
    __syncthreads();
    if (tile) {
#pragma unroll
      for (int q = 0; q < 7; ++q) sm[L::ZU + q * L::NC + t] = zup[q];
    }
  }
}
