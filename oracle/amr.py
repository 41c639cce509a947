"""FP64 oracle of the subcycled AMR step (Sec. 2.2 life cycle, Sec. 2.3
extended ghosts), refinement ratio 2, static hierarchy.

TEST INFRASTRUCTURE ONLY (see oracle.py).  The metadata -- ghost copies,
prolongation items, flux-register boxes, deposits -- is generated here by
brute-force box intersection, independently of the product's host code, and
every level operation runs in the C oracle.

One coarse step (the paper's AMR(0)):
  dt_0 = min over levels l of 2^l * (CFL dt of level l)   [Sec. 2.2, dt_l = dt_{l-1}/R]
  fill level-0 ghosts (periodic images, same-level copies)
  step(0, grow 0, dt_0)
step(l, k, dt):
  P: prolong the pre-advance level-l data into the ghost zones of level l+1,
     then same-level copies on level l+1 (ghost cells that lie in a
     neighbour's interior)
  A: advance every level-l patch (update box = interior grown by k),
     capturing dt*F and dt*E on the coarse-fine faces and edges
  if l+1 exists:  step(l+1, 2, dt/2);  S: same-level copies on l+1;
                  step(l+1, 0, dt/2)   (Sec. 2.3: 2 n_ghost then 0 extra layers)
     reflux: correction planes from the flux registers, applied to level l
     R: restrict level l+1 onto the covered level-l cells and faces
The fine patches capture dt_f*F / dt_f*E on their own boundary in both
substeps (set, then add).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def isect(a, b):
    lo = tuple(max(a[0][d], b[0][d]) for d in range(3))
    hi = tuple(min(a[1][d], b[1][d]) for d in range(3))
    return (lo, hi) if all(lo[d] <= hi[d] for d in range(3)) else None


def vol(b):
    return (b[1][0] - b[0][0] + 1) * (b[1][1] - b[0][1] + 1) * (b[1][2] - b[0][2] + 1)


def ghost_slabs(lo, hi, g):
    """The ghost region of a box grown by g, as 6 disjoint boxes."""
    el = tuple(v - g for v in lo)
    eh = tuple(v + g for v in hi)
    return [((el[0], el[1], el[2]), (eh[0], eh[1], lo[2] - 1)),
            ((el[0], el[1], hi[2] + 1), (eh[0], eh[1], eh[2])),
            ((el[0], el[1], lo[2]), (eh[0], lo[1] - 1, hi[2])),
            ((el[0], hi[1] + 1, lo[2]), (eh[0], eh[1], hi[2])),
            ((el[0], lo[1], lo[2]), (lo[0] - 1, hi[1], hi[2])),
            ((hi[0] + 1, lo[1], lo[2]), (eh[0], hi[1], hi[2]))]


class OPatch:
    def __init__(self, lev, idx, lo, hi, state, dx, g):
        self.lev, self.idx, self.lo, self.hi, self.g = lev, idx, tuple(lo), tuple(hi), g
        self.n = tuple(hi[d] - lo[d] + 1 for d in range(3))
        self.state = state
        self.dx = dx
        self.P = O.patch(state, self.n, g, dx)
        self.glo = tuple(lo[d] - g for d in range(3))

    def arr(self, b):
        """global box -> array-index box"""
        return (tuple(b[0][d] - self.glo[d] for d in range(3)), tuple(b[1][d] - self.glo[d] for d in range(3)))


class OHierarchy:
    def __init__(self, boxes, n0, states, dx0, g=4, prm=None):
        """boxes[l] = [(lo, hi)], states[l][i] = float64 array of synth layout."""
        self.n0, self.g = n0, g
        self.prm = prm if prm is not None else O.params()
        self.levels = []
        for l, bl in enumerate(boxes):
            dx = tuple(v / 2 ** l for v in dx0)
            self.levels.append([OPatch(l, i, lo, hi, states[l][i], dx, g) for i, (lo, hi) in enumerate(bl)])
        self._build_metadata()

    # ------------------------------------------------------------ metadata
    def copies(self, l):
        """(src, dst, box, off) same-level ghost copies of level l; periodic
        images of the level-l domain included."""
        n = self.n0 * 2 ** l
        out = []
        pats = self.levels[l]
        shifts = [(a, b, c) for c in (-n, 0, n) for b in (-n, 0, n) for a in (-n, 0, n)]
        for D in pats:
            # ghost-extended box grown by one cell: its outer cell layer
            # carries the faces on the outer planes of D's face arrays
            ext = (tuple(v - self.g - 1 for v in D.lo), tuple(v + self.g + 1 for v in D.hi))
            for S in pats:
                for sh in shifts:
                    if S is D and sh == (0, 0, 0):
                        continue
                    img = (tuple(S.lo[d] + sh[d] for d in range(3)), tuple(S.hi[d] + sh[d] for d in range(3)))
                    b = isect(ext, img)
                    if b:
                        out.append((S.idx, D.idx, b, tuple(-s for s in sh)))
        return out

    def prolongs(self, l):
        """(coarse, fine, coarse box) items filling the ghost zones of level l+1."""
        out = []
        for F in self.levels[l + 1]:
            for slab in ghost_slabs(F.lo, F.hi, self.g):
                cb = (tuple(v // 2 for v in slab[0]), tuple(v // 2 for v in slab[1]))
                for Cp in self.levels[l]:
                    b = isect(cb, (Cp.lo, Cp.hi))
                    if b:
                        out.append((Cp.idx, F.idx, b))
        return out

    def restricts(self, l):
        """(fine, coarse, coarse box): the coarsened fine interior clipped to the
        coarse interior grown by one cell (so that coarse faces on the coarse
        patch's boundary that the fine patch covers are restricted too)."""
        out = []
        for F in self.levels[l + 1]:
            cb = (tuple(v // 2 for v in F.lo), tuple((v + 1) // 2 - 1 for v in F.hi))
            for Cp in self.levels[l]:
                b = isect(cb, (tuple(v - 1 for v in Cp.lo), tuple(v + 1 for v in Cp.hi)))
                if b:
                    out.append((F.idx, Cp.idx, b))
        return out

    def _build_metadata(self):
        self.reg = {}   # (lev, fine idx, side, kind, axis) -> fine register info
        self.cap = {}   # (lev, patch idx) -> list of (kind, axis, global box, key)
        self.dep = {}   # lev (coarse) -> list of deposits
        for l in range(len(self.levels)):
            self.cap[l] = {P.idx: [] for P in self.levels[l]}
        for l in range(1, len(self.levels)):
            deps = []
            for F in self.levels[l]:
                for d in range(3):
                    for side in (0, 1):
                        fidx = F.lo[d] if side == 0 else F.hi[d] + 1
                        # fine face register over the whole side
                        flo, fhi = list(F.lo), list(F.hi)
                        flo[d] = fhi[d] = fidx
                        key = ("F", F.idx, d, side)
                        self.reg[(l,) + key] = {"lo": tuple(flo), "hi": tuple(fhi),
                                                "buf": np.zeros((5, vol((flo, fhi))))}
                        self.cap[l][F.idx].append(("face", d, (tuple(flo), tuple(fhi)), (l,) + key))
                        # coarse faces of this side, split by the coarse patch owning the outside cell
                        cidx = fidx // 2
                        out_cell = cidx - 1 if side == 0 else cidx
                        clo = [v // 2 for v in F.lo]
                        chi = [(v + 1) // 2 - 1 for v in F.hi]
                        clo[d] = chi[d] = cidx
                        for Cp in self.levels[l - 1]:
                            if not (Cp.lo[d] <= out_cell <= Cp.hi[d]):
                                continue
                            t = [e for e in range(3) if e != d]
                            blo, bhi = list(clo), list(chi)
                            ok = True
                            for e in t:
                                blo[e] = max(clo[e], Cp.lo[e])
                                bhi[e] = min(chi[e], Cp.hi[e])
                                ok = ok and blo[e] <= bhi[e]
                            if not ok:
                                continue
                            ckey = ("FC", F.idx, d, side, Cp.idx)
                            box = (tuple(blo), tuple(bhi))
                            self.reg[(l,) + ckey] = {"lo": box[0], "hi": box[1], "buf": np.zeros((5, vol(box)))}
                            self.cap[l - 1][Cp.idx].append(("face", d, box, (l,) + ckey))
                            deps.append(("face", Cp.idx, d, box, (l,) + key, (l,) + ckey))
                        # edges on this side: the two axes a != d
                        for a in range(3):
                            if a == d:
                                continue
                            tt = 3 - a - d
                            elo, ehi = list(F.lo), list(F.hi)
                            elo[d] = ehi[d] = fidx
                            ehi[tt] = F.hi[tt] + 1
                            ekey = ("E", F.idx, d, side, a)
                            ebox = (tuple(elo), tuple(ehi))
                            self.reg[(l,) + ekey] = {"lo": ebox[0], "hi": ebox[1], "buf": np.zeros((1, vol(ebox)))}
                            self.cap[l][F.idx].append(("edge", a, ebox, (l,) + ekey))
                            cl, ch = [v // 2 for v in F.lo], [(v + 1) // 2 - 1 for v in F.hi]
                            cl[d] = ch[d] = cidx
                            ch[tt] = (F.hi[tt] + 1) // 2
                            for Cp in self.levels[l - 1]:
                                # edges used by Cp's interior face updates
                                blo = [max(cl[e], Cp.lo[e]) for e in range(3)]
                                bhi = [min(ch[e], Cp.hi[e] + (0 if e == a else 1)) for e in range(3)]
                                if any(blo[e] > bhi[e] for e in range(3)):
                                    continue
                                box = (tuple(blo), tuple(bhi))
                                ckey = ("EC", F.idx, d, side, a, Cp.idx)
                                self.reg[(l,) + ckey] = {"lo": box[0], "hi": box[1], "buf": np.zeros((1, vol(box)))}
                                self.cap[l - 1][Cp.idx].append(("edge", a, box, (l,) + ckey))
                                deps.append(("edge", Cp.idx, a, box, (l,) + ekey, (l,) + ckey))
            self.dep[l - 1] = deps
        self.copy_lists = [self.copies(l) for l in range(len(self.levels))]
        self.prolong_lists = [self.prolongs(l) for l in range(len(self.levels) - 1)]
        self.restrict_lists = [self.restricts(l) for l in range(len(self.levels) - 1)]
        self.corr = {}
        for l in range(len(self.levels) - 1):
            for Cp in self.levels[l]:
                if any(dd[1] == Cp.idx for dd in self.dep[l]):
                    self.corr[(l, Cp.idx)] = np.zeros((18,) + Cp.state.shape[1:])

    # ------------------------------------------------------------ operations
    def fill(self, l):
        pats = self.levels[l]
        for pass_ in (0, 1):
            for (s, d, b, off) in self.copy_lists[l]:
                O.copy(pats[s].P, pats[s].lo, pats[d].P, pats[d].lo, b[0], b[1], off, pass_)

    def prolong(self, l):
        C, F = self.levels[l], self.levels[l + 1]
        for (c, f, b) in self.prolong_lists[l]:
            O.prolong(C[c].P, C[c].lo, F[f].P, F[f].lo, b[0], b[1])

    def restrict(self, l):
        C, F = self.levels[l], self.levels[l + 1]
        for pass_ in (0, 1):
            for (f, c, b) in self.restrict_lists[l]:
                O.restrict(F[f].P, F[f].lo, C[c].P, C[c].lo, b[0], b[1], pass_)

    def advance(self, l, k, dt, first):
        for P in self.levels[l]:
            faces, edges = [], []
            for (kind, ax, box, key) in self.cap[l][P.idx]:
                fine_side = key[1] in ("F", "E")
                mode = 0 if (not fine_side or first) else 1
                buf = self.reg[key]["buf"]
                ab = P.arr(box)
                (faces if kind == "face" else edges).append((ax, ab[0], ab[1], mode, buf))
            cap = O.captures(faces) if faces else None
            ecap = O.captures(edges) if edges else None
            nneg = O.advance(P.P, self.prm, dt, k, cap, ecap)
            if nneg:
                raise FloatingPointError("oracle AMR: %d non-positive cells on level %d" % (nneg, l))

    def reflux(self, l):
        for key in self.corr:
            if key[0] == l:
                self.corr[key][...] = 0.0
        C = self.levels[l]
        for (kind, c, ax, box, fkey, ckey) in self.dep[l]:
            fr, cr = self.reg[fkey], self.reg[ckey]
            corr = self.corr[(l, c)]
            fn = O.deposit_faces if kind == "face" else O.deposit_edges
            fn(C[c].P, C[c].lo, corr, ax, box[0], box[1], fr["buf"], fr["lo"], fr["hi"], cr["buf"])
        for (ll, c), corr in self.corr.items():
            if ll == l:
                O.correct(C[c].P, corr)

    def cfl_dt0(self):
        dts = []
        for l, pats in enumerate(self.levels):
            for P in pats:
                dts.append(O.cfl_dt(P.P, self.prm) * 2 ** l)
        return min(dts)

    def step(self, l, k, dt, first=True):
        last = l + 1 >= len(self.levels)
        if not last:
            self.prolong(l)
            self.fill(l + 1)
        self.advance(l, k, dt, first)
        if not last:
            self.step(l + 1, 2, 0.5 * dt, True)
            self.fill(l + 1)
            self.step(l + 1, 0, 0.5 * dt, False)
            self.reflux(l)
            self.restrict(l)
            if self.prm.p_floor > 0.0 or self.prm.rho_floor > 0.0:
                # refluxing changes cells outside any advance: the floors
                # again (reading R33)
                for P in self.levels[l]:
                    O.floor(P.P, self.prm)

    def initialise(self):
        for l in range(len(self.levels) - 2, -1, -1):
            self.restrict(l)

    def coarse_step(self, dt=None):
        dt0 = self.cfl_dt0() if dt is None else dt
        self.fill(0)
        self.step(0, 0, dt0)
        return dt0

    def sums(self):
        """Composite totals: after restriction the base level holds them."""
        return sum(O.sums(P.P) for P in self.levels[0])

    def divb_max(self):
        return max(O.divb_max(P.P) for pats in self.levels for P in pats)
