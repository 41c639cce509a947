"""Oracle of the grid generation step of regridding: covering the cells a
level flags for refinement with boxes (Sec. 2.1 regridding; the paper leaves
the rule open and cites Berger's AMR papers, so the clustering here is the
point-clustering algorithm of Berger & Rigoutsos, IEEE Trans. SMC 21, 1278
(1991)), and the overlap lists between two iterations of a level (Sec. 2.1:
a new grid takes the data of the previous iteration's grids where they
overlap it).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product.  Plain
numpy on flag arrays and Python integers on boxes.

Clustering of the flagged cells of an integer array (readings, each also
listed with the design notes):
  1. a candidate box is first shrunk to the bounding box of its flags (no
     flags: no box);
  2. it is accepted when its efficiency (flagged cells / cells) is at least
     `eff`, or when no axis is at least 2 * min_size long (it cannot be cut
     into two pieces of min_size cells);
  3. otherwise it is cut between slices i and i+1 of one axis, both pieces
     at least min_size long: at a hole of the signature (a slice with no
     flags) if there is one, the hole nearest the box centre, ties to the
     lower slice, the axes tried in order; else at the strongest inflection,
     the sign change of the signature's second difference
     D(i) = S(i-1) - 2 S(i) + S(i+1) with the largest |D(i+1) - D(i)| over
     all axes, ties to the position nearer the centre, then the lower axis
     and slice; else at the middle of the longest axis;
  4. both pieces are clustered again; boxes come out in depth-first order
     (low piece first).
Pinned by what the algorithm must do: a solid block of flags gives exactly
that block, separated blocks are separated at their gap, an L of two blocks
is cut at its corner, every flagged cell is covered once, boxes are disjoint
and each accepted box meets the efficiency or the size bound.
"""
from __future__ import annotations

import numpy as np


def _bbox(flags, lo, hi):
    """Bounding box (inclusive) of the flags inside [lo, hi], or None."""
    sl = tuple(slice(lo[d], hi[d] + 1) for d in range(flags.ndim))
    sub = flags[sl]
    if not sub.any():
        return None
    nlo, nhi = [], []
    for d in range(flags.ndim):
        other = tuple(k for k in range(flags.ndim) if k != d)
        s = sub.any(axis=other)
        idx = np.nonzero(s)[0]
        nlo.append(lo[d] + int(idx[0]))
        nhi.append(lo[d] + int(idx[-1]))
    return tuple(nlo), tuple(nhi)


def signature(flags, lo, hi, d):
    """Flag counts of the slices of [lo, hi] normal to axis d."""
    sl = tuple(slice(lo[k], hi[k] + 1) for k in range(flags.ndim))
    sub = flags[sl].astype(np.int64)
    other = tuple(k for k in range(flags.ndim) if k != d)
    return [int(v) for v in sub.sum(axis=other)]


def choose_cut(flags, lo, hi, min_size):
    """(axis, i): cut after slice i (relative to lo) per reading 3, or None
    when no axis can be cut into two pieces of min_size cells."""
    nd = flags.ndim
    ext = [hi[d] - lo[d] + 1 for d in range(nd)]
    sigs = [signature(flags, lo, hi, d) for d in range(nd)]
    # holes: a slice with no flags; cut just below it (the hole goes to the
    # high piece) or just above it, whichever keeps both pieces long enough
    best = None
    for d in range(nd):
        L = ext[d]
        c2 = L - 1  # twice the centre in slice units
        for i in range(L):
            if sigs[d][i] != 0:
                continue
            for cut in (i - 1, i):  # cut after slice `cut`
                if cut + 1 < min_size or L - cut - 1 < min_size:
                    continue
                key = (abs(2 * i - c2), i, cut)
                if best is None or key < best[0]:
                    best = (key, d, cut)
        if best is not None:
            return best[1], best[2]
    # inflections: sign change between D(i) and D(i+1), cut after slice i
    best = None
    for d in range(nd):
        L = ext[d]
        s = sigs[d]
        if L < 4:
            continue
        D = [None] * L
        for i in range(1, L - 1):
            D[i] = s[i - 1] - 2 * s[i] + s[i + 1]
        for i in range(1, L - 2):
            a, b = D[i], D[i + 1]
            if not ((a < 0 < b) or (b < 0 < a)):
                continue
            if i + 1 < min_size or L - i - 1 < min_size:
                continue
            key = (-abs(b - a), abs(2 * i + 1 - (L - 1)), d, i)
            if best is None or key < best[0]:
                best = (key, d, i)
    if best is not None:
        return best[1], best[2]
    # the middle of the longest axis
    d = max(range(nd), key=lambda k: (ext[k], -k))
    if ext[d] < 2 * min_size:
        return None
    return d, ext[d] // 2 - 1


def cluster(flags, eff=0.7, min_size=2):
    """Boxes (lo, hi) covering the True cells of `flags` (an n-d bool array)."""
    flags = np.asarray(flags, dtype=bool)
    nd = flags.ndim
    out = []

    def rec(lo, hi):
        bb = _bbox(flags, lo, hi)
        if bb is None:
            return
        lo, hi = bb
        cells = 1
        for d in range(nd):
            cells *= hi[d] - lo[d] + 1
        sl = tuple(slice(lo[d], hi[d] + 1) for d in range(nd))
        n = int(flags[sl].sum())
        if n * 1.0 >= eff * cells:
            out.append((lo, hi))
            return
        cut = choose_cut(flags, lo, hi, min_size)
        if cut is None:
            out.append((lo, hi))
            return
        d, i = cut
        ahi = list(hi)
        ahi[d] = lo[d] + i
        blo = list(lo)
        blo[d] = lo[d] + i + 1
        rec(lo, tuple(ahi))
        rec(tuple(blo), hi)

    rec((0,) * nd, tuple(s - 1 for s in flags.shape))
    return out


def overlaps(new_boxes, old_boxes, grow=0):
    """(new, old, box) for every old-iteration box meeting a new box grown by
    `grow` cells (its ghost region), with the intersection (Sec. 2.1: a new
    grid takes the previous iteration's data where they overlap)."""
    out = []
    for i, (nlo, nhi) in enumerate(new_boxes):
        glo = [v - grow for v in nlo]
        ghi = [v + grow for v in nhi]
        for j, (olo, ohi) in enumerate(old_boxes):
            lo = tuple(max(glo[d], olo[d]) for d in range(len(nlo)))
            hi = tuple(min(ghi[d], ohi[d]) for d in range(len(nlo)))
            if all(lo[d] <= hi[d] for d in range(len(nlo))):
                out.append((i, j, (lo, hi)))
    return out
