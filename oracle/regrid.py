"""Oracle of regridding a hierarchy's levels (Sec. 2.1: each iteration of a
level's grids is made from its parent level's flags; the O step of Sec. 2.2
moves the data into it), ratio 2, in plain numpy loops, level by level from
the coarsest regridded one, each new level from the new level below it.

TEST INFRASTRUCTURE ONLY (imported by tests/), sharing no code with the
library.

The steps, with the readings the paper leaves open (each listed with the
design notes):
  1. the parent level (the one below the level made) gets its ghost zones
     as at the start of its step (level 0 filled, then each finer level
     prolonged and filled) and its interior cells are flagged (orc_flag);
  2. the flags are grown by `buffer` cells (every cell within the cube of
     half-width `buffer` of a flagged cell) and kept only where the new
     level is properly nested: at least `margin` parent cells inside the
     union of the parent grids, the outside of that union and the domain
     boundary counting as outside;
  3. the kept flags, over the bounding box of the parent grids, are
     clustered (oracle/cluster.py, Berger & Rigoutsos), and each box is
     halved until it lies in the nested region (fit);
  4. each cluster box is cut by every parent grid it meets and each piece
     refined by 2 (new grids nested in one parent each);
  5. every new patch is filled by the data transfer (oracle/transfer.py):
     the previous iteration's cells and shared faces where they meet, the
     parent's prolongation elsewhere.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O
from . import transfer as T
from .cluster import cluster


def _cube_or(m, r):
    """m grown by the cube of half-width r (brute force over the offsets)."""
    nz, ny, nx = m.shape
    p = np.zeros((nz + 2 * r, ny + 2 * r, nx + 2 * r), dtype=bool)
    p[r:r + nz, r:r + ny, r:r + nx] = m
    out = np.zeros_like(m)
    for dz in range(2 * r + 1):
        for dy in range(2 * r + 1):
            for dx in range(2 * r + 1):
                out |= p[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    return out


def _cube_and(m, r):
    """Cells whose whole cube of half-width r lies in m (outside is False)."""
    nz, ny, nx = m.shape
    p = np.zeros((nz + 2 * r, ny + 2 * r, nx + 2 * r), dtype=bool)
    p[r:r + nz, r:r + ny, r:r + nx] = m
    out = np.ones_like(m)
    for dz in range(2 * r + 1):
        for dy in range(2 * r + 1):
            for dx in range(2 * r + 1):
                out &= p[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    return out


def children(cluster_boxes, parent_boxes):
    """Step 4: every (cluster box, parent grid) intersection, refined by 2."""
    out = []
    for clo, chi in cluster_boxes:
        for plo, phi in parent_boxes:
            lo = [clo[d] if clo[d] > plo[d] else plo[d] for d in range(3)]
            hi = [chi[d] if chi[d] < phi[d] else phi[d] for d in range(3)]
            if lo[0] <= hi[0] and lo[1] <= hi[1] and lo[2] <= hi[2]:
                out.append((tuple(2 * v for v in lo), tuple(2 * v + 1 for v in hi)))
    return out


def fit(boxes, flags, allowed):
    """Step 3b: each cluster box shrunk to its flags' bounding box; one with
    a cell outside the nested region is cut in two across its longest axis
    (lowest axis on ties, the low piece one slice longer when the length is
    odd) and each piece treated the same way, the low piece first."""
    out = []
    stack = [tuple(b) for b in reversed(boxes)]
    while stack:
        lo, hi = stack.pop()
        cells = [(z, y, x) for z in range(lo[0], hi[0] + 1) for y in range(lo[1], hi[1] + 1)
                 for x in range(lo[2], hi[2] + 1) if flags[z, y, x]]
        if not cells:
            continue
        lo = tuple(min(c[d] for c in cells) for d in range(3))
        hi = tuple(max(c[d] for c in cells) for d in range(3))
        if allowed[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1].all():
            out.append((lo, hi))
            continue
        ext = [hi[d] - lo[d] + 1 for d in range(3)]
        d = ext.index(max(ext))
        cut = lo[d] + (ext[d] + 1) // 2          # first slice of the high piece
        a_hi = tuple(cut - 1 if e == d else hi[e] for e in range(3))
        b_lo = tuple(cut if e == d else lo[e] for e in range(3))
        stack.append((b_lo, hi))
        stack.append((lo, a_hi))
    return out


def flags_of_parent(oh, theta, lp=None):
    """Step 1: the flags of level lp (default: the one below the finest),
    one (nz, ny, nx) array per grid."""
    lp = len(oh.levels) - 2 if lp is None else lp
    oh.fill(0)
    for k in range(1, lp + 1):
        oh.prolong(k - 1)
        oh.fill(k)
    return [O.flag(P.P, oh.prm, theta) for P in oh.levels[lp]]


def _next_level(oh, lp, old, theta, buffer, margin, eff, min_size, energy_mode, empty):
    """Steps 1-5 for level lp + 1 of `oh` (whose levels 0..lp hold the new
    iteration's data) from its previous iteration `old` (a list of OPatch).
    Returns (boxes, states, fallbacks)."""
    parents = oh.levels[lp]
    flags = flags_of_parent(oh, theta, lp)
    blo = [min(P.lo[d] for P in parents) for d in range(3)]
    bhi = [max(P.hi[d] for P in parents) for d in range(3)]
    shape = (bhi[2] - blo[2] + 1, bhi[1] - blo[1] + 1, bhi[0] - blo[0] + 1)
    f = np.zeros(shape, dtype=bool)
    inside = np.zeros(shape, dtype=bool)
    for P, fl in zip(parents, flags):
        z0, y0, x0 = P.lo[2] - blo[2], P.lo[1] - blo[1], P.lo[0] - blo[0]
        nx, ny, nz = P.n
        f[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] |= fl.astype(bool)
        inside[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx] = True
    if buffer > 0:
        f = _cube_or(f, buffer)
    allowed = _cube_and(inside, margin)
    f &= allowed
    if not f.any():
        return [], [], 0
    cl = []
    for lo, hi in fit(cluster(f, eff, min_size), f, allowed):   # (z, y, x), box-local
        cl.append(((lo[2] + blo[0], lo[1] + blo[1], lo[0] + blo[2]),
                   (hi[2] + blo[0], hi[1] + blo[1], hi[0] + blo[2])))
    new = children(cl, [(P.lo, P.hi) for P in parents])
    dxf = tuple(v / 2 for v in parents[0].dx)
    olds = [(P.state, (P.lo, P.hi)) for P in old]
    coarse = [(P.state, (P.lo, P.hi), P.g, P.dx) for P in parents]
    states, nfall = [], 0
    for lo, hi in new:
        n = tuple(hi[d] - lo[d] + 1 for d in range(3))
        st = empty(n, oh.g)
        nfall += T.transfer(st, (lo, hi), oh.g, dxf, olds, coarse, energy_mode)
        states.append(st)
    return new, states, nfall


def regrid_levels(oh, theta, first=None, buffer=1, margin=3, eff=0.7, min_size=2, energy_mode=1, empty=None):
    """Levels `first` (default: the finest) .. finest replaced, coarsest
    first, each from the flags of the new level below it; a level with no
    kept flag ends the hierarchy.  Returns (boxes, states, fallbacks) (the
    kept levels' states are the hierarchy's own arrays).  `empty(n, g)`
    makes a zero patch array of the library's layout."""
    from .amr import OHierarchy
    L = len(oh.levels)
    first = L - 1 if first is None else first
    boxes = [[(P.lo, P.hi) for P in lv] for lv in oh.levels[:first]]
    states = [[P.state for P in lv] for lv in oh.levels[:first]]
    nfall = 0
    dx0 = oh.levels[0][0].dx
    for m in range(first, L):
        parent = oh if m == first else OHierarchy(boxes, oh.n0, states, dx0, g=oh.g, prm=oh.prm)
        nb, ns, nf = _next_level(parent, m - 1, oh.levels[m], theta, buffer, margin, eff, min_size,
                                 energy_mode, empty)
        nfall += nf
        if not nb:
            break
        boxes.append(nb)
        states.append(ns)
    return boxes, states, nfall


def regrid_finest(oh, theta, buffer=1, margin=3, eff=0.7, min_size=2, energy_mode=1, empty=None):
    """regrid_levels of the finest level alone."""
    return regrid_levels(oh, theta, len(oh.levels) - 1, buffer, margin, eff, min_size, energy_mode, empty)
