"""Seeded synthetic AMR hierarchies (static, refinement ratio 2) and their
initial blast-wave data.  Box placement only: no solver arithmetic.

A hierarchy is a list of levels; level l is a list of interior boxes
``(lo, hi)`` (inclusive, level-l global cell index; the level-l domain has
``n0 * 2**l`` cells per side on the periodic cube [-1/2, 1/2]^3).  Every fine
box is aligned to its level (even lower corner, even extent) and lies inside
the union of the parent level's boxes eroded by ``margin`` parent cells (a
cube erosion), so a fine patch's ghost region and the slope stencil of its
prolongation stay inside parent interiors, and fine patches are at least
``margin`` parent cells away from the domain boundary.
"""
from __future__ import annotations

import math

import numpy as np

from . import GAMMA, _set_cells, empty_patch, uniform_pm1


def _even_down(v):
    return v - (v % 2)


def _box_meets_shell(lo, hi, n, r1, r2):
    """Does the box of cells [lo, hi] (level with n cells a side on
    [-1/2, 1/2]^3) contain points at radius in [r1, r2]?"""
    dx = 1.0 / n
    dmin2, dmax2 = 0.0, 0.0
    for d in range(3):
        a, b = -0.5 + lo[d] * dx, -0.5 + (hi[d] + 1) * dx
        near = 0.0 if a <= 0.0 <= b else min(abs(a), abs(b))
        far = max(abs(a), abs(b))
        dmin2 += near * near
        dmax2 += far * far
    return math.sqrt(dmin2) <= r2 and math.sqrt(dmax2) >= r1


def _cuts(rng, lo, hi, smin, smax):
    """Split [lo, hi] into consecutive even-length pieces of log-uniform size."""
    out = []
    a = lo
    while a <= hi:
        s = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        s = max(smin, s - (s % 2))
        b = min(hi, a + s - 1)
        if hi - b < smin:  # do not leave a sliver
            b = hi
        out.append((a, b))
        a = b + 1
    return out


def shell_hierarchy(n0=64, levels=4, seed=1112, r_in=0.25, r_out=0.35, jitter=0.1,
                    size_min=8, size_max=64, margin=3, level0_split=1):
    """Levels 1.. cover the shell r in [r_in, r_out] * (1 +- jitter) (jittered
    per level) with uneven boxes; level 0 is the periodic domain, optionally
    split into level0_split^3 patches."""
    rng = np.random.default_rng(seed)
    L0 = []
    edges = np.linspace(0, n0, level0_split + 1).astype(int)
    for k in range(level0_split):
        for j in range(level0_split):
            for i in range(level0_split):
                L0.append(((int(edges[i]), int(edges[j]), int(edges[k])),
                           (int(edges[i + 1]) - 1, int(edges[j + 1]) - 1, int(edges[k + 1]) - 1)))
    H = [L0]
    for lev in range(1, levels):
        n = n0 * 2 ** lev
        r1 = r_in * (1.0 + jitter * rng.uniform(-1, 1))
        r2 = r_out * (1.0 + jitter * rng.uniform(-1, 1))
        allowed = _allowed_mask(H[-1], n // 2, margin)  # parent resolution
        boxes = []
        # tile the refined domain with uneven boxes; keep those that meet the
        # shell, halving the ones that stick out of the allowed region
        lo_all, hi_all = 2 * margin, n - 2 * margin - 1
        cx = _cuts(rng, lo_all, hi_all, size_min, size_max)
        cy = _cuts(rng, lo_all, hi_all, size_min, size_max)
        cz = _cuts(rng, lo_all, hi_all, size_min, size_max)
        stack = [((x0, y0, z0), (x1, y1, z1)) for (z0, z1) in cz for (y0, y1) in cy for (x0, x1) in cx]
        while stack:
            lo, hi = stack.pop()
            if not _box_meets_shell(lo, hi, n, r1, r2):
                continue
            sub = allowed[lo[2] // 2:(hi[2] + 1) // 2, lo[1] // 2:(hi[1] + 1) // 2, lo[0] // 2:(hi[0] + 1) // 2]
            if sub.all():
                boxes.append((lo, hi))
                continue
            if not sub.any():
                continue
            ext = [hi[d] - lo[d] + 1 for d in range(3)]
            d = int(np.argmax(ext))
            if ext[d] < 2 * size_min:
                continue
            mid = lo[d] + _even_down(ext[d] // 2)
            a_hi, b_lo = list(hi), list(lo)
            a_hi[d], b_lo[d] = mid - 1, mid
            stack.append((lo, tuple(a_hi)))
            stack.append((tuple(b_lo), hi))
        if not boxes:
            break
        boxes.sort(key=lambda b: (b[0][2], b[0][1], b[0][0]))
        H.append(boxes)
    return H


def _allowed_mask(parents, n, margin):
    """Parent-level cells at least `margin` cells inside the union of the
    parent boxes (array [z, y, x])."""
    m = np.zeros((n, n, n), dtype=bool)
    for (lo, hi) in parents:
        m[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
    out = m.copy()
    for d in range(3):  # separable erosion by the cube of half-width `margin`
        cur = out.copy()
        for s in range(1, margin + 1):
            out &= np.roll(cur, s, axis=d) & np.roll(cur, -s, axis=d)
    # the domain boundary counts as outside for refined levels
    if margin:
        out[:margin] = out[-margin:] = False
        out[:, :margin] = out[:, -margin:] = False
        out[:, :, :margin] = out[:, :, -margin:] = False
    return out


def check_hierarchy(H, n0, margin=3):
    """Alignment, disjointness within a level, proper nesting with margin."""
    for lev, boxes in enumerate(H):
        n = n0 * 2 ** lev
        for (lo, hi) in boxes:
            for d in range(3):
                assert 0 <= lo[d] <= hi[d] < n
                if lev:
                    assert lo[d] % 2 == 0 and (hi[d] + 1) % 2 == 0
        for a in range(len(boxes)):
            for b in range(a + 1, len(boxes)):
                la, ha = boxes[a]
                lb, hb = boxes[b]
                assert any(ha[d] < lb[d] or hb[d] < la[d] for d in range(3)), (lev, a, b)
        if lev:
            allowed = _allowed_mask(H[lev - 1], n // 2, margin)
            for (lo, hi) in boxes:
                sub = allowed[lo[2] // 2:(hi[2] + 1) // 2, lo[1] // 2:(hi[1] + 1) // 2, lo[0] // 2:(hi[0] + 1) // 2]
                assert sub.size and sub.all(), (lev, lo, hi)


def blast_patch(lo, hi, lev, n0, g, seed=1112, noise=0.01, p_in=10.0, p_out=0.1, r0=0.1,
                bfield=(1.0 / math.sqrt(2.0), 1.0 / math.sqrt(2.0), 0.0), align=8):
    """Blast-wave data (rho = 1 + noise U(-1,1) with the level-l counter, p =
    p_in for r < r0 else p_out, v = 0, uniform B) on the interior of one
    patch; ghosts left at zero."""
    n = n0 * 2 ** lev
    nn = tuple(hi[d] - lo[d] + 1 for d in range(3))
    st = empty_patch(nn, g, align=align)
    nx, ny, nz = nn
    st[5, g:g + nz, g:g + ny, g:g + nx + 1] = bfield[0]
    st[6, g:g + nz, g:g + ny + 1, g:g + nx] = bfield[1]
    st[7, g:g + nz + 1, g:g + ny, g:g + nx] = bfield[2]
    dx = 1.0 / n
    x = -0.5 + (np.arange(lo[0], hi[0] + 1) + 0.5) * dx
    y = -0.5 + (np.arange(lo[1], hi[1] + 1) + 0.5) * dx
    z = -0.5 + (np.arange(lo[2], hi[2] + 1) + 0.5) * dx
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    p = np.where(X * X + Y * Y + Z * Z < r0 * r0, p_in, p_out)
    idx = (np.arange(lo[0], hi[0] + 1, dtype=np.uint64)[None, None, :]
           + np.uint64(n) * (np.arange(lo[1], hi[1] + 1, dtype=np.uint64)[None, :, None]
                             + np.uint64(n) * np.arange(lo[2], hi[2] + 1, dtype=np.uint64)[:, None, None]))
    rho = 1.0 + noise * uniform_pm1(seed + lev, idx)
    _set_cells(st, nn, g, rho, 0.0, 0.0, 0.0, p, GAMMA)
    return st, (dx, dx, dx)
