"""Seeded deep AMR hierarchies on a k^-4 random velocity field (static,
refinement ratio 2).  Input generation only: no solver arithmetic.

Field: each velocity component has Fourier amplitudes |v(k)|^2 ~ |k|^-4 for
1 <= |k| <= k_max (base-box wavenumbers) with Gaussian random phases (no
Helmholtz projection), generated on an m^3 grid by an inverse FFT and scaled
so that the rms speed is `mach` times the sound speed; rho = 1, p = 1/gamma
(sound speed 1), a uniform field B = sqrt(2 p) x (plasma beta 1).

Hierarchy: level 0 is the periodic base cube of n0 cells per side; level l
has n0 2^l cells per side.  Candidate boxes for level l are uneven seeded cuts
(even corners and extents between size_min and size_max) of every level-(l-1)
box refined, shrunk by `margin` parent cells and clipped to `margin` parent
cells inside the domain (so each fine box, coarsened and grown by the margin,
lies in its parent); candidates are taken in decreasing order of the mean refinement
indicator |curl v| + |div v| (the m^3 field's central differences) until the
level holds about n_cells[l] cells.
"""
from __future__ import annotations

import math

import numpy as np

from . import GAMMA, _set_cells, empty_patch


def kminus4_velocity(m=64, kmax=16, mach=5.0, seed=5, gamma=GAMMA):
    """Velocity field (3, m, m, m) [z, y, x] on the unit periodic cube."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(m, d=1.0 / m)
    kr = np.fft.rfftfreq(m, d=1.0 / m)
    KZ, KY, KX = np.meshgrid(k, k, kr, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    shell = (kk >= 1.0) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[shell] = kk[shell] ** -2.0  # |v(k)| ~ |k|^-2, so |v(k)|^2 ~ |k|^-4
    v = np.empty((3, m, m, m))
    for c in range(3):
        ph = rng.normal(size=kk.shape) + 1j * rng.normal(size=kk.shape)
        v[c] = np.fft.irfftn(amp * ph, s=(m, m, m), axes=(0, 1, 2))
    cs = 1.0  # p = 1/gamma, rho = 1
    rms = math.sqrt(float(np.mean(np.sum(v * v, axis=0))))
    return v * (mach * cs / rms)


def indicator(v):
    """|curl v| + |div v| on the periodic grid (central differences, unit box)."""
    m = v.shape[1]
    h = 1.0 / m

    def d(f, axis):  # axis: 0 x, 1 y, 2 z  (array axes are z, y, x)
        ax = 2 - axis
        return (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / (2 * h)

    vx, vy, vz = v[0], v[1], v[2]
    cx = d(vz, 1) - d(vy, 2)
    cy = d(vx, 2) - d(vz, 0)
    cz = d(vy, 0) - d(vx, 1)
    div = d(vx, 0) + d(vy, 1) + d(vz, 2)
    return np.sqrt(cx * cx + cy * cy + cz * cz) + np.abs(div)


def _prefix3(a):
    """Zero-padded 3D prefix sums of a[z, y, x]."""
    s = np.zeros(tuple(n + 1 for n in a.shape))
    s[1:, 1:, 1:] = a.cumsum(0).cumsum(1).cumsum(2)
    return s


def _box_mean(pref, m, lo, hi, n):
    """Mean of the m^3 field over the level box [lo, hi] (level with n cells a
    side), each box mapped onto the m^3 grid (at least one cell)."""
    a = [int(math.floor(lo[d] * m / n)) for d in range(3)]
    b = [max(a[d] + 1, int(math.ceil((hi[d] + 1) * m / n))) for d in range(3)]
    x0, y0, z0 = a
    x1, y1, z1 = b
    tot = (pref[z1, y1, x1] - pref[z0, y1, x1] - pref[z1, y0, x1] - pref[z1, y1, x0] + pref[z0, y0, x1]
           + pref[z0, y1, x0] + pref[z1, y0, x0] - pref[z0, y0, x0])
    return tot / ((x1 - x0) * (y1 - y0) * (z1 - z0))


def _cuts(rng, lo, hi, smin, smax):
    """Seeded uneven even-length cuts of [lo, hi] (lo even, hi + 1 - lo even)."""
    out = []
    a = lo
    while a <= hi:
        rest = hi + 1 - a
        if rest <= smax:
            out.append((a, hi))
            break
        s = int(rng.integers(smin // 2, smax // 2 + 1)) * 2
        if rest - s < smin:
            s = rest - smin
        out.append((a, a + s - 1))
        a += s
    return out


def _covered(lo, hi, plo, phi):
    """Is the box [lo, hi] covered by the union of disjoint boxes (plo, phi)?"""
    ilo = np.maximum(plo, np.asarray(lo))
    ihi = np.minimum(phi, np.asarray(hi))
    ext = np.clip(ihi - ilo + 1, 0, None)
    return int(np.prod(ext, axis=1).sum()) == int(np.prod(np.asarray(hi) - np.asarray(lo) + 1))


def deep_hierarchy(n0=32, levels=8, n_cells=None, m=64, kmax=16, mach=5.0, seed=5, size_min=8, size_max=64,
                   margin=3):
    """Returns (boxes per level, velocity field, indicator field)."""
    if n_cells is None:
        n_cells = [n0 ** 3 * 3 ** l for l in range(levels)]
    v = kminus4_velocity(m, kmax, mach, seed)
    ind = indicator(v)
    pref = _prefix3(ind)
    rng = np.random.default_rng(seed)
    H = [[((0, 0, 0), (n0 - 1,) * 3)]]
    for lev in range(1, levels):
        n = n0 * 2 ** lev
        parents = H[-1]
        plo = np.array([p[0] for p in parents])
        phi = np.array([p[1] for p in parents])
        cands = []
        for (lo, hi) in parents:
            # the refined parent shrunk by `margin` parent cells (proper nesting),
            # clipped to `margin` parent cells inside the domain
            flo = [max(2 * (v_ + margin), 2 * margin) for v_ in lo]
            fhi = [min(2 * (v_ - margin) + 1, n - 2 * margin - 1) for v_ in hi]
            if any(fhi[d] - flo[d] + 1 < size_min for d in range(3)):
                continue
            cx = _cuts(rng, flo[0], fhi[0], size_min, size_max)
            cy = _cuts(rng, flo[1], fhi[1], size_min, size_max)
            cz = _cuts(rng, flo[2], fhi[2], size_min, size_max)
            for (z0, z1) in cz:
                for (y0, y1) in cy:
                    for (x0, x1) in cx:
                        cands.append(((x0, y0, z0), (x1, y1, z1)))
        scored = []
        for (lo, hi) in cands:
            # coarsened and grown by the margin: inside the parents' union and the domain
            glo = [lo[d] // 2 - margin for d in range(3)]
            ghi = [hi[d] // 2 + margin for d in range(3)]
            if min(glo) < 0 or max(ghi) > n // 2 - 1:
                continue
            if not _covered(glo, ghi, plo, phi):
                continue
            scored.append((_box_mean(pref, m, lo, hi, n), lo, hi))
        scored.sort(key=lambda t: -t[0])
        level, cells = [], 0
        for sc, lo, hi in scored:
            if cells >= n_cells[lev]:
                break
            level.append((tuple(lo), tuple(hi)))
            cells += int(np.prod(np.asarray(hi) - np.asarray(lo) + 1))
        if not level:
            break
        H.append(sorted(level))
    return H, v, ind


def _sample(v, lo, hi, res):
    """Trilinear interpolation of the periodic m^3 field v (3, m, m, m) at the
    centres of the level cells [lo, hi] (level with res cells a side)."""
    m = v.shape[1]
    ws, ids = [], []
    for d in range(3):
        u = (np.arange(lo[d], hi[d] + 1) + 0.5) / res * m - 0.5
        i0 = np.floor(u).astype(int)
        f = u - i0
        ids.append(((i0 % m), ((i0 + 1) % m)))
        ws.append((1.0 - f, f))
    out = np.zeros((3, hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1))
    for c in (0, 1):
        for b in (0, 1):
            for a in (0, 1):
                w = ws[2][c][:, None, None] * ws[1][b][None, :, None] * ws[0][a][None, None, :]
                sel = np.ix_(ids[2][c], ids[1][b], ids[0][a])
                for q in range(3):
                    out[q] += w * v[q][sel]
    return out


def turb_patch(lo, hi, lev, n0, g, v, gamma=GAMMA):
    """Interior state of one patch (ghosts left at zero, as the hierarchy fills
    them): rho = 1, p = 1/gamma, v the m^3 field interpolated trilinearly to
    the cell centres (smooth on every level, so refinement adds no velocity
    jumps), B = sqrt(2 p) along x on every face.  Returns (state, dx)."""
    nn = tuple(hi[d] - lo[d] + 1 for d in range(3))
    nx, ny, nz = nn
    st = empty_patch(nn, g)
    res = n0 * 2 ** lev
    vc = _sample(v, lo, hi, res)
    p = 1.0 / gamma
    st[5, g:g + nz, g:g + ny, g:g + nx + 1] = math.sqrt(2.0 * p)
    _set_cells(st, nn, g, 1.0, vc[0], vc[1], vc[2], p, gamma)
    dx = 1.0 / res
    return st, (dx, dx, dx)
