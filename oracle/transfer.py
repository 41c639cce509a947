"""Oracle of the data transfer into a new iteration of a level (regridding,
Sec. 2.1; the O step of Sec. 2.2), ratio 2, by brute force over cells.

TEST INFRASTRUCTURE ONLY (imported by tests/), sharing no code with the
library.

A new fine patch F (level l+1) takes the previous iteration's data where it
meets an old patch O of level l+1: the cells of the intersection of the two
interiors, and every face that belongs to both face sets (interior faces
of F and of O, boundary faces included).  Everywhere else F's interior is
prolonged from the level-l patches (orc_prolong_new), coarse cell by coarse
cell: a coarse cell whose children lie in some old interior is skipped
(copied), and on the prolonged cells the coarse faces that lie in some old
patch's face set keep the copied sub-face values.  Old patches are aligned to
the coarse grid (even lower index, odd upper index), so a coarse cell is
either wholly old or wholly new.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import oracle as O


def _coarse_box(lo, hi):
    return tuple(v // 2 for v in lo), tuple((v + 1) // 2 - 1 for v in hi)


def copy_items(new_box, old_boxes):
    """(old index, kind, lo, hi) of every copy into the new box: kind -1 the
    cells of the intersection of the interiors, kind a the axis-a faces
    common to both face sets (normal index in [lo, hi + 1] of both)."""
    nlo, nhi = new_box
    out = []
    for j, (olo, ohi) in enumerate(old_boxes):
        lo = [max(nlo[d], olo[d]) for d in range(3)]
        hi = [min(nhi[d], ohi[d]) for d in range(3)]
        if all(lo[d] <= hi[d] for d in range(3)):
            out.append((j, -1, tuple(lo), tuple(hi)))
        for a in range(3):
            flo, fhi = list(lo), list(hi)
            fhi[a] = min(nhi[a] + 1, ohi[a] + 1)
            if all(flo[d] <= fhi[d] for d in range(3)):
                out.append((j, a, tuple(flo), tuple(fhi)))
    return out


def mask(new_box, old_boxes):
    """The prolongation mask of orc_prolong_new over the new box's coarse
    footprint, by testing every coarse cell and face against every old
    patch: bit 0 the cell lies in an old (coarsened) interior, bit 1 + 2 a +
    s its side-s axis-a face lies in an old patch's (coarsened) face set."""
    clo, chi = _coarse_box(*new_box)
    ext = [chi[d] - clo[d] + 1 for d in range(3)]
    m = np.zeros((ext[2], ext[1], ext[0]), np.uint8)
    oc = [_coarse_box(lo, hi) for lo, hi in old_boxes]
    for K, J, I in itertools.product(range(ext[2]), range(ext[1]), range(ext[0])):
        C3 = (clo[0] + I, clo[1] + J, clo[2] + K)
        bits = 0
        for olo, ohi in oc:
            if all(olo[d] <= C3[d] <= ohi[d] for d in range(3)):
                bits |= 1
            for a in range(3):
                for s in (0, 1):
                    f = C3[a] + s
                    inside = olo[a] <= f <= ohi[a] + 1 and all(
                        olo[d] <= C3[d] <= ohi[d] for d in range(3) if d != a)
                    if inside:
                        bits |= 1 << (1 + 2 * a + s)
        m[K, J, I] = bits
    return m, clo


def transfer(new_state, new_box, g, dx, old, coarse, energy_mode=1):
    """Fills the interior of a new fine patch (array new_state, interior
    new_box) from the old patches `old` [(state, (lo, hi))] and the level-l
    patches `coarse` [(state, (lo, hi), g_c, dx_c)].  Returns the count of
    energy fallbacks."""
    nlo, nhi = new_box
    n = tuple(nhi[d] - nlo[d] + 1 for d in range(3))
    Pf = O.patch(new_state, n, g, dx)
    for j, kind, lo, hi in copy_items(new_box, [b for _, b in old]):
        st, (olo, ohi) = old[j]
        on = tuple(ohi[d] - olo[d] + 1 for d in range(3))
        Po = O.patch(st, on, g, dx)
        O.transfer_copy(Po, olo, Pf, nlo, kind, lo, hi)
    m, mlo = mask(new_box, [b for _, b in old])
    clo, chi = _coarse_box(nlo, nhi)
    nfall = 0
    for st, (plo, phi), gc, dxc in coarse:
        lo = [max(clo[d], plo[d]) for d in range(3)]
        hi = [min(chi[d], phi[d]) for d in range(3)]
        if not all(lo[d] <= hi[d] for d in range(3)):
            continue
        pn = tuple(phi[d] - plo[d] + 1 for d in range(3))
        Pc = O.patch(st, pn, gc, dxc)
        nfall += O.prolong_new(Pc, plo, Pf, nlo, lo, hi, m, mlo, energy_mode)
    return nfall
