"""Grid generation for regridding (Sec. 2.1) through ``libmhdgpu.so``: the
boxes covering a level's flagged cells (``mhd_cluster_flags``, the
Berger-Rigoutsos point clustering on the host), and the overlap lists by
which a new iteration of a level takes the previous iteration's data where
they meet (Sec. 2.1 overlaps, the O of the grid life cycle).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi


def cluster(flags, eff: float = 0.7, min_size: int = 2):
    """Boxes [(lo, hi)] (inclusive, axis order of `flags`) covering the
    nonzero cells of the 2-D or 3-D array `flags`."""
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    dim = f.ndim
    shape = np.array(f.shape, np.int32)
    cap = max(16, int(f.sum()))
    lo = np.zeros((cap, dim), np.int32)
    hi = np.zeros((cap, dim), np.int32)
    n = C.c_int32(0)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    r = capi.load().mhd_cluster_flags(p(f), dim, p(shape), float(eff), int(min_size), cap, p(lo), p(hi),
                                      C.byref(n))
    if r != capi.MHD_OK:
        raise capi.MHDError(r, "mhd_cluster_flags")
    return [(tuple(int(v) for v in lo[k]), tuple(int(v) for v in hi[k])) for k in range(n.value)]


def overlaps(new_boxes, old_boxes, grow: int = 0):
    """(new, old, (lo, hi)) for every box of the previous iteration meeting a
    new box grown by `grow` cells, with their intersection."""
    out = []
    if not new_boxes or not old_boxes:
        return out
    olo = np.array([b[0] for b in old_boxes], np.int64)
    ohi = np.array([b[1] for b in old_boxes], np.int64)
    for i, (nlo, nhi) in enumerate(new_boxes):
        lo = np.maximum(olo, np.array(nlo) - grow)
        hi = np.minimum(ohi, np.array(nhi) + grow)
        for j in np.nonzero(np.all(lo <= hi, axis=1))[0]:
            out.append((i, int(j), (tuple(int(v) for v in lo[j]), tuple(int(v) for v in hi[j]))))
    return out


def children(cluster_boxes, coarse_boxes, ratio: int = 2):
    """Level-(l+1) boxes from level-l cluster boxes: each cluster box cut by
    every level-l grid it meets, so that each child lies inside one parent
    grid (Sec. 2: grids are nested in a coarser parent), then refined by
    `ratio`.  With disjoint cluster boxes and disjoint level-l grids the
    children are disjoint; they come in (cluster box, grid) order."""
    out = []
    for clo, chi in cluster_boxes:
        for plo, phi in coarse_boxes:
            lo = [max(clo[d], plo[d]) for d in range(len(clo))]
            hi = [min(chi[d], phi[d]) for d in range(len(clo))]
            if all(lo[d] <= hi[d] for d in range(len(lo))):
                out.append((tuple(ratio * v for v in lo), tuple(ratio * v + ratio - 1 for v in hi)))
    return out
