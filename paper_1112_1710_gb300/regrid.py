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


def flag(ctx, patches, theta: float, stream=None):
    """Error flags of the interiors of `patches` (Patch objects of one
    dtype) on the device (``mhd_flag_cells``): a list of uint8 tensors, one
    per patch, shaped (nz, ny, nx)."""
    import torch
    dev = patches[0].state.device
    total = sum(p.cells for p in patches)
    out = torch.empty(max(1, total), dtype=torch.uint8, device=dev)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    capi.mhd_flag_cells(ctx, [p.desc() for p in patches], theta, out.data_ptr(), s)
    res, o = [], 0
    for p in patches:
        nx, ny, nz = p.n
        res.append(out[o:o + p.cells].view(nz, ny, nx))
        o += p.cells
    return res


def _cbox(lo, hi):
    return np.asarray(lo) // 2, (np.asarray(hi) + 1) // 2 - 1


def transfer_items(new_boxes, old_boxes):
    """Copies of the previous iteration's data into the new patches
    (``mhd_transfer_copy`` items): per (new, old) pair the cells of the
    intersection of the interiors and, per axis, the faces common to both
    face sets."""
    out = []
    if not old_boxes:
        return out
    olo = np.array([b[0] for b in old_boxes], np.int64)
    ohi = np.array([b[1] for b in old_boxes], np.int64)
    for i, (nlo, nhi) in enumerate(new_boxes):
        lo = np.maximum(olo, nlo)
        hi = np.minimum(ohi, nhi)
        for kind in (-1, 0, 1, 2):
            h = hi.copy()
            if kind >= 0:
                h[:, kind] = np.minimum(ohi[:, kind], nhi[kind]) + 1
            for j in np.nonzero(np.all(lo <= h, axis=1))[0]:
                it = capi.mhd_transfer_item()
                it.src, it.dst, it.kind = int(j), int(i), kind
                it.box = capi.box(lo[j], h[j])
                out.append(it)
    return out


def transfer_mask(new_box, old_boxes):
    """The mask of ``mhd_prolong_new`` over the coarse footprint of a new
    patch: bit 0 where the coarse cell's children lie in an old interior,
    bit 1 + 2 a + s where its side-s axis-a face lies in an old face set.
    Returns (uint8 array (z, y, x), coarse lo)."""
    clo, chi = _cbox(*new_box)
    ext = chi - clo + 1
    I = [np.arange(clo[d], chi[d] + 1) for d in range(3)]
    m = np.zeros((ext[2], ext[1], ext[0]), np.uint8)
    for olo, ohi in old_boxes:
        ol, oh = _cbox(olo, ohi)
        inside = [(I[d] >= ol[d]) & (I[d] <= oh[d]) for d in range(3)]
        cell = inside[2][:, None, None] & inside[1][None, :, None] & inside[0][None, None, :]
        m |= cell.astype(np.uint8)
        for a in range(3):
            for s in (0, 1):
                f = I[a] + s
                ok = [inside[d] if d != a else (f >= ol[a]) & (f <= oh[a] + 1) for d in range(3)]
                face = ok[2][:, None, None] & ok[1][None, :, None] & ok[0][None, None, :]
                m |= (face.astype(np.uint8) << (1 + 2 * a + s)).astype(np.uint8)
    return m, tuple(int(v) for v in clo)


def transfer(ctx, old, fresh, coarse, energy_mode: int = 1, stream=None):
    """Fills the interiors of the new patches `fresh` (Patch objects of level
    l+1) from the previous iteration `old` (Patch objects of level l+1) and
    the level-l patches `coarse`: the copies first, then the prolongation of
    the rest under each new patch's mask.  Returns the device count of energy
    fallbacks (a one-element tensor)."""
    import torch
    dev = fresh[0].state.device
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    nb = [(p.lo, p.hi) for p in fresh]
    ob = [(p.lo, p.hi) for p in old]
    items = transfer_items(nb, ob)
    if items:
        capi.mhd_transfer_copy(ctx, [p.desc() for p in old], [p.desc() for p in fresh], items, s)
    masks, pitems = [], []
    clo_all = np.array([p.lo for p in coarse], np.int64)
    chi_all = np.array([p.hi for p in coarse], np.int64)
    for i, (lo, hi) in enumerate(nb):
        m, mlo = transfer_mask((lo, hi), ob)
        dm = torch.as_tensor(m, device=dev).contiguous()
        masks.append(dm)
        cl, ch = _cbox(lo, hi)
        blo = np.maximum(clo_all, cl)
        bhi = np.minimum(chi_all, ch)
        for k in np.nonzero(np.all(blo <= bhi, axis=1))[0]:
            it = capi.mhd_prolong_new_item()
            it.coarse, it.fine = int(k), i
            it.box = capi.box(blo[k], bhi[k])
            it.mask = dm.data_ptr()
            it.mask_box = capi.box(mlo, tuple(int(v) for v in ch))
            pitems.append(it)
    nfall = torch.zeros(1, dtype=torch.int64, device=dev)
    capi.mhd_prolong_new(ctx, [p.desc() for p in coarse], [p.desc() for p in fresh], pitems, energy_mode,
                         nfall.data_ptr(), s)
    transfer._keep = masks          # the masks must live until the launch has run
    return nfall
