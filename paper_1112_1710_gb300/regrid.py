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
    per patch, shaped (nz, ny, nx), written on `stream` (the current stream
    if None): synchronise with it before reading them elsewhere."""
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
    (``mhd_transfer_copy`` items, as one ctypes array; [] when there is
    none): per (new, old) pair the cells of the intersection of the
    interiors and, per axis, the faces common to both face sets; new patch
    by new patch, cells then the faces of each axis, old patches ascending."""
    if not old_boxes or not new_boxes:
        return []
    olo = np.array([b[0] for b in old_boxes], np.int64)
    ohi = np.array([b[1] for b in old_boxes], np.int64)
    rows = []
    for i, (nlo, nhi) in enumerate(new_boxes):
        lo = np.maximum(olo, nlo)
        hi = np.minimum(ohi, nhi)
        for kind in (-1, 0, 1, 2):
            h = hi.copy()
            if kind >= 0:
                h[:, kind] = np.minimum(ohi[:, kind], nhi[kind]) + 1
            js = np.nonzero(np.all(lo <= h, axis=1))[0]
            if len(js):
                r = np.zeros((len(js), 10), np.int32)   # src, dst, kind, pad, box lo, box hi
                r[:, 0] = js
                r[:, 1] = i
                r[:, 2] = kind
                r[:, 4:7] = lo[js]
                r[:, 7:10] = h[js]
                rows.append(r)
    if not rows:
        return []
    a = np.ascontiguousarray(np.concatenate(rows))
    return (capi.mhd_transfer_item * len(a)).from_buffer_copy(a)


# numpy layout of mhd_prolong_new_item (include/mhd_gpu.h)
_PNEW_DT = np.dtype({"names": ["coarse", "fine", "lo", "hi", "mask", "mlo", "mhi"],
                     "formats": ["<i4", "<i4", ("<i4", 3), ("<i4", 3), "<u8", ("<i4", 3), ("<i4", 3)],
                     "offsets": [0, 4, 8, 20, 32, 40, 52], "itemsize": 64})


def prolong_new_items(new_boxes, coarse_boxes, mask_los, mask_ptrs):
    """``mhd_prolong_new`` items (one ctypes array; [] when there is none):
    per new patch i (coarse footprint of new_boxes[i]) and every coarse
    patch k meeting it, the intersection, with the new patch's mask at
    device address mask_ptrs[i] over the box from mask_los[i] to the
    footprint's upper corner; new patches in order, coarse ones ascending."""
    if not new_boxes or not coarse_boxes:
        return []
    clo_all = np.array([b[0] for b in coarse_boxes], np.int64)
    chi_all = np.array([b[1] for b in coarse_boxes], np.int64)
    parts = []
    for i, (lo, hi) in enumerate(new_boxes):
        cl, ch = _cbox(lo, hi)
        blo = np.maximum(clo_all, cl)
        bhi = np.minimum(chi_all, ch)
        ks = np.nonzero(np.all(blo <= bhi, axis=1))[0]
        if not len(ks):
            continue
        r = np.zeros(len(ks), _PNEW_DT)
        r["coarse"] = ks
        r["fine"] = i
        r["lo"] = blo[ks]
        r["hi"] = bhi[ks]
        r["mask"] = mask_ptrs[i]
        r["mlo"] = mask_los[i]
        r["mhi"] = ch
        parts.append(r)
    if not parts:
        return []
    a = np.concatenate(parts)
    return (capi.mhd_prolong_new_item * len(a)).from_buffer_copy(a)


def transfer_mask(new_box, old_boxes):
    """The mask of ``mhd_prolong_new`` over the coarse footprint of a new
    patch: bit 0 where the coarse cell's children lie in an old interior,
    bit 1 + 2 a + s where its side-s axis-a face lies in an old face set.
    Returns (uint8 array (z, y, x), coarse lo)."""
    clo, chi = _cbox(*new_box)
    ext = chi - clo + 1
    I = [np.arange(clo[d], chi[d] + 1) for d in range(3)]
    m = np.zeros((ext[2], ext[1], ext[0]), np.uint8)
    if len(old_boxes):
        # only the old patches whose coarse footprint, grown by one face,
        # meets this one's contribute
        ol = np.array([b[0] for b in old_boxes], np.int64) // 2
        oh = (np.array([b[1] for b in old_boxes], np.int64) + 1) // 2 - 1
        near = np.all((ol <= chi + 1) & (oh + 1 >= clo), axis=1)
        old_boxes = [old_boxes[k] for k in np.nonzero(near)[0]]
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


def transfer_masks(new_boxes, old_boxes):
    """transfer_mask of every new patch at once: the old interiors and the
    old face sets are painted once over the coarse bounding box of the new
    patches (one array per mask bit's set), and each new patch's mask is
    read off them.  Returns [(uint8 array (z, y, x), coarse lo)]."""
    if not new_boxes:
        return []
    cb = [_cbox(lo, hi) for lo, hi in new_boxes]
    glo = np.min([c[0] for c in cb], axis=0)
    ghi = np.max([c[1] for c in cb], axis=0)
    ext = ghi - glo + 1
    cell = np.zeros((ext[2], ext[1], ext[0]), bool)
    face = []
    for a in range(3):
        e = ext.copy()
        e[a] += 1
        face.append(np.zeros((e[2], e[1], e[0]), bool))
    for olo, ohi in old_boxes:
        ol, oh = _cbox(olo, ohi)
        lo = np.maximum(ol, glo) - glo
        hi = np.minimum(oh, ghi) - glo
        if np.all(lo <= hi):
            cell[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
        for a in range(3):
            flo, fhi = lo.copy(), hi.copy()
            # faces ol_a .. oh_a + 1 along a, clipped to the painted range
            flo[a] = max(ol[a], glo[a]) - glo[a]
            fhi[a] = min(oh[a] + 1, ghi[a] + 1) - glo[a]
            if np.all(flo <= fhi):
                face[a][flo[2]:fhi[2] + 1, flo[1]:fhi[1] + 1, flo[0]:fhi[0] + 1] = True
    out = []
    for clo, chi in cb:
        l, h = clo - glo, chi - glo
        m = cell[l[2]:h[2] + 1, l[1]:h[1] + 1, l[0]:h[0] + 1].astype(np.uint8)
        for a in range(3):
            for sd in (0, 1):
                sh = [0, 0, 0]
                sh[a] = sd
                f = face[a][l[2] + sh[2]:h[2] + sh[2] + 1, l[1] + sh[1]:h[1] + sh[1] + 1,
                            l[0] + sh[0]:h[0] + sh[0] + 1]
                m |= (f.astype(np.uint8) << (1 + 2 * a + sd)).astype(np.uint8)
        out.append((m, tuple(int(v) for v in clo)))
    return out


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
    hm = transfer_masks(nb, ob)
    # all masks in one device buffer (one copy), each at a 16-byte offset
    offs, o = [], 0
    for m, _ in hm:
        offs.append(o)
        o += (m.size + 15) // 16 * 16
    buf = np.zeros(max(o, 16), np.uint8)
    for (m, _), off in zip(hm, offs):
        buf[off:off + m.size] = m.ravel()
    dm = torch.as_tensor(buf, device=dev)
    base = dm.data_ptr()
    pitems = prolong_new_items(nb, [(p.lo, p.hi) for p in coarse], [m[1] for m in hm],
                               [base + off for off in offs])
    masks = [dm]
    nfall = torch.zeros(1, dtype=torch.int64, device=dev)
    if stream is not None:
        # the masks and the count were written on the current stream
        stream.wait_stream(torch.cuda.current_stream(dev))
    capi.mhd_prolong_new(ctx, [p.desc() for p in coarse], [p.desc() for p in fresh], pitems, energy_mode,
                         nfall.data_ptr(), s)
    transfer._keep = masks          # the masks must live until the launch has run
    return nfall


def _grow(m, r: int, value: bool):
    """Separable dilation (value True) or erosion (value False) of a boolean
    array by the cube of half-width r, the outside counting as not set."""
    out = m
    for ax in range(m.ndim):
        pad = [(0, 0)] * m.ndim
        pad[ax] = (r, r)
        p = np.pad(out, pad, constant_values=False)
        acc = out.copy()
        for s in range(-r, r + 1):
            sl = [slice(None)] * m.ndim
            sl[ax] = slice(r + s, r + s + m.shape[ax])
            acc = (acc | p[tuple(sl)]) if value else (acc & p[tuple(sl)])
        out = acc
    return out


def fit_boxes(boxes, flags, allowed):
    """Cluster boxes (inclusive, array axis order) made to lie in `allowed`:
    each box is shrunk to the bounding box of its flagged cells; a box with a
    cell outside `allowed` is halved across its longest axis (the lower axis
    on ties; the low half takes the extra slice) and both halves treated
    again, low half first.  Every flagged cell must be allowed."""
    out = []

    def rec(lo, hi):
        sl = tuple(slice(lo[d], hi[d] + 1) for d in range(3))
        f = flags[sl]
        if not f.any():
            return
        nz = [np.nonzero(f.any(axis=tuple(e for e in range(3) if e != d)))[0] for d in range(3)]
        lo = tuple(lo[d] + int(nz[d][0]) for d in range(3))
        hi = tuple(lo[d] - int(nz[d][0]) + int(nz[d][-1]) for d in range(3))
        hi = tuple(int(v) for v in hi)
        sl = tuple(slice(lo[d], hi[d] + 1) for d in range(3))
        if allowed[sl].all():
            out.append((lo, hi))
            return
        ext = [hi[d] - lo[d] + 1 for d in range(3)]
        d = int(np.argmax(ext))
        mid = lo[d] + (ext[d] - 1) // 2
        a_hi, b_lo = list(hi), list(lo)
        a_hi[d], b_lo[d] = mid, mid + 1
        rec(lo, tuple(a_hi))
        rec(tuple(b_lo), hi)

    for lo, hi in boxes:
        rec(tuple(int(v) for v in lo), tuple(int(v) for v in hi))
    return out


def _next_level(h, old, theta, buffer, margin, eff, min_size, energy_mode, tm):
    """The next iteration of level h.nlev (whose previous iteration is the
    Patch list `old`) from the flags of h's finest level, which must hold
    its data (interiors; its ghost zones are filled here from the levels
    below, as at the start of its step).  Returns (boxes, patches, fallbacks);
    no boxes when nothing is flagged."""
    import time

    import torch

    from .patch import Patch, patch_shape
    t0 = time.perf_counter()
    lp = h.nlev - 1
    h.fill(0)
    for k in range(1, lp + 1):
        h.prolong(k - 1)
        h.fill(k)
    parents = h.levels[lp]
    cur = torch.cuda.current_stream(h.device)
    h.stream.wait_stream(cur)
    fl = flag(h.ctx, parents, theta, h.stream)
    h.stream.synchronize()
    t1 = time.perf_counter()
    tm["flags"] = tm.get("flags", 0.0) + t1 - t0
    # flags over the bounding box of the parent grids (x, y, z -> array z, y, x)
    blo = np.min([p.lo for p in parents], axis=0)
    bhi = np.max([p.hi for p in parents], axis=0)
    ext = bhi - blo + 1
    dense = np.zeros((ext[2], ext[1], ext[0]), dtype=bool)
    inside = np.zeros_like(dense)
    for p, f in zip(parents, fl):
        lo, hi = np.asarray(p.lo) - blo, np.asarray(p.hi) - blo
        dense[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] |= f.cpu().numpy().astype(bool)
        inside[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
    if buffer > 0:
        dense = _grow(dense, buffer, True)
    allowed = _grow(inside, margin, False)
    dense &= allowed
    t2 = time.perf_counter()
    tm["masks"] = tm.get("masks", 0.0) + t2 - t1
    if not dense.any():
        return [], [], torch.zeros(1, dtype=torch.int64, device=h.device)
    cl = cluster(dense.astype(np.uint8), eff, min_size)            # (z, y, x) order, box-local
    cl = fit_boxes(cl, dense, allowed)
    t3 = time.perf_counter()
    tm["clustering"] = tm.get("clustering", 0.0) + t3 - t2
    cl = [(tuple(int(v) for v in np.asarray(lo[::-1]) + blo), tuple(int(v) for v in np.asarray(hi[::-1]) + blo))
          for lo, hi in cl]
    new = children(cl, [(p.lo, p.hi) for p in parents])
    dx = tuple(v / 2 ** (lp + 1) for v in h.dx0)
    tdt = {"f32": torch.float32, "f64": torch.float64}[h.dtype]
    fresh = []
    for i, (lo, hi) in enumerate(new):
        nn = tuple(hi[d] - lo[d] + 1 for d in range(3))
        st = torch.zeros(patch_shape(nn, h.g), dtype=tdt, device=h.device)
        fresh.append(Patch(st, tuple(lo), nn, h.g, dx, lp + 1, i))
    h.stream.wait_stream(cur)               # the zeroed arrays
    nfall = transfer(h.ctx, old, fresh, parents, energy_mode, h.stream)
    cur.wait_stream(h.stream)
    h.stream.synchronize()
    tm["transfer"] = tm.get("transfer", 0.0) + time.perf_counter() - t3
    return [(tuple(lo), tuple(hi)) for lo, hi in new], fresh, nfall


def regrid_levels(h, theta: float, first: int | None = None, buffer: int = 1, margin: int = 3, eff: float = 0.7,
                  min_size: int = 2, energy_mode: int = 1, timing=None):
    """The next iteration of every level from `first` (default: the finest)
    to the finest (Sec. 2.1), coarsest first: each new level is made from the
    flags of the level below it in the new hierarchy (``mhd_flag_cells``,
    after that level's ghost zones are filled from the levels below), the
    flags grown by `buffer` cells and kept where the new level is properly
    nested (at least `margin` parent cells inside the parent level's grids;
    the domain boundary counts as outside), clustered into boxes
    (Berger-Rigoutsos), cut by the parent grids and refined; the new patches
    take the previous iteration of their level where they meet it and the
    new parent level's prolongation elsewhere (``mhd_transfer_copy``,
    ``mhd_prolong_new``).  A level with no flagged cell ends the hierarchy.
    Returns (boxes, states, fallbacks): every level's boxes and state tensors
    for a new Hierarchy (the kept levels' tensors are the hierarchy's own)
    and the device count of energy fallbacks.  `timing` (a dict, optional)
    receives the seconds of each phase (flags, masks, clustering, transfer,
    and the metadata of the intermediate hierarchies)."""
    import time

    import torch
    tm = timing if timing is not None else {}
    L = h.nlev
    first = L - 1 if first is None else first
    if L < 2 or not 1 <= first <= L - 1:
        raise ValueError("regridding needs levels 1 .. %d of a hierarchy of %d levels" % (L - 1, L))
    boxes = [[(p.lo, p.hi) for p in lv] for lv in h.levels[:first]]
    states = [[p.state for p in lv] for lv in h.levels[:first]]
    nfall = torch.zeros(1, dtype=torch.int64, device=h.device)
    tmp = None
    try:
        for m in range(first, L):
            if m == first:
                parent = _Prefix(h, m)          # h's own levels 0..m-1
            else:
                t0 = time.perf_counter()
                if tmp is not None:
                    tmp.close()
                tmp = type(h)(boxes, h.n0, states, h.dx0, g=h.g, dtype=h.dtype, ctx=h.ctx, stream=h.stream,
                              device=h.device)
                tm["metadata"] = tm.get("metadata", 0.0) + time.perf_counter() - t0
                parent = tmp
            nb, fresh, nf = _next_level(parent, h.levels[m], theta, buffer, margin, eff, min_size, energy_mode, tm)
            nfall += nf
            if not nb:
                break
            boxes.append(nb)
            states.append([p.state for p in fresh])
    finally:
        if tmp is not None:
            tmp.close()
    return boxes, states, nfall


class _Prefix:
    """Levels 0..m-1 of a hierarchy, with its operations (the parent levels
    of a regridding)."""

    def __init__(self, h, m):
        self._h, self.nlev = h, m
        self.levels = h.levels[:m]
        self.ctx, self.stream, self.device, self.dtype = h.ctx, h.stream, h.device, h.dtype
        self.g, self.n0, self.dx0 = h.g, h.n0, h.dx0

    def fill(self, l):
        self._h.fill(l)

    def prolong(self, l):
        self._h.prolong(l)


def regrid_finest(h, theta: float, **kw):
    """regrid_levels of the finest level alone."""
    return regrid_levels(h, theta, first=h.nlev - 1, **kw)
