"""Space-filling-curve ordering and Hilbert splitting of grids (Sec. 5.1,
5.2) through ``libmhdgpu.so``: ``mhd_hilbert_keys`` and ``mhd_box_distances``
on the device, ``mhd_hilbert_split`` on the host.

On one GPU the "processors" of Sec. 5 are the workers that take patches in
turn (the batched launches of a level, the serving slots); the curve orders
the patches of a level so that neighbours along the curve are neighbours in
space, and the splitting cuts a large grid into pieces of given shares.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import capi


def bits_for(extent: int) -> int:
    """Smallest b with 2^b >= extent (the curve resolution of a domain)."""
    b = 0
    while (1 << b) < extent:
        b += 1
    return b


def _stream(device):
    return torch.cuda.current_stream(device).cuda_stream


def keys(points: torch.Tensor, bits: int) -> torch.Tensor:
    """Hilbert indices (uint64 values in an int64 tensor) of the int32 device
    points [n, dim]; UINT64_MAX (-1 as int64) outside [0, 2^bits)^dim."""
    pts = points.to(torch.int32).contiguous()
    n, dim = pts.shape
    out = torch.empty(n, dtype=torch.int64, device=pts.device)
    r = capi.load().mhd_hilbert_keys(pts.data_ptr(), n, dim, bits, out.data_ptr(), _stream(pts.device))
    if r != capi.MHD_OK:
        raise capi.MHDError(r, "mhd_hilbert_keys")
    return out


def box_distances(lo: torch.Tensor, hi: torch.Tensor, bits: int) -> torch.Tensor:
    """Corner-sum distances along the curve of the inclusive int32 device
    boxes [n, dim]; INT64_MAX for empty boxes or boxes outside the curve."""
    lo = lo.to(torch.int32).contiguous()
    hi = hi.to(torch.int32).contiguous()
    n, dim = lo.shape
    out = torch.empty(n, dtype=torch.int64, device=lo.device)
    r = capi.load().mhd_box_distances(lo.data_ptr(), hi.data_ptr(), n, dim, bits, out.data_ptr(),
                                      _stream(lo.device))
    if r != capi.MHD_OK:
        raise capi.MHDError(r, "mhd_box_distances")
    return out


def order_boxes(boxes, bits: int, device="cuda") -> np.ndarray:
    """Indices of `boxes` ((lo, hi) pairs) in order of their distance along
    the curve, ties by position in the list (Sec. 5.1): distances on the
    device, the small sort of the patch list on the host."""
    if not boxes:
        return np.zeros(0, np.int64)
    lo = torch.tensor(np.array([b[0] for b in boxes], np.int32), device=device)
    hi = torch.tensor(np.array([b[1] for b in boxes], np.int32), device=device)
    d = box_distances(lo, hi, bits).cpu().numpy()
    return np.lexsort((np.arange(len(boxes)), d))


def split(lo, hi, weights, bits: int, ghost: int = 2):
    """Pieces [(lo, hi)] of the inclusive box [lo, hi], one per weight in
    weight order, by the recursive Hilbert bisection of Sec. 5.2."""
    dim = len(lo)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    k = len(w)
    a = np.ascontiguousarray(lo, dtype=np.int32)
    b = np.ascontiguousarray(hi, dtype=np.int32)
    olo = np.zeros((k, dim), np.int32)
    ohi = np.zeros((k, dim), np.int32)
    p = lambda x: x.ctypes.data_as(C.c_void_p)
    r = capi.load().mhd_hilbert_split(p(a), p(b), dim, p(w), k, bits, ghost, p(olo), p(ohi))
    if r != capi.MHD_OK:
        raise capi.MHDError(r, "mhd_hilbert_split")
    return [(tuple(int(v) for v in olo[i]), tuple(int(v) for v in ohi[i])) for i in range(k)]


def global_offsets(local_counts) -> np.ndarray:
    """Sec. 5.1: an item's global sort index is its local index plus the item
    counts of all lower-numbered holders; returns those offsets."""
    c = np.asarray(local_counts, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(c)[:-1]]) if len(c) else np.zeros(0, np.int64)


def hilbert_order_hierarchy(boxes, n0, device="cuda"):
    """Permutations ordering each level's patches along the curve of that
    level's periodic domain (n0 2^l cells a side): perm[l][k] is the old index
    of the k-th patch."""
    out = []
    for l, bl in enumerate(boxes):
        out.append(order_boxes(bl, bits_for(n0 << l), device=device))
    return out
