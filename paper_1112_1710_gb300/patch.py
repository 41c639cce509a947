"""Host-side patch descriptors, copy lists and update-box schedules.

A patch (the paper's grid, Sec. 2) is one torch tensor of shape
``(8, NZ+1, NY+1, PX)`` on the device: planes 0..4 hold rho, Mx, My, Mz, E at
cell centres and planes 5..7 hold Bx, By, Bz on the lower faces of each cell
(one extra entry along each normal).  ``N* = n* + 2g``; ``PX >= NX + 1``.
PyTorch only provides the memory; every operation on it runs in
``libmhdgpu.so`` through ``capi``.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import torch

from . import capi

DTYPES = {"f64": (torch.float64, capi.MHD_F64), "f32": (torch.float32, capi.MHD_F32)}


def patch_shape(n, g: int, align: int = 8):
    nx, ny, nz = (int(v) for v in n)
    NX, NY, NZ = nx + 2 * g, ny + 2 * g, nz + 2 * g
    px = -(-(NX + 1) // align) * align
    return (8, NZ + 1, NY + 1, px)


@dataclass
class Patch:
    state: torch.Tensor        # (8, NZ+1, NY+1, PX)
    lo: tuple                  # interior lower corner, level index space
    n: tuple                   # interior cells per axis
    g: int
    dx: tuple
    level: int = 0
    patch_id: int = 0

    @property
    def hi(self):
        return tuple(self.lo[d] + self.n[d] - 1 for d in range(3))

    @property
    def dtype_code(self) -> int:
        return capi.MHD_F64 if self.state.dtype == torch.float64 else capi.MHD_F32

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def desc(self) -> capi.mhd_patch_desc:
        st = self.state
        if not st.is_cuda or not st.is_contiguous():
            raise ValueError("patch state must be a contiguous CUDA tensor")
        d = capi.mhd_patch_desc()
        d.level = self.level
        d.nghost = self.g
        d.dtype = self.dtype_code
        d.patch_id = self.patch_id
        d.interior.lo[:] = tuple(int(v) for v in self.lo)
        d.interior.hi[:] = tuple(int(v) for v in self.hi)
        base = st.data_ptr()
        plane = st.stride(0) * st.element_size()
        for q in range(5):
            d.U[q] = base + q * plane
        for a in range(3):
            d.B[a] = base + (5 + a) * plane
        d.stride[:] = (1, st.stride(2), st.stride(1))
        d.dx[:] = tuple(float(v) for v in self.dx)
        return d

    @staticmethod
    def from_array(arr, lo, n, g, dx, dtype="f64", device="cuda", level=0, patch_id=0) -> "Patch":
        tdt, _ = DTYPES[dtype]
        t = torch.as_tensor(arr).to(device=device, dtype=tdt).contiguous()
        if tuple(t.shape[:3]) != patch_shape(n, g)[:3] or t.shape[3] < n[0] + 2 * g + 1:
            raise ValueError("array shape %s does not match n=%s g=%d" % (tuple(t.shape), n, g))
        return Patch(t, tuple(lo), tuple(n), g, tuple(dx), level, patch_id)


def periodic_copies(n, g: int, lo=(0, 0, 0), index: int = 0):
    """Ghost-fill copies of one patch that covers a periodic domain: every
    periodic image of the interior, clipped to the ghost-extended box grown by
    one cell (the outer layer carries the faces on the outer planes of the face
    arrays), as a box with its image offset (up to ceil((g+1)/n) periods, so a
    patch thinner than its ghost width works)."""
    out = []
    reach = [(g + int(n[d])) // int(n[d]) for d in range(3)]
    ranges = [range(-reach[d], reach[d] + 1) for d in range(3)]
    for o in itertools.product(*ranges):
        if o == (0, 0, 0):
            continue
        blo, bhi = [], []
        ok = True
        for d in range(3):
            a = lo[d] + o[d] * n[d]
            b = a + n[d] - 1
            a2, b2 = max(a, lo[d] - g - 1), min(b, lo[d] + n[d] + g)
            if a2 > b2:
                ok = False
                break
            blo.append(a2)
            bhi.append(b2)
        if not ok:
            continue
        c = capi.mhd_copy()
        c.src = index
        c.dst = index
        c.box.lo[:] = blo
        c.box.hi[:] = bhi
        c.offset[:] = tuple(-o[d] * n[d] for d in range(3))
        out.append(c)
    return out


def update_box_schedule(n, R: int, n_ghost: int):
    """Update boxes of the R substeps of an isolated patch with extended ghost
    zones (Sec. 2.3, Sec. 4): substep i (1-based) updates the interior grown by
    n_ghost * (R - i) layers.  Returns [(grow, cells updated), ...]."""
    out = []
    for i in range(1, R + 1):
        k = n_ghost * (R - i)
        cells = 1
        for v in n:
            cells *= int(v) + 2 * k
        out.append((k, cells))
    return out
