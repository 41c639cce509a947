"""Thin ctypes binding of ``include/mhd_gpu.h`` (``libmhdgpu.so``).

Argument marshalling only: every step of the patch advance runs in the CUDA
library.  Functions keep the C names (``mhd_patch_advance`` ...) and raise
``MHDError`` on a negative status.  There is no CPU fallback: importing this
module without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_ENEGATIVE, MHD_ETIMEOUT = 0, -1, -2, -3, -4, -5
MHD_ETOOBIG = -6
MHD_F64, MHD_F32 = 0, 1
STATUS_NAMES = {0: "MHD_OK", -1: "MHD_EINVAL", -2: "MHD_ENOMEM", -3: "MHD_ECUDA",
                -4: "MHD_ENEGATIVE", -5: "MHD_ETIMEOUT", -6: "MHD_ETOOBIG"}

# Exported functions of include/mhd_gpu.h (checked against the header by the tests).
EXPORTS = ("mhd_ctx_create", "mhd_ctx_destroy", "mhd_last_error", "mhd_cfl_dt", "mhd_patch_advance",
           "mhd_ghost_fill", "mhd_conservation_sums", "mhd_get_device_status", "mhd_version",
           "mhd_launch_count", "mhd_timing_enable", "mhd_timing_read", "mhd_timing_reset",
           "mhd_kernel_name", "mhd_conservation_sums_static", "mhd_prolong", "mhd_restrict", "mhd_reflux",
           "mhd_restrict_prolong", "mhd_autotune_advance", "mhd_tree_parents", "mhd_tree_inherit",
           "mhd_ctx_clone", "mhd_hilbert_keys", "mhd_box_distances", "mhd_hilbert_split",
           "mhd_patch_step_cfl", "mhd_cluster_flags", "mhd_alu_probe", "mhd_fluxreg_create",
           "mhd_fluxreg_destroy", "mhd_fluxreg_face", "mhd_fluxreg_edge", "mhd_fluxreg_zero", "mhd_flag_cells",
           "mhd_transfer_copy", "mhd_prolong_new", "mhd_floor_count", "mhd_floor")
N_KERNELS = 16
MHD_CAP_FACE, MHD_CAP_EDGE = 0, 1
MHD_PROLONG, MHD_RESTRICT = 0, 1
MHD_REFLUX, MHD_SYNC = 0, 1


class MHDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class mhd_box(C.Structure):
    _fields_ = [("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3)]


class mhd_patch_desc(C.Structure):
    _fields_ = [("level", C.c_int32), ("nghost", C.c_int32), ("dtype", C.c_int32),
                ("patch_id", C.c_int32), ("interior", mhd_box), ("U", C.c_void_p * 5),
                ("B", C.c_void_p * 3), ("stride", C.c_int64 * 3), ("dx", C.c_double * 3)]


class mhd_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("limiter", C.c_int32),
                ("emf", C.c_int32), ("upwind_eps", C.c_double), ("fp64_contract", C.c_int32),
                ("advance_kernel", C.c_int32), ("fused_chunk", C.c_int32), ("kernel_shape", C.c_int32),
                ("p_floor", C.c_double), ("rho_floor", C.c_double)]


class mhd_copy(C.Structure):
    _fields_ = [("src", C.c_int32), ("dst", C.c_int32), ("box", mhd_box), ("offset", C.c_int32 * 3)]


class mhd_prolong_item(C.Structure):
    _fields_ = [("coarse", C.c_int32), ("fine", C.c_int32), ("box", mhd_box)]


class mhd_level_item(C.Structure):
    _fields_ = [("fine", C.c_int32), ("coarse", C.c_int32), ("box", mhd_box)]


class mhd_restrict_item(C.Structure):
    _fields_ = [("fine", C.c_int32), ("coarse", C.c_int32), ("box", mhd_box)]


class mhd_capture(C.Structure):
    _fields_ = [("patch", C.c_int32), ("kind", C.c_int32), ("axis", C.c_int32), ("mode", C.c_int32),
                ("box", mhd_box), ("dst", C.c_void_p)]


class mhd_transfer_item(C.Structure):
    _fields_ = [("src", C.c_int32), ("dst", C.c_int32), ("kind", C.c_int32), ("pad", C.c_int32), ("box", mhd_box)]


class mhd_prolong_new_item(C.Structure):
    _fields_ = [("coarse", C.c_int32), ("fine", C.c_int32), ("box", mhd_box), ("mask", C.c_void_p),
                ("mask_box", mhd_box)]


class mhd_deposit(C.Structure):
    _fields_ = [("coarse", C.c_int32), ("kind", C.c_int32), ("axis", C.c_int32), ("mode", C.c_int32),
                ("box", mhd_box), ("fine_box", mhd_box), ("fine", C.c_void_p), ("coarse_reg", C.c_void_p)]


def box(lo, hi) -> mhd_box:
    b = mhd_box()
    b.lo[:] = tuple(int(v) for v in lo)
    b.hi[:] = tuple(int(v) for v in hi)
    return b


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libmhdgpu.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError("libmhdgpu.so is not built: run __graft_entry__.build() "
                              "(nvcc for sm_103a); there is no CPU fallback")
        _build.build()
    L = C.CDLL(_build.LIB)
    P = C.c_void_p
    i32, i64 = C.c_int32, C.c_int64
    dp = C.POINTER(C.c_double)
    L.mhd_ctx_create.restype = i32
    L.mhd_ctx_create.argtypes = [C.POINTER(mhd_params), i32, C.POINTER(P)]
    L.mhd_ctx_clone.restype = i32
    L.mhd_ctx_clone.argtypes = [P, C.POINTER(P)]
    L.mhd_ctx_destroy.restype = None
    L.mhd_ctx_destroy.argtypes = [P]
    L.mhd_last_error.restype = C.c_char_p
    L.mhd_last_error.argtypes = [P]
    L.mhd_cfl_dt.restype = i32
    L.mhd_cfl_dt.argtypes = [P, C.POINTER(mhd_patch_desc), i32, dp, P, P]
    L.mhd_patch_advance.restype = i32
    L.mhd_patch_advance.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(i32), P, dp,
                                    C.POINTER(mhd_capture), i32, P]
    L.mhd_prolong.restype = i32
    L.mhd_prolong.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_patch_desc), i32,
                              C.POINTER(mhd_prolong_item), i32, P]
    L.mhd_restrict.restype = i32
    L.mhd_restrict.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_patch_desc), i32,
                               C.POINTER(mhd_restrict_item), i32, P]
    L.mhd_restrict_prolong.restype = i32
    L.mhd_restrict_prolong.argtypes = [P, i32, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_patch_desc), i32,
                                       C.POINTER(mhd_level_item), i32, P]
    L.mhd_autotune_advance.restype = i32
    L.mhd_autotune_advance.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(i32), C.POINTER(mhd_capture),
                                     i32, P, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_float), P]
    L.mhd_reflux.restype = i32
    L.mhd_reflux.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(C.c_void_p),
                             C.POINTER(mhd_deposit), i32, P]
    L.mhd_ghost_fill.restype = i32
    L.mhd_ghost_fill.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_copy), i32, P]
    L.mhd_conservation_sums.restype = i32
    L.mhd_conservation_sums.argtypes = [P, C.POINTER(mhd_patch_desc), i32, P, P]
    L.mhd_get_device_status.restype = i32
    L.mhd_get_device_status.argtypes = [P, C.POINTER(i32)]
    L.mhd_version.restype = C.c_char_p
    L.mhd_version.argtypes = []
    L.mhd_launch_count.restype = i64
    L.mhd_launch_count.argtypes = [P]
    L.mhd_timing_enable.restype = i32
    L.mhd_timing_enable.argtypes = [P, i32]
    L.mhd_timing_read.restype = i32
    L.mhd_timing_read.argtypes = [P, i32, dp, C.POINTER(i64)]
    L.mhd_timing_reset.restype = i32
    L.mhd_timing_reset.argtypes = [P]
    L.mhd_kernel_name.restype = C.c_char_p
    L.mhd_kernel_name.argtypes = [i32]
    L.mhd_conservation_sums_static.restype = i32
    L.mhd_conservation_sums_static.argtypes = [C.POINTER(mhd_patch_desc), i32, P, P]
    L.mhd_tree_parents.restype = i32
    L.mhd_tree_parents.argtypes = [P, P, i32, P, P, i32, P, P, P, P]
    L.mhd_tree_inherit.restype = i32
    L.mhd_tree_inherit.argtypes = [P, P, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P]
    L.mhd_patch_step_cfl.restype = i32
    L.mhd_patch_step_cfl.argtypes = [P, C.POINTER(mhd_patch_desc), i32, P, P]
    L.mhd_cluster_flags.restype = i32
    L.mhd_cluster_flags.argtypes = [P, i32, P, C.c_double, i32, i32, P, P, P]
    L.mhd_hilbert_keys.restype = i32
    L.mhd_hilbert_keys.argtypes = [P, i64, i32, i32, P, P]
    L.mhd_box_distances.restype = i32
    L.mhd_box_distances.argtypes = [P, P, i64, i32, i32, P, P]
    L.mhd_hilbert_split.restype = i32
    L.mhd_hilbert_split.argtypes = [P, P, i32, P, i32, i32, i32, P, P]
    L.mhd_alu_probe.restype = i32
    L.mhd_alu_probe.argtypes = [i32, i32, dp, dp]
    L.mhd_fluxreg_create.restype = i32
    L.mhd_fluxreg_create.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(P)]
    L.mhd_fluxreg_destroy.restype = None
    L.mhd_fluxreg_destroy.argtypes = [P]
    L.mhd_fluxreg_face.restype = P
    L.mhd_fluxreg_face.argtypes = [P, i32, i32, i32, C.POINTER(mhd_box)]
    L.mhd_fluxreg_edge.restype = P
    L.mhd_fluxreg_edge.argtypes = [P, i32, i32, i32, i32, C.POINTER(mhd_box)]
    L.mhd_floor.restype = i32
    L.mhd_floor.argtypes = [P, C.POINTER(mhd_patch_desc), i32, P]
    L.mhd_floor_count.restype = i32
    L.mhd_floor_count.argtypes = [P, C.POINTER(i64)]
    L.mhd_transfer_copy.restype = i32
    L.mhd_transfer_copy.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_patch_desc), i32,
                                    C.POINTER(mhd_transfer_item), i32, P]
    L.mhd_prolong_new.restype = i32
    L.mhd_prolong_new.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.POINTER(mhd_patch_desc), i32,
                                  C.POINTER(mhd_prolong_new_item), i32, i32, P, P]
    L.mhd_flag_cells.restype = i32
    L.mhd_flag_cells.argtypes = [P, C.POINTER(mhd_patch_desc), i32, C.c_double, P, P]
    L.mhd_fluxreg_zero.restype = i32
    L.mhd_fluxreg_zero.argtypes = [P, P]
    _lib = L
    return L


def _check(ctx, r):
    if r != MHD_OK:
        msg = load().mhd_last_error(ctx).decode() if ctx else ""
        raise MHDError(r, msg)


def _arr(ctype, seq):
    seq = list(seq)
    a = (ctype * max(1, len(seq)))()
    for i, v in enumerate(seq):
        a[i] = v
    return a


def _descs(patches):
    ds = list(patches)
    arr = (mhd_patch_desc * max(1, len(ds)))(*ds)
    return arr, len(ds)


# ------------------------------------------------------------------ C names
def mhd_ctx_create(gamma=5.0 / 3.0, cfl=0.4, limiter=0, emf=0, upwind_eps=0.0, device=0, fp64_contract=0,
                   advance_kernel=0, fused_chunk=0, p_floor=0.0, rho_floor=0.0, kernel_shape=0):
    prm = mhd_params(gamma, cfl, limiter, emf, upwind_eps, fp64_contract, advance_kernel, fused_chunk, kernel_shape,
                     float(p_floor), float(rho_floor))
    out = C.c_void_p()
    r = load().mhd_ctx_create(C.byref(prm), device, C.byref(out))
    _check(None, r)
    return out.value


def mhd_ctx_clone(ctx):
    out = C.c_void_p()
    _check(ctx, load().mhd_ctx_clone(ctx, C.byref(out)))
    return out.value


def mhd_ctx_destroy(ctx) -> None:
    load().mhd_ctx_destroy(ctx)


def mhd_last_error(ctx) -> str:
    return load().mhd_last_error(ctx).decode()


def mhd_version() -> str:
    return load().mhd_version().decode()


def mhd_launch_count(ctx) -> int:
    return int(load().mhd_launch_count(ctx))


def mhd_cfl_dt(ctx, patches, d_dt_out: int, stream: int = 0, scale=None) -> None:
    arr, n = _descs(patches)
    sc = _arr(C.c_double, scale) if scale is not None else None
    _check(ctx, load().mhd_cfl_dt(ctx, arr, n, sc, d_dt_out, stream))


def _structs(ctype, items):
    if isinstance(items, C.Array) and items._type_ is ctype:
        return items, len(items)
    items = list(items)
    return (ctype * max(1, len(items)))(*items), len(items)


def mhd_patch_advance(ctx, patches, d_dt: int, stream: int = 0, grow=None, dt_scale=None, caps=None) -> None:
    arr, n = _descs(patches)
    gr = _arr(C.c_int32, grow) if grow is not None else None
    sc = _arr(C.c_double, dt_scale) if dt_scale is not None else None
    if caps is None:
        ca, nca = None, 0
    elif isinstance(caps, tuple):  # (prebuilt ctypes array, count)
        ca, nca = caps
    else:
        ca, nca = _structs(mhd_capture, caps)
    _check(ctx, load().mhd_patch_advance(ctx, arr, n, gr, d_dt, sc, ca, nca, stream))


def mhd_patch_step_cfl(ctx, patches, d_dt_out: int, stream: int = 0) -> None:
    arr, n = _descs(patches)
    _check(ctx, load().mhd_patch_step_cfl(ctx, arr, n, d_dt_out, stream))


def mhd_prolong(ctx, coarse, fine, items, stream: int = 0) -> None:
    ca, nc = _descs(coarse)
    fa, nf = _descs(fine)
    it, ni = items if isinstance(items, tuple) else _structs(mhd_prolong_item, items)
    _check(ctx, load().mhd_prolong(ctx, ca, nc, fa, nf, it, ni, stream))


def mhd_restrict(ctx, fine, coarse, items, stream: int = 0) -> None:
    fa, nf = _descs(fine)
    ca, nc = _descs(coarse)
    it, ni = items if isinstance(items, tuple) else _structs(mhd_restrict_item, items)
    _check(ctx, load().mhd_restrict(ctx, fa, nf, ca, nc, it, ni, stream))


def mhd_restrict_prolong(ctx, mode, fine, coarse, items, stream: int = 0) -> None:
    fa, nf = _descs(fine)
    ca, nc = _descs(coarse)
    it, ni = items if isinstance(items, tuple) else _structs(mhd_level_item, items)
    _check(ctx, load().mhd_restrict_prolong(ctx, mode, fa, nf, ca, nc, it, ni, stream))


def mhd_autotune_advance(ctx, patches, d_dt: int, reps: int = 3, grow=None, stream: int = 0, caps=None):
    """Returns (choice, chunk, ms per advance): choice -3 - s = the fused pass
    in shape s, -2 / -1 = the staged kernels with the untiled / tiled
    predictor, s >= 0 = the fused kernel in shape s."""
    arr, n = _descs(patches)
    gr = _arr(C.c_int32, grow) if grow is not None else None
    if caps is None:
        ca, nca = None, 0
    elif isinstance(caps, tuple):  # (prebuilt ctypes array, count)
        ca, nca = caps
    else:
        ca, nca = _structs(mhd_capture, caps)
    v, cz, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(ctx, load().mhd_autotune_advance(ctx, arr, n, gr, ca, nca, d_dt, reps, C.byref(v), C.byref(cz),
                                            C.byref(ms), stream))
    return int(v.value), int(cz.value), float(ms.value)


def mhd_reflux(ctx, coarse, corr_ptrs, deposits, stream: int = 0) -> None:
    ca, nc = _descs(coarse)
    cp = (C.c_void_p * max(1, nc))(*[p or None for p in corr_ptrs])
    dp_, nd = deposits if isinstance(deposits, tuple) else _structs(mhd_deposit, deposits)
    _check(ctx, load().mhd_reflux(ctx, ca, nc, cp, dp_, nd, stream))


def mhd_flag_cells(ctx, patches, theta: float, d_flags: int, stream: int = 0) -> None:
    arr, n = _descs(patches)
    _check(ctx, load().mhd_flag_cells(ctx, arr, n, float(theta), d_flags, stream))


def mhd_floor(ctx, patches, stream: int = 0) -> None:
    arr, n = _descs(patches)
    _check(ctx, load().mhd_floor(ctx, arr, n, stream))


def mhd_floor_count(ctx) -> int:
    """Cells the pressure floor raised since the last call (synchronises)."""
    v = C.c_int64()
    _check(ctx, load().mhd_floor_count(ctx, C.byref(v)))
    return int(v.value)


def mhd_transfer_copy(ctx, old, fresh, items, stream: int = 0) -> None:
    oa, no = _descs(old)
    na, nn = _descs(fresh)
    ia, ni = _structs(mhd_transfer_item, items)
    _check(ctx, load().mhd_transfer_copy(ctx, oa, no, na, nn, ia, ni, stream))


def mhd_prolong_new(ctx, coarse, fine, items, energy_mode: int = 1, d_fallbacks: int = 0, stream: int = 0) -> None:
    ca, nc = _descs(coarse)
    fa, nf = _descs(fine)
    ia, ni = _structs(mhd_prolong_new_item, items)
    _check(ctx, load().mhd_prolong_new(ctx, ca, nc, fa, nf, ia, ni, int(energy_mode), d_fallbacks or None, stream))


def mhd_fluxreg_create(ctx, patches):
    """Library-owned FP64 boundary registers of `patches` (opaque handle)."""
    arr, n = _descs(patches)
    out = C.c_void_p()
    _check(ctx, load().mhd_fluxreg_create(ctx, arr, n, C.byref(out)))
    return out.value


def mhd_fluxreg_destroy(reg) -> None:
    load().mhd_fluxreg_destroy(reg)


def mhd_fluxreg_face(reg, patch: int, axis: int, side: int):
    """(device pointer, (lo, hi)) of a patch's boundary-face register."""
    b = mhd_box()
    ptr = load().mhd_fluxreg_face(reg, patch, axis, side, C.byref(b))
    if not ptr:
        raise MHDError(-1, "mhd_fluxreg_face: bad index")
    return ptr, (tuple(b.lo), tuple(b.hi))


def mhd_fluxreg_edge(reg, patch: int, face_axis: int, side: int, edge_axis: int):
    """(device pointer, (lo, hi)) of the register of a patch's axis-edge_axis
    edges in its boundary face (face_axis, side)."""
    b = mhd_box()
    ptr = load().mhd_fluxreg_edge(reg, patch, face_axis, side, edge_axis, C.byref(b))
    if not ptr:
        raise MHDError(-1, "mhd_fluxreg_edge: bad index")
    return ptr, (tuple(b.lo), tuple(b.hi))


def mhd_fluxreg_zero(reg, stream: int = 0) -> None:
    r = load().mhd_fluxreg_zero(reg, stream)
    if r != 0:
        raise MHDError(r, "mhd_fluxreg_zero failed")


def mhd_ghost_fill(ctx, patches, copies, stream: int = 0) -> None:
    arr, n = _descs(patches)
    carr, nc = copies if isinstance(copies, tuple) else _structs(mhd_copy, copies)
    _check(ctx, load().mhd_ghost_fill(ctx, arr, n, carr, nc, stream))


def mhd_conservation_sums(ctx, patches, d_out8: int, stream: int = 0) -> None:
    arr, n = _descs(patches)
    _check(ctx, load().mhd_conservation_sums(ctx, arr, n, d_out8, stream))


def mhd_conservation_sums_static(patches, d_out8: int, stream: int = 0) -> None:
    """Allocation-free conservation sums (no context; fixed capacity)."""
    arr, n = _descs(patches)
    r = load().mhd_conservation_sums_static(arr, n, d_out8, stream)
    if r != MHD_OK:
        raise MHDError(r, "mhd_conservation_sums_static rejected the request")


def mhd_get_device_status(ctx) -> int:
    v = C.c_int32(0)
    _check(ctx, load().mhd_get_device_status(ctx, C.byref(v)))
    return int(v.value)


def mhd_alu_probe(dtype: str = "f32", iters: int = 4096) -> tuple:
    """Measured FMA rate of the current device: (TFLOP/s, ms of the timed launch)."""
    t, ms = C.c_double(), C.c_double()
    r = load().mhd_alu_probe(0 if dtype == "f64" else 1, int(iters), C.byref(t), C.byref(ms))
    if r != 0:
        raise MHDError(r, "mhd_alu_probe failed")
    return t.value, ms.value


def mhd_timing_enable(ctx, on: bool = True) -> None:
    _check(ctx, load().mhd_timing_enable(ctx, 1 if on else 0))


def mhd_timing_reset(ctx) -> None:
    _check(ctx, load().mhd_timing_reset(ctx))


def mhd_kernel_name(kernel: int) -> str:
    return load().mhd_kernel_name(kernel).decode()


def mhd_timing_read(ctx) -> dict:
    """{kernel name: (total ms, launches)} since the last reset."""
    out = {}
    for k in range(N_KERNELS):
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        _check(ctx, load().mhd_timing_read(ctx, k, C.byref(ms), C.byref(n)))
        out[mhd_kernel_name(k)] = (float(ms.value), int(n.value))
    return out

