"""ctypes front end of the FP64 CPU oracle (``mhd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the bench's ``cpu_baseline`` / ``--impl reference`` leg, never by the product
package.  It shares no code with the CUDA path.

A patch is a float64 numpy array of shape ``(8, NZ+1, NY+1, PX)`` (the layout
``synth.patch_shape`` makes): planes 0..4 are rho, Mx, My, Mz, E at cell
centres, planes 5..7 are Bx, By, Bz on their faces.  Cell ``(i, j, k)`` (array
indices, ghosts included) is element ``[q, k, j, i]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Patch(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("g", C.c_int32), ("s", C.c_int64 * 3),
                ("dx", C.c_double * 3), ("U", C.c_void_p * 5), ("B", C.c_void_p * 3)]


class _Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("limiter", C.c_int32),
                ("emf", C.c_int32), ("upwind_eps", C.c_double), ("p_floor", C.c_double),
                ("rho_floor", C.c_double)]


class _Capture(C.Structure):
    _fields_ = [("d", C.c_int32), ("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3),
                ("mode", C.c_int32), ("dst", C.c_void_p)]


def bind(L):
    """Declares the C signatures of the oracle's exports on a loaded library."""
    dp = C.POINTER(C.c_double)
    L.orc_limiter.restype = C.c_double
    L.orc_limiter.argtypes = [C.c_int32, C.c_double, C.c_double]
    L.orc_fast_speed.restype = C.c_double
    L.orc_fast_speed.argtypes = [C.c_double] * 6
    L.orc_flux.restype = None
    L.orc_flux.argtypes = [C.c_int32, dp, C.c_double, dp]
    L.orc_hlld.restype = None
    L.orc_hlld.argtypes = [C.c_int32, dp, dp, C.c_double, C.c_double, C.c_double, dp, dp]
    L.orc_hlld_fan.restype = None
    L.orc_hlld_fan.argtypes = [C.c_int32, dp, dp, C.c_double, C.c_double, dp, dp, dp]
    L.orc_fill_periodic.restype = None
    L.orc_fill_periodic.argtypes = [C.POINTER(_Patch)]
    L.orc_cfl_dt.restype = C.c_double
    L.orc_cfl_dt.argtypes = [C.POINTER(_Patch), C.POINTER(_Params)]
    L.orc_advance.restype = C.c_int64
    L.orc_advance.argtypes = [C.POINTER(_Patch), C.POINTER(_Params), C.c_double,
                              C.c_int32, C.POINTER(_Capture), C.c_int32,
                              C.POINTER(_Capture), C.c_int32]
    L.orc_sums.restype = None
    L.orc_sums.argtypes = [C.POINTER(_Patch), dp]
    L.orc_divb_max.restype = C.c_double
    L.orc_divb_max.argtypes = [C.POINTER(_Patch)]
    i3 = C.POINTER(C.c_int32)
    pp = C.POINTER(C.c_void_p)
    L.orc_prolong.restype = None
    L.orc_prolong.argtypes = [C.POINTER(_Patch), i3, C.POINTER(_Patch), i3, i3, i3]
    L.orc_restrict.restype = None
    L.orc_restrict.argtypes = [C.POINTER(_Patch), i3, C.POINTER(_Patch), i3, i3, i3, C.c_int32]
    for nm in ("orc_deposit_faces", "orc_deposit_edges"):
        f = getattr(L, nm)
        f.restype = None
        f.argtypes = [C.POINTER(_Patch), i3, pp, C.c_int32, i3, i3, dp, i3, i3, dp]
    for nm in ("orc_sync_faces", "orc_sync_edges"):
        f = getattr(L, nm)
        f.restype = None
        f.argtypes = [C.POINTER(_Patch), i3, pp, C.c_int32, i3, i3, dp, dp]
    L.orc_floor.restype = C.c_int64
    L.orc_floor.argtypes = [C.POINTER(_Patch), C.POINTER(_Params)]
    L.orc_floor_count.restype = C.c_int64
    L.orc_floor_count.argtypes = []
    L.orc_set_threads.restype = None
    L.orc_set_threads.argtypes = [C.c_int32]
    L.orc_get_threads.restype = C.c_int32
    L.orc_get_threads.argtypes = []
    L.orc_transfer_copy.restype = None
    L.orc_transfer_copy.argtypes = [C.POINTER(_Patch), i3, C.POINTER(_Patch), i3, C.c_int32, i3, i3]
    L.orc_prolong_new.restype = C.c_int64
    L.orc_prolong_new.argtypes = [C.POINTER(_Patch), i3, C.POINTER(_Patch), i3, i3, i3, C.c_void_p, i3, i3,
                                  C.c_int32]
    L.orc_flag.restype = C.c_int64
    L.orc_flag.argtypes = [C.POINTER(_Patch), C.POINTER(_Params), C.c_double, C.c_void_p]
    L.orc_correct.restype = None
    L.orc_correct.argtypes = [C.POINTER(_Patch), pp]
    L.orc_copy.restype = None
    L.orc_copy.argtypes = [C.POINTER(_Patch), i3, C.POINTER(_Patch), i3, i3, i3, i3, C.c_int32]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(C.CDLL(_LIB))
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


UPWIND_EPS = 1e-10


def params(gamma=5.0 / 3.0, cfl=0.4, limiter=0, emf=0, upwind_eps=UPWIND_EPS, p_floor=0.0,
           rho_floor=0.0) -> _Params:
    return _Params(gamma, cfl, limiter, emf, upwind_eps, p_floor, rho_floor)


def floor(P: _Patch, prm: _Params) -> int:
    """The floors applied to P's interior cells; the number changed."""
    return int(lib().orc_floor(C.byref(P), C.byref(prm)))


def floor_count() -> int:
    """Cells the last advance raised to the pressure floor."""
    return int(lib().orc_floor_count())


def patch(state: np.ndarray, n, g: int, dx) -> _Patch:
    """Describe a numpy state array (see module docstring) to the oracle."""
    assert state.dtype == np.float64 and state.flags.c_contiguous and state.ndim == 4
    _, nz1, ny1, px = state.shape
    n = tuple(int(v) for v in n)
    assert nz1 == n[2] + 2 * g + 1 and ny1 == n[1] + 2 * g + 1 and px >= n[0] + 2 * g + 1
    s = (1, px, px * ny1)
    base = state.ctypes.data
    plane = state.strides[0]
    P = _Patch()
    P.n[:] = n
    P.g = g
    P.s[:] = s
    P.dx[:] = tuple(float(v) for v in dx)
    for q in range(5):
        P.U[q] = base + q * plane
    for a in range(3):
        P.B[a] = base + (5 + a) * plane
    P._keep = state  # keep the buffer alive
    return P


# --------------------------------------------------------------- point functions
def limiter(lim: int, a: float, b: float) -> float:
    return lib().orc_limiter(lim, a, b)


def fast_speed(rho, p, bn, bt1, bt2, gamma=5.0 / 3.0) -> float:
    return lib().orc_fast_speed(rho, p, bn, bt1, bt2, gamma)


def flux(d: int, w, gamma=5.0 / 3.0) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(8)
    lib().orc_flux(d, _dp(w), gamma, _dp(f))
    return f


def hlld(d: int, wl, wr, bn: float, gamma=5.0 / 3.0, eps_up=UPWIND_EPS, with_upwind=False):
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(8)
    up = np.zeros(1)
    lib().orc_hlld(d, _dp(wl), _dp(wr), float(bn), gamma, eps_up, _dp(f), _dp(up))
    return (f, float(up[0])) if with_upwind else f


def hlld_fan(d: int, wl, wr, bn: float, gamma=5.0 / 3.0):
    """(speeds[5], states[6, 8], fluxes[2, 8]) of the HLLD fan, rotated frame."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    sp, st, fl = np.zeros(5), np.zeros(48), np.zeros(16)
    lib().orc_hlld_fan(d, _dp(wl), _dp(wr), float(bn), gamma, _dp(sp), _dp(st), _dp(fl))
    return sp, st.reshape(6, 8), fl.reshape(2, 8)


# --------------------------------------------------------------- patch functions
def fill_periodic(P: _Patch) -> None:
    lib().orc_fill_periodic(C.byref(P))


def cfl_dt(P: _Patch, prm: _Params) -> float:
    return lib().orc_cfl_dt(C.byref(P), C.byref(prm))


def captures(items):
    """items: iterable of (d, lo3, hi3, mode, dst ndarray float64)."""
    items = list(items)
    arr = (_Capture * max(1, len(items)))()
    keep = []
    for t, (d, lo, hi, mode, dst) in enumerate(items):
        assert dst.dtype == np.float64 and dst.flags.c_contiguous
        arr[t].d = d
        arr[t].lo[:] = lo
        arr[t].hi[:] = hi
        arr[t].mode = mode
        arr[t].dst = dst.ctypes.data
        keep.append(dst)
    arr._keep = keep
    return arr, len(items)


def advance(P: _Patch, prm: _Params, dt: float, k: int = 0, cap=None, ecap=None) -> int:
    cp, nc = cap if cap is not None else (None, 0)
    ep, ne = ecap if ecap is not None else (None, 0)
    r = lib().orc_advance(C.byref(P), C.byref(prm), float(dt), int(k), cp, nc, ep, ne)
    if r < 0:
        raise ValueError("orc_advance rejected its arguments (k + 2 > g?)")
    return int(r)


def sums(P: _Patch) -> np.ndarray:
    out = np.zeros(8)
    lib().orc_sums(C.byref(P), _dp(out))
    return out


def divb_max(P: _Patch) -> float:
    return lib().orc_divb_max(C.byref(P))


def _i3(v):
    return (C.c_int32 * 3)(*[int(x) for x in v])


def prolong(Pc: _Patch, cglo, Pf: _Patch, fglo, clo, chi) -> None:
    lib().orc_prolong(C.byref(Pc), _i3(cglo), C.byref(Pf), _i3(fglo), _i3(clo), _i3(chi))


def restrict(Pf: _Patch, fglo, Pc: _Patch, cglo, clo, chi, pass_) -> None:
    lib().orc_restrict(C.byref(Pf), _i3(fglo), C.byref(Pc), _i3(cglo), _i3(clo), _i3(chi), int(pass_))


def _planes(corr: np.ndarray):
    assert corr.dtype == np.float64 and corr.flags.c_contiguous and corr.shape[0] == 18
    arr = (C.c_void_p * 18)(*[corr.ctypes.data + q * corr.strides[0] for q in range(18)])
    return arr


def deposit_faces(Pc, cglo, corr, d, clo, chi, fine, flo, fhi, coarse) -> None:
    lib().orc_deposit_faces(C.byref(Pc), _i3(cglo), _planes(corr), int(d), _i3(clo), _i3(chi),
                            _dp(fine), _i3(flo), _i3(fhi), _dp(coarse))


def deposit_edges(Pc, cglo, corr, a, clo, chi, fine, flo, fhi, coarse) -> None:
    lib().orc_deposit_edges(C.byref(Pc), _i3(cglo), _planes(corr), int(a), _i3(clo), _i3(chi),
                            _dp(fine), _i3(flo), _i3(fhi), _dp(coarse))


def sync_faces(P, glo, corr, d, lo, hi, other, own) -> None:
    lib().orc_sync_faces(C.byref(P), _i3(glo), _planes(corr), int(d), _i3(lo), _i3(hi), _dp(other), _dp(own))


def sync_edges(P, glo, corr, a, lo, hi, other, own) -> None:
    lib().orc_sync_edges(C.byref(P), _i3(glo), _planes(corr), int(a), _i3(lo), _i3(hi), _dp(other), _dp(own))


def transfer_copy(Ps, sglo, Pd, dglo, kind, lo, hi) -> None:
    lib().orc_transfer_copy(C.byref(Ps), _i3(sglo), C.byref(Pd), _i3(dglo), int(kind), _i3(lo), _i3(hi))


def prolong_new(Pc, cglo, Pf, fglo, clo, chi, mask: np.ndarray, mlo, energy_mode: int = 1) -> int:
    """mask: uint8 array shaped (mext_z, mext_y, mext_x) over coarse cells from mlo."""
    assert mask.dtype == np.uint8 and mask.flags.c_contiguous
    mext = (mask.shape[2], mask.shape[1], mask.shape[0])
    return int(lib().orc_prolong_new(C.byref(Pc), _i3(cglo), C.byref(Pf), _i3(fglo), _i3(clo), _i3(chi),
                                     mask.ctypes.data, _i3(mlo), _i3(mext), int(energy_mode)))


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (n <= 0: all cores)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def flag(P: _Patch, prm: _Params, theta: float) -> np.ndarray:
    """Refinement flags of the interior cells, shape (nz, ny, nx), uint8."""
    nx, ny, nz = P.n
    out = np.zeros((nz, ny, nx), dtype=np.uint8)
    lib().orc_flag(C.byref(P), C.byref(prm), float(theta), out.ctypes.data)
    return out


def correct(P, corr) -> None:
    lib().orc_correct(C.byref(P), _planes(corr))


def copy(Ps, sglo, Pd, dglo, lo, hi, off, pass_) -> None:
    lib().orc_copy(C.byref(Ps), _i3(sglo), C.byref(Pd), _i3(dglo), _i3(lo), _i3(hi), _i3(off), int(pass_))


def run_periodic(state: np.ndarray, n, g: int, dx, prm: _Params, steps: int,
                 dt: float | None = None) -> list:
    """Single periodic patch: per step fill ghosts, compute dt (unless fixed),
    advance the interior.  Returns the list of dt values used."""
    P = patch(state, n, g, dx)
    dts = []
    for _ in range(steps):
        fill_periodic(P)
        h = cfl_dt(P, prm) if dt is None else dt
        nneg = advance(P, prm, h, 0)
        if nneg:
            raise FloatingPointError("oracle produced %d non-positive cells" % nneg)
        dts.append(h)
    fill_periodic(P)
    return dts
