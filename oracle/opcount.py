"""Algorithmic floating-point operation counts of the advance, per stage and
per unit of work, from the oracle compiled with a counting scalar
(``opcount.cpp``).

MEASUREMENT INFRASTRUCTURE ONLY (like the oracle itself).  Running this file
prints the counts of the periodic blast wave of a given size (ghost fill,
CFL dt and one advance of the interior) as JSON; the ALU roofline of the GPU
kernels divides these counts by measured kernel times.

Stages (the oracle's order; the GPU kernel that does the same work in
brackets) and their units:
  1 primitives + cell E^n      (k_prim)   cells of the update box grown by 2
  2 slopes + Hancock predictor (k_pred)   cells of the update box grown by 1
  3 edge E^n                   (k_edge)   edges around the box grown by 1
  4 CT half step of face B     (k_flux)   faces, with stage 5
  5 HLLD fluxes                (k_flux)   faces of the update box
  6 edge EMFs                  (k_emf)    edges of the update box
  7 cell and face update       (k_update) cells of the update box
  8 CFL dt                     (k_cfl)    interior cells
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opcount.cpp")
_LIB = os.path.join(_HERE, "libopcount.so")
OPS = ("add", "mul", "div", "sqrt", "cmp")


def build(force: bool = False) -> str:
    deps = [_SRC, os.path.join(_HERE, "mhd_oracle.c")]
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in deps):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-fvisibility=hidden", "-Wno-unknown-pragmas", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        from . import oracle as O
        L = O.bind(C.CDLL(build()))
        L.opc_reset.restype = None
        L.opc_read.restype = None
        L.opc_read.argtypes = [C.POINTER(C.c_int64)]
        L.opc_shape.restype = C.c_int32
        L.opc_shape.argtypes = [C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def read():
    L = lib()
    nops = C.c_int32()
    ns = L.opc_shape(C.byref(nops))
    buf = (C.c_int64 * (ns * nops.value))()
    L.opc_read(buf)
    return np.array(buf[:], dtype=np.int64).reshape(ns, nops.value)


def units(n, k=0):
    """Units of work of each stage for an n = (nx, ny, nz) interior and update
    box grown by k (the same element counts the GPU kernels launch over)."""
    u = [v + 2 * k for v in n]
    cells = lambda e: (u[0] + e) * (u[1] + e) * (u[2] + e)
    faces = sum((u[d] + 1) * (u[(d + 1) % 3] + 2) * (u[(d + 2) % 3] + 2) for d in range(3))
    return {1: cells(4), 2: cells(2),
            3: sum((u[a] + 2) * (u[(a + 1) % 3] + 3) * (u[(a + 2) % 3] + 3) for a in range(3)),
            4: faces, 5: faces,
            6: sum(u[a] * (u[(a + 1) % 3] + 1) * (u[(a + 2) % 3] + 1) for a in range(3)),
            7: cells(0), 8: n[0] * n[1] * n[2]}


def count_step(state, n, g, dx, prm, dt=None):
    """Counts of one ghost fill + CFL dt + advance (k = 0) of a periodic patch;
    returns ({stage: {op: count}}, dt used).  `state` is advanced in place."""
    from . import oracle as O
    L = lib()
    P = O.patch(state, n, g, dx)
    L.opc_reset()
    L.orc_fill_periodic(C.byref(P))
    h = L.orc_cfl_dt(C.byref(P), C.byref(prm))
    if dt is not None:
        h = dt
    L.orc_advance(C.byref(P), C.byref(prm), h, 0, None, 0, None, 0)
    c = read()
    out = {s: dict(zip(OPS, (int(v) for v in c[s]))) for s in range(c.shape[0]) if c[s].any()}
    return out, h


def per_unit(counts, n, k=0):
    """{stage: {op: per-unit count, 'flops': add+mul+div+sqrt per unit}}."""
    u = units(n, k)
    out = {}
    for s, ops in counts.items():
        if s not in u:
            continue
        d = {op: v / u[s] for op, v in ops.items()}
        d["flops"] = (ops["add"] + ops["mul"] + ops["div"] + ops["sqrt"]) / u[s]
        d["units"] = u[s]
        out[s] = d
    return out


def main(argv):
    import synth
    from . import oracle as O
    n = int(argv[0]) if argv else 128
    steps = int(argv[1]) if len(argv) > 1 else 1
    pr = synth.blast(n)
    prm = O.params(gamma=5.0 / 3.0, cfl=0.4, limiter=0, emf=1)
    st = pr.state.copy()
    res = []
    for s in range(steps):
        c, h = count_step(st, pr.n, pr.g, pr.dx, prm)
        res.append({"step": s, "dt": h, "per_unit": per_unit(c, pr.n)})
    print(json.dumps({"workload": "blast %d^3, van Leer, arithmetic EMF" % n, "steps": res}, indent=1))


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(_HERE))
    main(sys.argv[1:])
