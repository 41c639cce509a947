"""Pins of the oracle's upwinded edge EMF (Gardiner & Stone 2005, J. Comput.
Phys. 205:509; the edge-EMF step of the hyperbolic advance of each grid,
Sec. 2.3) -- no GPU.

The corner EMF adds to the mean of the four face EMFs two derivative terms
per direction, each taken on the side of the face that the contact (mass
flux) comes from, and averaged over both sides when the mass flux is zero.
Uniform states, conservation, div B, the Alfven-wave order and the
symmetries that a consistent mistake preserves do not see which side is
taken.  These pins do:

* field loop (the advection test GS05 built the scheme on): a weak loop of
  field carried by a uniform flow is passive, so its magnetic energy may only
  decay (numerical dissipation); taking the downwind side of the contact is
  anti-dissipative and the energy grows within a few steps.  Flows along
  each in-plane axis alone catch a mistake on one axis; the loop in each of
  the three coordinate planes puts every edge orientation under test;
* mirror symmetry: a loop carried along x is mirror-symmetric in y, and the
  faces on the mirror plane carry exactly zero mass flux, where both sides
  must be averaged;
* transposition covariance: exchanging x and y (with the vector components)
  is a symmetry of ideal MHD, and the two derivative terms of a corner must
  enter alike; a swirling flow makes the contact side change from row to
  row and column to column.

``test_pins_catch_planted_mistakes`` compiles copies of the oracle with
plausible mistakes planted in this step (swapped sides, the side of one axis
swapped, the row of the deciding face shifted, the sign of the correction
flipped, one side taken at zero mass flux, a derivative term dropped, the
reference cells swapped) and checks that each one fails a pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import synth

LOOP_N = 24
LOOP_STEPS = 30


def _run(L, orc, pr, steps, prm, dt=None):
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    for _ in range(steps):
        L.orc_fill_periodic(C.byref(P))
        h = L.orc_cfl_dt(C.byref(P), C.byref(prm)) if dt is None else dt
        L.orc_advance(C.byref(P), C.byref(prm), h, 0, None, 0, None, 0)
        yield


def _magnetic_energy(pr):
    st, g = pr.state, pr.g
    nx, ny, nz = pr.n
    bx = 0.5 * (st[5, g:g + nz, g:g + ny, g:g + nx] + st[5, g:g + nz, g:g + ny, g + 1:g + nx + 1])
    by = 0.5 * (st[6, g:g + nz, g:g + ny, g:g + nx] + st[6, g:g + nz, g + 1:g + ny + 1, g:g + nx])
    bz = 0.5 * (st[7, g:g + nz, g:g + ny, g:g + nx] + st[7, g + 1:g + nz + 1, g:g + ny, g:g + nx])
    return 0.5 * float(np.sum(bx * bx + by * by + bz * bz))


def _loop_cases():
    out = []
    for normal in range(3):
        t1, t2 = (normal + 1) % 3, (normal + 2) % 3
        for a, b in ((1.0, 0.0), (0.0, -1.0), (-1.0, 0.5)):
            v = [0.0, 0.0, 0.0]
            v[t1], v[t2] = a, b
            out.append((normal, tuple(v)))
    return out


def field_loop_failures(L, orc):
    """Cases whose magnetic energy rose in some step or fell below 0.7 of
    its start (the loop destroyed) within LOOP_STEPS steps."""
    bad = []
    for normal, v in _loop_cases():
        pr = synth.field_loop(LOOP_N, normal, v)
        e = [_magnetic_energy(pr)]
        for _ in _run(L, orc, pr, LOOP_STEPS, orc.params()):
            e.append(_magnetic_energy(pr))
        e = np.array(e)
        rises = int(np.sum(np.diff(e) > 1e-13 * e[0]))
        if rises or not (0.7 < e[-1] / e[0] <= 1.0):
            bad.append((normal, v, rises, e[-1] / e[0]))
    return bad


def mirror_error(L, orc):
    """Largest departure from the y-mirror symmetry of a loop carried along
    +x and along -x (densities and momenta absolute, fields relative to the
    loop's field strength)."""
    worst = 0.0
    for v in ((1.0, 0.0, 0.0), (-1.0, 0.0, 0.0)):
        pr = synth.field_loop(LOOP_N, 2, v)
        for _ in _run(L, orc, pr, LOOP_STEPS, orc.params()):
            pass
        st, g, n = pr.state, pr.g, LOOP_N
        rho = st[0, g, g:g + n, g:g + n]
        my = st[2, g, g:g + n, g:g + n]
        bx = st[5, g, g:g + n, g:g + n + 1]
        by = st[6, g, g:g + n + 1, g:g + n]
        worst = max(worst, np.abs(rho - rho[::-1]).max(), np.abs(my + my[::-1]).max(),
                    np.abs(bx + bx[::-1]).max() / 1e-3, np.abs(by - by[::-1]).max() / 1e-3)
    return float(worst)


def _transpose(st, n, g):
    """The 2D state with x and y exchanged (cells, momenta, face fields)."""
    N = n + 2 * g
    t = np.zeros_like(st)
    z = slice(0, 1 + 2 * g)
    for q, src in ((0, 0), (1, 2), (2, 1), (3, 3), (4, 4)):
        t[q, z, :N, :N] = np.transpose(st[src, z, :N, :N], (0, 2, 1))
    t[5, z, :N, :N + 1] = np.transpose(st[6, z, :N + 1, :N], (0, 2, 1))
    t[6, z, :N + 1, :N] = np.transpose(st[5, z, :N, :N + 1], (0, 2, 1))
    t[7, 0:2 + 2 * g, :N, :N] = np.transpose(st[7, 0:2 + 2 * g, :N, :N], (0, 2, 1))
    return t


def transposition_error(L, orc, n=24, steps=10):
    pr = synth.swirl_2d(n)
    tr = synth.Problem("swirl_t", _transpose(pr.state, n, pr.g), pr.n, pr.g, pr.dx, pr.xlo)
    for p in (pr, tr):
        for _ in _run(L, orc, p, steps, orc.params(), dt=2e-3):
            pass
    back = _transpose(tr.state, n, pr.g)
    g = pr.g
    sl = (slice(None), slice(g, g + 1), slice(g, g + n), slice(g, g + n))
    return float(np.abs(back[sl] - pr.state[sl]).max())


# ----------------------------------------------------------------- the pins
def test_field_loop_energy_never_rises(orc):
    bad = field_loop_failures(orc.lib(), orc)
    assert not bad, bad


def test_field_loop_mirror_symmetry(orc):
    assert mirror_error(orc.lib(), orc) <= 1e-12


def test_transposition_covariance_swirl(orc):
    assert transposition_error(orc.lib(), orc) <= 1e-12


# ------------------------------------------------- planted mistakes, on the CPU
def _stage6(src):
    a = src.index("ORC_STAGE(6)")
    b = src.index("flux-register capture (before")
    return a, b


def _plant(src, pairs):
    a, b = _stage6(src)
    seg = src[a:b]
    for old, new in pairs:
        assert old in seg, "planting target not found in the edge-EMF step: %r" % old
        seg = seg.replace(old, new)
    return src[:a] + seg + src[b:]


def _swap_sign_tests(text):
    return text.replace("> 0.0)", "@GT@").replace("< 0.0)", "> 0.0)").replace("@GT@", "< 0.0)")


MB = ("if (mb_hi > 0.0) dc14 = r01 - ec_lo;\n          else if (mb_hi < 0.0) dc14 = r11 - ec_hi;",
      "if (mb_lo > 0.0) dc34 = ec_lo - r00;\n          else if (mb_lo < 0.0) dc34 = ec_hi - r10;")
MC = ("if (mc_hi > 0.0) db14 = r10 - eb_lo;\n          else if (mc_hi < 0.0) db14 = r11 - eb_hi;",
      "if (mc_lo > 0.0) db34 = eb_lo - r00;\n          else if (mc_lo < 0.0) db34 = eb_hi - r01;")
ZERO = [("else dc14 = 0.5 * ((r01 - ec_lo) + (r11 - ec_hi));", "else dc14 = r01 - ec_lo;"),
        ("else dc34 = 0.5 * ((ec_lo - r00) + (ec_hi - r10));", "else dc34 = ec_lo - r00;"),
        ("else db14 = 0.5 * ((r10 - eb_lo) + (r11 - eb_hi));", "else db14 = r10 - eb_lo;"),
        ("else db34 = 0.5 * ((eb_lo - r00) + (eb_hi - r01));", "else db34 = eb_lo - r00;")]
CORR = "0.25 * (dc34 - dc14 + db34 - db14)"
MISTAKES = {
    "both sides swapped": [(s, _swap_sign_tests(s)) for s in MB + MC],
    "x-contact side swapped": [(s, _swap_sign_tests(s)) for s in MB],
    "y-contact side swapped": [(s, _swap_sign_tests(s)) for s in MC],
    "deciding face one row off": [("double mb_lo = Up[b][c - s[cc]];\n          double mb_hi = Up[b][c];",
                                   "double mb_hi = Up[b][c - s[cc]];\n          double mb_lo = Up[b][c];")],
    "correction sign flipped": [(CORR, "0.25 * (dc14 - dc34 + db14 - db34)")],
    "one side at zero mass flux": ZERO,
    "one derivative term dropped": [(CORR, "0.25 * (dc34 - dc14)")],
    "reference cells swapped": [("double r10 = Er[a][c - s[cc]];\n          double r01 = Er[a][c - s[b]];",
                                 "double r01 = Er[a][c - s[cc]];\n          double r10 = Er[a][c - s[b]];")],
}


def _build_planted(tmp_path, name, src):
    c = tmp_path / ("orc_%s.c" % name.replace(" ", "_"))
    so = c.with_suffix(".so")
    c.write_text(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                           "-shared", "-fvisibility=hidden", str(c), "-o", str(so), "-lm"])
    return so


def test_pins_catch_planted_mistakes(orc, tmp_path):
    src_path = os.path.join(os.path.dirname(orc.__file__), "mhd_oracle.c")
    with open(src_path) as f:
        src = f.read()
    missed = []
    for name, pairs in MISTAKES.items():
        L = orc.bind(C.CDLL(str(_build_planted(tmp_path, name, _plant(src, pairs)))))
        caught = bool(field_loop_failures(L, orc))
        caught = caught or mirror_error(L, orc) > 1e-12
        caught = caught or transposition_error(L, orc) > 1e-12
        if not caught:
            missed.append(name)
    assert not missed, "pins pass with a planted mistake: %s" % missed


@pytest.mark.parametrize("lim", [0, 1, 2])
def test_field_loop_energy_every_limiter(orc, lim):
    """The energy pin holds with every limiter (loop along the diagonal)."""
    pr = synth.field_loop(LOOP_N, 2, (1.0, 0.5, 0.0))
    e = [_magnetic_energy(pr)]
    for _ in _run(orc.lib(), orc, pr, LOOP_STEPS, orc.params(limiter=lim)):
        e.append(_magnetic_energy(pr))
    assert np.all(np.diff(e) <= 1e-13 * e[0]) and e[-1] / e[0] > 0.7, e
