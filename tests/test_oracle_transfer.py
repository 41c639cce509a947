"""Pins of the oracle's data transfer into a new iteration of a level
(regridding, Sec. 2.1; O step of Sec. 2.2) -- no GPU.

A global fine field (32^3, smooth or linear, face field from a vector
potential so div B = 0) defines the previous iteration: the old fine patches
are sub-boxes of it, and the coarse level (16^3, one periodic patch) is its
restriction.  A new fine patch that partly overlaps two old patches is
filled by oracle.transfer.  Pins:
  * the copied cells and faces equal the old data bit for bit;
  * div B of every fine cell of the new interior is zero to rounding (the
    seams between copied and prolonged cells included);
  * every coarse cell of the new footprint keeps its totals: the eight
    children's rho, M (and E, with the conservative energy option) sum to 8
    times the coarse value, and every coarse face's four sub-faces to 4 times
    the coarse face, to rounding;
  * a linear field (rho, M, B linear, B divergence-free) comes back exactly
    in rho, M and B;
  * the conservative energy keeps every child's thermal energy positive;
  * without old data the seam correction never fires and the result does not
    depend on the mask's face bits."""
import numpy as np
import pytest

import synth

G = 4
NF = 32
GAMMA = 5.0 / 3.0


def global_fine(kind, seed=3):
    """(state of the whole 32^3 fine domain with G ghost layers, dx)."""
    n = (NF, NF, NF)
    dx = (1.0 / NF,) * 3
    st = synth.empty_patch(n, G)
    rng = np.random.default_rng(seed)
    N = NF + 2 * G
    xc = (np.arange(N) - G + 0.5) / NF          # cell centres, ghosts included
    X, Y, Z = xc[None, None, :], xc[None, :, None], xc[:, None, None]
    if kind == "linear":
        ax = lambda x, y, z: 0.0 * x + 0.3 * y * z     # noqa: E731  curl gives B = (0.3 x?, ...) linear
        A = (lambda x, y, z: 0.2 * y * z, lambda x, y, z: -0.1 * x * z + 0.05 * z * z,
             lambda x, y, z: 0.15 * x * y)
        rho = 1.0 + 0.2 * X + 0.1 * Y - 0.05 * Z
        v = (0.1 + 0.0 * X, 0.05 + 0.0 * Y, -0.02 + 0.0 * Z)
        mom = [rho * v[0], rho * v[1], rho * v[2]]
        mom = [0.3 + 0.1 * X - 0.2 * Z, -0.1 + 0.3 * Y, 0.2 + 0.1 * X + 0.1 * Z]
        eth = 1.0 + 0.1 * X + 0.2 * Y + 0.1 * Z
    else:
        k = [rng.integers(1, 3, 3) for _ in range(3)]
        ph = rng.uniform(0, 2 * np.pi, 3)
        A = tuple((lambda kk, p: (lambda x, y, z: 0.05 * np.cos(2 * np.pi * (kk[0] * x + kk[1] * y + kk[2] * z) + p)))(k[c], ph[c])
                  for c in range(3))
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * (X + 2 * Y)) * np.cos(2 * np.pi * Z)
        mom = [0.4 * np.sin(2 * np.pi * Y) + 0 * X, 0.3 * np.cos(2 * np.pi * (X + Z)) + 0 * Y,
               0.2 * np.sin(2 * np.pi * (X - Y)) + 0 * Z]
        eth = 1.0 + 0.2 * np.cos(2 * np.pi * (Y + Z)) + 0 * X
    # faces on the whole array (ghosts too): potential sampled on edges
    sl = slice(0, N)
    full = synth.empty_patch((N, N, N), 0)
    synth._face_b_from_potential(full, (N, N, N), 0, (-G / NF,) * 3, dx, (0, 0, 0), A)
    st[5:8, :N + 1, :N + 1, :N + 1] = full[5:8, :N + 1, :N + 1, :N + 1]
    st[0, :N, :N, :N] = rho * np.ones((N, N, N))
    for a in range(3):
        st[1 + a, :N, :N, :N] = mom[a] * np.ones((N, N, N))
    bx = 0.5 * (st[5, :N, :N, :N] + st[5, :N, :N, 1:N + 1])
    by = 0.5 * (st[6, :N, :N, :N] + st[6, :N, 1:N + 1, :N])
    bz = 0.5 * (st[7, :N, :N, :N] + st[7, 1:N + 1, :N, :N])
    st[4, :N, :N, :N] = eth * np.ones((N, N, N)) + 0.5 * (st[1, :N, :N, :N] ** 2 + st[2, :N, :N, :N] ** 2 +
                                                          st[3, :N, :N, :N] ** 2) / st[0, :N, :N, :N] + \
        0.5 * (bx * bx + by * by + bz * bz)
    return st, dx


def sub_patch(gst, lo, hi):
    """The patch of the global fine field with interior [lo, hi] (ghosts from
    the global array)."""
    n = tuple(hi[d] - lo[d] + 1 for d in range(3))
    st = synth.empty_patch(n, G)
    sz = [n[d] + 2 * G + 1 for d in range(3)]
    st[:, :sz[2], :sz[1], :sz[0]] = gst[:, lo[2]:lo[2] + sz[2], lo[1]:lo[1] + sz[1], lo[0]:lo[0] + sz[0]]
    return st


def coarse_level(orc, gst, dxf):
    """The 16^3 restriction of the global fine field (one patch, G ghosts,
    periodic images as ghosts)."""
    nc = NF // 2
    cst = synth.empty_patch((nc, nc, nc), G)
    Pf = orc.patch(gst, (NF, NF, NF), G, dxf)
    Pc = orc.patch(cst, (nc, nc, nc), G, tuple(2 * v for v in dxf))
    for ps in (0, 1):
        orc.restrict(Pf, (0, 0, 0), Pc, (0, 0, 0), (0, 0, 0), (nc - 1,) * 3, ps)
    orc.fill_periodic(Pc)
    return cst


OLD = [((8, 8, 8), (15, 15, 15)), ((16, 8, 8), (23, 19, 15))]
NEW = ((12, 10, 6), (27, 21, 19))


def run(orc, kind, energy_mode=1, old=OLD):
    from oracle import transfer
    gst, dxf = global_fine(kind)
    cst = coarse_level(orc, gst, dxf)
    olds = [(sub_patch(gst, lo, hi), (lo, hi)) for lo, hi in old]
    n = tuple(NEW[1][d] - NEW[0][d] + 1 for d in range(3))
    new = synth.empty_patch(n, G)
    nf = transfer.transfer(new, NEW, G, dxf, olds, [(cst, ((0, 0, 0), (15, 15, 15)), G, tuple(2 * v for v in dxf))],
                           energy_mode)
    return gst, cst, new, n, dxf, nf


def interior(st, n):
    return st[:, G:G + n[2], G:G + n[1], G:G + n[0]]


def global_at(gst, box_lo, n):
    return gst[:, G + box_lo[2]:G + box_lo[2] + n[2] + 1, G + box_lo[1]:G + box_lo[1] + n[1] + 1,
               G + box_lo[0]:G + box_lo[0] + n[0] + 1]


def test_copied_region_equals_old_data(orc):
    from oracle import transfer
    gst, cst, new, n, dxf, _ = run(orc, "smooth")
    ref = global_at(gst, NEW[0], n)
    for j, kind, lo, hi in transfer.copy_items(NEW, OLD):
        sl = tuple(slice(lo[d] - NEW[0][d], hi[d] - NEW[0][d] + 1) for d in (2, 1, 0))
        got = new[:, G:, G:, G:]
        planes = range(5) if kind < 0 else [5 + kind]
        for q in planes:
            assert np.array_equal(got[q][sl], ref[q][sl]), (j, kind, q)


@pytest.mark.parametrize("kind", ["smooth", "linear"])
def test_div_free_and_conservative(orc, kind):
    gst, cst, new, n, dxf, nfall = run(orc, kind)
    assert nfall == 0
    P = orc.patch(new, n, G, dxf)
    scale = np.abs(new[5:8]).max()
    assert orc.divb_max(P) * dxf[0] <= 1e-13 * scale
    # per coarse cell totals and per coarse face sub-face sums
    c0 = [v // 2 for v in NEW[0]]
    nc = [v // 2 for v in n]
    ci = cst[:, G + c0[2]:G + c0[2] + nc[2], G + c0[1]:G + c0[1] + nc[1], G + c0[0]:G + c0[0] + nc[0]]
    fi = interior(new, n)
    for q in range(5):
        s8 = fi[q].reshape(nc[2], 2, nc[1], 2, nc[0], 2).sum(axis=(1, 3, 5))
        assert np.abs(s8 - 8 * ci[q]).max() <= 1e-13 * np.abs(ci[q]).max(), q
    for a in range(3):
        ext = list(n)
        ext[a] += 1
        f = new[5 + a, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
        # coarse faces: every other fine face along a, 2 x 2 sub-faces across
        take = [slice(None)] * 3
        take[2 - a] = slice(0, None, 2)
        f = f[tuple(take)]
        sh = [f.shape[0], f.shape[1], f.shape[2]]
        t = [d for d in range(3) if d != 2 - a]
        for d in t:
            sh[d] //= 2
        ff = f.reshape([sh[0], 2 if 0 in t else 1, sh[1], 2 if 1 in t else 1, sh[2], 2 if 2 in t else 1]).sum(
            axis=(1, 3, 5))
        cext = list(nc)
        cext[a] += 1
        cf = cst[5 + a, G + c0[2]:G + c0[2] + cext[2], G + c0[1]:G + c0[1] + cext[1], G + c0[0]:G + c0[0] + cext[0]]
        assert np.abs(ff - 4 * cf).max() <= 1e-13 * np.abs(cf).max(), a


def test_linear_field_exact(orc):
    gst, cst, new, n, dxf, _ = run(orc, "linear")
    ref = global_at(gst, NEW[0], n)
    got = new[:, G:, G:, G:]
    for q in (0, 1, 2, 3):
        a = got[q][:n[2], :n[1], :n[0]]
        b = ref[q][:n[2], :n[1], :n[0]]
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), q
    for a_ in range(3):
        ext = list(n)
        ext[a_] += 1
        a = got[5 + a_][:ext[2], :ext[1], :ext[0]]
        b = ref[5 + a_][:ext[2], :ext[1], :ext[0]]
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max(), a_


def test_conservative_energy_positive_thermal(orc):
    gst, cst, new, n, dxf, _ = run(orc, "smooth", energy_mode=1)
    fi = interior(new, n)
    bx = 0.5 * (new[5, G:G + n[2], G:G + n[1], G:G + n[0]] + new[5, G:G + n[2], G:G + n[1], G + 1:G + n[0] + 1])
    by = 0.5 * (new[6, G:G + n[2], G:G + n[1], G:G + n[0]] + new[6, G:G + n[2], G + 1:G + n[1] + 1, G:G + n[0]])
    bz = 0.5 * (new[7, G:G + n[2], G:G + n[1], G:G + n[0]] + new[7, G + 1:G + n[2] + 1, G:G + n[1], G:G + n[0]])
    e = fi[4] - 0.5 * (fi[1] ** 2 + fi[2] ** 2 + fi[3] ** 2) / fi[0] - 0.5 * (bx * bx + by * by + bz * bz)
    assert e.min() > 0


def test_no_old_data_needs_no_seam_correction(orc):
    """Without old patches the mask holds no bits: the result equals a run
    where the mask is recomputed from no boxes (no copies, no kept faces),
    and is divergence-free and conservative as above."""
    gst, cst, new, n, dxf, nfall = run(orc, "smooth", old=[])
    P = orc.patch(new, n, G, dxf)
    assert orc.divb_max(P) * dxf[0] <= 1e-13 * np.abs(new[5:8]).max()
    from oracle import transfer
    m, _ = transfer.mask(NEW, [])
    assert not m.any()
