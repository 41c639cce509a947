"""Pins of the oracle's whole patch advance (single periodic patch) against
invariants and closed forms -- no GPU."""
import math

import numpy as np
import pytest

import synth

G = 5.0 / 3.0


def interior(st, n, g):
    nx, ny, nz = n
    return st[:, g:g + nz, g:g + ny, g:g + nx]


def test_uniform_state_preserved_exactly(orc):
    pr = synth.uniform((8, 6, 5))
    prm = orc.params()
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    orc.fill_periodic(P)
    ref = pr.state.copy()
    for lim in (0, 1, 2):
        for emf in (0, 1):
            prm = orc.params(limiter=lim, emf=emf)
            for _ in range(25):
                orc.fill_periodic(P)
                assert orc.advance(P, prm, orc.cfl_dt(P, prm), 0) == 0
            orc.fill_periodic(P)
            assert np.array_equal(pr.state, ref)


def test_cfl_dt_closed_form(orc):
    pr = synth.uniform((8, 6, 5), rho=1.3, v=(0.3, -0.2, 0.1), p=0.7, B=(0.4, -0.5, 0.6))
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    orc.fill_periodic(P)
    prm = orc.params(cfl=0.4)
    rho, v, p, B = 1.3, np.array([0.3, -0.2, 0.1]), 0.7, np.array([0.4, -0.5, 0.6])
    a2, b2 = G * p / rho, B @ B / rho
    best = []
    for d in range(3):
        cf = math.sqrt(0.5 * (a2 + b2 + math.sqrt((a2 + b2) ** 2 - 4 * a2 * B[d] ** 2 / rho)))
        best.append(pr.dx[d] / (abs(v[d]) + cf))
    assert orc.cfl_dt(P, prm) == pytest.approx(0.4 * min(best), rel=1e-14)


@pytest.mark.parametrize("problem", ["ot", "blast"])
def test_periodic_conservation_and_divb(orc, problem):
    pr = synth.orszag_tang(32) if problem == "ot" else synth.blast(16)
    prm = orc.params()
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    orc.fill_periodic(P)
    s0 = orc.sums(P)
    dv = pr.dx[0] * pr.dx[1] * pr.dx[2]
    scale0 = np.abs(interior(pr.state, pr.n, pr.g)).reshape(8, -1).sum(axis=1) * dv
    bmax = np.abs(interior(pr.state, pr.n, pr.g)[5:8]).max()
    for step in range(15):
        orc.fill_periodic(P)
        assert orc.advance(P, prm, orc.cfl_dt(P, prm), 0) == 0
        orc.fill_periodic(P)
        assert orc.divb_max(P) * min(pr.dx) / bmax <= 1e-13
    s1 = orc.sums(P)
    # roundoff of the per-cell updates summed over the patch and the steps;
    # a dropped or mis-signed flux term moves these by O(1e-3) of the scale
    scale = np.maximum(scale0, np.abs(interior(pr.state, pr.n, pr.g)).reshape(8, -1).sum(axis=1) * dv)
    assert np.all(np.abs(s1 - s0) <= 1e-12 * scale), (s1 - s0) / scale


def test_linear_alfven_wave_second_order_2d(orc):
    """Oblique 2D Alfven wave, k = 2 pi (1, 2): L1 error of the transverse
    velocity after one period falls by ~4 per doubling of resolution (the
    limiter clips the extrema at coarse resolution, so the order is taken
    from the finest pair)."""
    errs = []
    for n in (32, 64, 128):
        pr, exact, period = synth.alfven_wave(n, ndim=2, amp=1e-6)
        prm = orc.params()
        P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
        orc.fill_periodic(P)
        dt0 = orc.cfl_dt(P, prm)
        nsteps = int(math.ceil(period / dt0))
        orc.run_periodic(pr.state, pr.n, pr.g, pr.dx, prm, nsteps, dt=period / nsteps)
        st = interior(pr.state, pr.n, pr.g)
        vz = st[3] / st[0]
        ex = exact(period)["v"][2]
        errs.append(np.abs(vz - ex).mean() / 1e-6)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] >= 1.9, (errs, orders)
    assert math.log2(errs[0] / errs[-1]) / 2 >= 1.8, (errs, orders)
    assert errs[-1] < 0.006


def test_linear_alfven_wave_3d_converges(orc):
    errs = []
    for n in (8, 16):
        pr, exact, period = synth.alfven_wave(n, ndim=3, amp=1e-6)
        prm = orc.params()
        P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
        orc.fill_periodic(P)
        dt0 = orc.cfl_dt(P, prm)
        nsteps = int(math.ceil(period / dt0))
        orc.run_periodic(pr.state, pr.n, pr.g, pr.dx, prm, nsteps, dt=period / nsteps)
        st = interior(pr.state, pr.n, pr.g)
        ex = exact(period)["v"]
        err = sum(np.abs(st[1 + c] / st[0] - ex[c]).mean() for c in range(3)) / 1e-6
        errs.append(err)
    assert math.log2(errs[0] / errs[1]) >= 1.7, errs


def test_orszag_tang_point_symmetry(orc):
    pr = synth.orszag_tang(32)
    orc.run_periodic(pr.state, pr.n, pr.g, pr.dx, orc.params(), 30)
    st = interior(pr.state, pr.n, pr.g)[:, 0]
    rho, p_like = st[0], st[4]
    assert np.abs(rho - rho[::-1, ::-1]).max() <= 1e-12 * np.abs(rho).max()
    assert np.abs(p_like - p_like[::-1, ::-1]).max() <= 1e-12 * np.abs(p_like).max()
    mx_ = st[1]
    assert np.abs(mx_ + mx_[::-1, ::-1]).max() <= 1e-12 * np.abs(mx_).max()


@pytest.mark.parametrize("emf", [0, 1])
def test_blast_symmetries(orc, emf):
    """Noise-free blast with B = (1,1,0)/sqrt 2: point inversion (v -> -v,
    B -> B) and the x <-> y exchange are symmetries of ideal MHD."""
    pr = synth.blast(16, noise=0.0)
    orc.run_periodic(pr.state, pr.n, pr.g, pr.dx, orc.params(emf=emf), 12)
    st = interior(pr.state, pr.n, pr.g)
    rho, e = st[0], st[4]
    assert np.abs(rho - rho[::-1, ::-1, ::-1]).max() <= 1e-12
    assert np.abs(e - e[::-1, ::-1, ::-1]).max() <= 1e-12 * np.abs(e).max()
    assert np.abs(rho - rho.transpose(0, 2, 1)).max() <= 1e-12
    mz = st[3]
    assert np.abs(mz + mz[::-1, ::-1, ::-1]).max() <= 1e-12


def test_cyclic_axis_permutation(orc):
    """Rotating the problem x -> y -> z -> x rotates the solution."""
    pr = synth.blast(12, noise=0.01, seed=3)
    g, n = pr.g, 12
    st0 = pr.state.copy()
    # rotated copy: new (x, y, z) = old (z, x, y)  -> array [q, k, j, i] new = old[q, j, i, k]
    rot = np.zeros_like(st0)
    def cell(a):  # (NZ, NY, NX) view of the cell block
        return a[:n + 2 * g, :n + 2 * g, :n + 2 * g]
    for q in range(5):
        src = cell(st0[q])
        rot[q, :n + 2 * g, :n + 2 * g, :n + 2 * g] = np.transpose(src, (1, 2, 0))
    # momentum components rotate too: new Mx = old Mz, new My = old Mx, new Mz = old My
    rot[[1, 2, 3]] = rot[[3, 1, 2]]
    # faces: new Bx on x-faces = old Bz on z-faces, etc.
    N = n + 2 * g
    rot[5, :N, :N, :N + 1] = np.transpose(st0[7, :N + 1, :N, :N], (1, 2, 0))
    rot[6, :N, :N + 1, :N] = np.transpose(st0[5, :N, :N, :N + 1], (1, 2, 0))
    rot[7, :N + 1, :N, :N] = np.transpose(st0[6, :N, :N + 1, :N], (1, 2, 0))
    a, b = st0.copy(), rot
    prm = orc.params()
    orc.run_periodic(a, pr.n, g, pr.dx, prm, 6, dt=2e-3)
    orc.run_periodic(b, pr.n, g, pr.dx, prm, 6, dt=2e-3)
    ra = interior(a, pr.n, g)[0]
    rb = interior(b, pr.n, g)[0]
    assert np.abs(np.transpose(ra, (1, 2, 0)) - rb).max() <= 1e-13
