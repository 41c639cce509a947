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


def test_pressure_floor_closed_form(orc):
    """The optional pressure floor (reading R33) at a level below every
    pressure of the initial state (0.1 outside the blast), so that it only
    acts after the update: every cell whose new pressure lies below p_floor
    has its energy raised by exactly (p_floor - p) / (gamma - 1), computed from
    the unfloored update; every other value is the unfloored one bit for bit,
    and p_floor = 0 changes nothing."""
    pr = synth.blast(12, noise=0.01, seed=4)
    g, n = pr.g, pr.n
    a, b = pr.state.copy(), pr.state.copy()
    Pa, Pb = orc.patch(a, n, g, pr.dx), orc.patch(b, n, g, pr.dx)
    for P in (Pa, Pb):
        orc.fill_periodic(P)
    dt = orc.cfl_dt(Pa, orc.params(emf=1))
    assert orc.advance(Pa, orc.params(emf=1), dt, 0) == 0
    assert orc.floor_count() == 0
    assert orc.advance(Pb, orc.params(emf=1, p_floor=0.099), dt, 0) == 0
    nfl = orc.floor_count()
    st = interior(a, n, g)
    bx = 0.5 * (a[5, g:g + n[2], g:g + n[1], g:g + n[0]] + a[5, g:g + n[2], g:g + n[1], g + 1:g + n[0] + 1])
    by = 0.5 * (a[6, g:g + n[2], g:g + n[1], g:g + n[0]] + a[6, g:g + n[2], g + 1:g + n[1] + 1, g:g + n[0]])
    bz = 0.5 * (a[7, g:g + n[2], g:g + n[1], g:g + n[0]] + a[7, g + 1:g + n[2] + 1, g:g + n[1], g:g + n[0]])
    ir = 1.0 / st[0]
    v = [st[1 + c] * ir for c in range(3)]
    p = (G - 1.0) * (st[4] - 0.5 * st[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - 0.5 * (bx * bx + by * by + bz * bz))
    low = p < 0.099
    assert nfl == int(low.sum()) and 0 < nfl < low.size
    want = st[4] + np.where(low, (0.099 - p) / (G - 1.0), 0.0)
    got = interior(b, n, g)
    assert np.array_equal(got[4][~low], st[4][~low])
    assert np.abs(got[4][low] - want[low]).max() <= 1e-15 * np.abs(want).max()
    assert np.array_equal(np.delete(got, 4, axis=0), np.delete(st, 4, axis=0))


def test_density_and_pressure_floor_closed_form(orc):
    """orc_floor on a state with planted low-density and low-pressure cells:
    a density below rho_floor becomes rho_floor with M and B kept and the
    pressure reset to p_floor; a pressure below p_floor (density above) is
    raised to p_floor; every other cell is left bit for bit."""
    pr = synth.blast(8, noise=0.01, seed=5)
    g, n = pr.g, pr.n
    st = pr.state.copy()
    P = orc.patch(st, n, g, pr.dx)
    orc.fill_periodic(P)
    lowrho = (g + 1, g + 2, g + 3)       # (i, j, k)
    st[0, lowrho[2], lowrho[1], lowrho[0]] = 1e-6
    before = st.copy()
    prm = orc.params(p_floor=0.2, rho_floor=1e-3)
    nch = orc.floor(P, prm)
    it = interior(st, n, g)
    ib = interior(before, n, g)
    bx = 0.5 * (ib[5] + before[5, g:g + n[2], g:g + n[1], g + 1:g + n[0] + 1])
    by = 0.5 * (ib[6] + before[6, g:g + n[2], g + 1:g + n[1] + 1, g:g + n[0]])
    bz = 0.5 * (ib[7] + before[7, g + 1:g + n[2] + 1, g:g + n[1], g:g + n[0]])
    me = 0.5 * (bx * bx + by * by + bz * bz)
    rho, m2 = ib[0], ib[1] ** 2 + ib[2] ** 2 + ib[3] ** 2
    p = (G - 1.0) * (ib[4] - 0.5 * rho * (m2 / rho ** 2) - me)
    dens = rho < 1e-3
    pres = ~dens & (p < 0.2)
    assert dens.sum() == 1 and pres.sum() > 0 and nch == dens.sum() + pres.sum()
    k, j, i = lowrho[2] - g, lowrho[1] - g, lowrho[0] - g
    assert it[0, k, j, i] == 1e-3
    e_want = 0.2 / (G - 1.0) + 0.5 * m2[k, j, i] / 1e-3 + me[k, j, i]
    assert abs(it[4, k, j, i] - e_want) <= 1e-14 * e_want
    assert np.all(np.abs(it[4][pres] - (ib[4][pres] + (0.2 - p[pres]) / (G - 1.0))) <= 1e-14 * np.abs(ib[4]).max())
    keep = ~dens & ~pres
    assert np.array_equal(it[:, keep], ib[:, keep])
    assert np.array_equal(it[1:4], ib[1:4]) and np.array_equal(st[5:8], before[5:8])


def test_thread_count_does_not_change_the_result(orc):
    """The oracle's OpenMP loops run over independent cells (each writes its
    own outputs; the CFL dt is a max), so one thread and all threads give the
    same bits: the one-core and all-core timings time the same arithmetic."""
    pr = synth.blast(16)
    a, b = pr.state.copy(), pr.state.copy()
    prm = orc.params()
    try:
        orc.set_threads(1)
        assert orc.get_threads() == 1
        orc.run_periodic(a, pr.n, pr.g, pr.dx, prm, 3)
        orc.set_threads(0)
        assert orc.get_threads() >= 1
        orc.run_periodic(b, pr.n, pr.g, pr.dx, prm, 3)
    finally:
        orc.set_threads(0)
    assert np.array_equal(a, b)
