"""Pins of the oracle's AMR operations and of the subcycled AMR step
(refinement ratio 2): prolongation exact for linear data and divergence-free,
restriction of a prolongation returns the coarse data, conservation and
div B with refluxing, single-valued shared faces, decomposition invariance,
prolongation from pre-advance data -- no GPU."""
import numpy as np
import pytest

import synth
import synth.amr as SA

G = 4


def _patch(orc, n, lo, dx):
    st = synth.empty_patch(n, G)
    return st, orc.patch(st, n, G, dx)


def _fill_linear(st, n, lo, dx, cell_fn, face_fns):
    """cells: cell_fn(x,y,z) at cell centres; faces: face_fns[a] at face centres
    (whole arrays, ghosts included)."""
    N = [v + 2 * G for v in n]
    for a in range(3):
        ext = list(N)
        ext[a] += 1
        idx = [np.arange(ext[d]) - G + lo[d] for d in range(3)]
        c = [(idx[d] + (0.0 if d == a else 0.5)) * dx[d] for d in range(3)]
        X, Y, Z = np.meshgrid(c[0], c[1], c[2], indexing="ij")
        st[5 + a, :ext[2], :ext[1], :ext[0]] = np.transpose(face_fns[a](X, Y, Z), (2, 1, 0))
    c = [(np.arange(N[d]) - G + lo[d] + 0.5) * dx[d] for d in range(3)]
    X, Y, Z = np.meshgrid(c[0], c[1], c[2], indexing="ij")
    for q in range(5):
        st[q, :N[2], :N[1], :N[0]] = np.transpose(cell_fn(q, X, Y, Z), (2, 1, 0))


def _set_energy_from_thermal(st, n, lo, dx, efn):
    """E = e + |M|^2/(2 rho) + |Bc|^2/2 with e linear (cell centres)."""
    N = [v + 2 * G for v in n]
    c = [(np.arange(N[d]) - G + lo[d] + 0.5) * dx[d] for d in range(3)]
    X, Y, Z = np.meshgrid(c[0], c[1], c[2], indexing="ij")
    e = np.transpose(efn(X, Y, Z), (2, 1, 0))
    sl = (slice(0, N[2]), slice(0, N[1]), slice(0, N[0]))
    rho, m = st[(0,) + sl], st[1:4, :N[2], :N[1], :N[0]]
    bx = 0.5 * (st[5, :N[2], :N[1], :N[0]] + st[5, :N[2], :N[1], 1:N[0] + 1])
    by = 0.5 * (st[6, :N[2], :N[1], :N[0]] + st[6, :N[2], 1:N[1] + 1, :N[0]])
    bz = 0.5 * (st[7, :N[2], :N[1], :N[0]] + st[7, 1:N[2] + 1, :N[1], :N[0]])
    st[(4,) + sl] = e + 0.5 * (m ** 2).sum(0) / rho + 0.5 * (bx * bx + by * by + bz * bz)
    return e


def _thermal(st, n):
    N = [v + 2 * G for v in n]
    rho, m = st[0, :N[2], :N[1], :N[0]], st[1:4, :N[2], :N[1], :N[0]]
    bx = 0.5 * (st[5, :N[2], :N[1], :N[0]] + st[5, :N[2], :N[1], 1:N[0] + 1])
    by = 0.5 * (st[6, :N[2], :N[1], :N[0]] + st[6, :N[2], 1:N[1] + 1, :N[0]])
    bz = 0.5 * (st[7, :N[2], :N[1], :N[0]] + st[7, 1:N[2] + 1, :N[1], :N[0]])
    return st[4, :N[2], :N[1], :N[0]] - 0.5 * (m ** 2).sum(0) / rho - 0.5 * (bx * bx + by * by + bz * bz)


def test_prolongation_exact_for_linear_data_and_divergence_free(orc):
    """Linear rho, M, thermal energy and a linear divergence-free field are
    reproduced exactly (rounding) by the prolongation."""
    nc, lo_c = (8, 8, 8), (0, 0, 0)
    dxc = (1.0, 1.0, 1.0)
    stc, Pc = _patch(orc, nc, lo_c, dxc)
    cell = lambda q, x, y, z: 3.0 + 0.1 * q + 0.3 * x - 0.2 * y + 0.05 * z
    efn = lambda x, y, z: 5.0 + 0.1 * x + 0.2 * y - 0.3 * z
    faces = [lambda x, y, z: 0.2 + 0.3 * y - 0.1 * z,
             lambda x, y, z: -0.4 + 0.2 * x + 0.25 * z,
             lambda x, y, z: 0.1 - 0.15 * x + 0.35 * y]
    _fill_linear(stc, nc, lo_c, dxc, cell, faces)
    _set_energy_from_thermal(stc, nc, lo_c, dxc, efn)
    nf, lo_f = (8, 8, 8), (4, 4, 4)
    dxf = (0.5, 0.5, 0.5)
    stf, Pf = _patch(orc, nf, lo_f, dxf)
    # prolong everything the fine patch holds (interior and ghosts): coarse box
    clo = tuple((v - G) // 2 for v in lo_f)
    chi = tuple((v + nf[d] + G) // 2 - 1 for d, v in enumerate(lo_f))
    stf[...] = 0.0
    # the prolongation skips the fine interior faces: fill those first so that
    # every face holds the linear field
    ref = np.zeros_like(stf)
    _fill_linear(ref, nf, lo_f, dxf, cell, faces)
    e_ref = _set_energy_from_thermal(ref, nf, lo_f, dxf, efn)
    stf[5:8] = ref[5:8]
    orc.prolong(Pc, lo_c, Pf, lo_f, clo, chi)
    N = [v + 2 * G for v in nf]
    assert np.abs(stf[:4, :N[2], :N[1], :N[0]] - ref[:4, :N[2], :N[1], :N[0]]).max() < 1e-13
    assert np.abs(_thermal(stf, nf) - e_ref).max() < 1e-12
    for a in range(3):
        ext = list(N)
        ext[a] += 1
        assert np.abs(stf[5 + a, :ext[2], :ext[1], :ext[0]] - ref[5 + a, :ext[2], :ext[1], :ext[0]]).max() < 1e-13


def test_prolongation_of_divergence_free_random_field(orc):
    """Faces from a random edge potential (discrete curl): every prolonged fine
    cell is divergence-free; restriction of the prolongation returns the
    coarse cells and faces."""
    rng = np.random.default_rng(3)
    nc = (8, 8, 8)
    stc, Pc = _patch(orc, nc, (0, 0, 0), (1.0, 1.0, 1.0))
    N = [v + 2 * G for v in nc]
    A = [rng.normal(size=(N[2] + 1, N[1] + 1, N[0] + 1)) for _ in range(3)]  # edge potential [k, j, i]
    # Bx(i,j,k) = (Az(j+1) - Az(j)) - (Ay(k+1) - Ay(k)), etc. (unit spacing)
    stc[5, :N[2], :N[1], :N[0] + 1] = (A[2][:N[2], 1:N[1] + 1, :] - A[2][:N[2], :N[1], :]) - (A[1][1:N[2] + 1, :N[1], :] - A[1][:N[2], :N[1], :])
    stc[6, :N[2], :N[1] + 1, :N[0]] = (A[0][1:N[2] + 1, :, :N[0]] - A[0][:N[2], :, :N[0]]) - (A[2][:N[2], :, 1:N[0] + 1] - A[2][:N[2], :, :N[0]])
    stc[7, :N[2] + 1, :N[1], :N[0]] = (A[1][:, :N[1], 1:N[0] + 1] - A[1][:, :N[1], :N[0]]) - (A[0][:, 1:N[1] + 1, :N[0]] - A[0][:, :N[1], :N[0]])
    stc[0] = rng.uniform(0.5, 2.0, stc.shape[1:])
    stc[1:5] = rng.normal(size=(4,) + stc.shape[1:])
    nf, lo_f = (8, 8, 8), (4, 4, 4)
    stf, Pf = _patch(orc, nf, lo_f, (0.5, 0.5, 0.5))
    # a fine patch whose own faces are left at zero: prolong only its ghosts
    # and check the ghost cells away from its interior
    clo = tuple((v - G) // 2 for v in lo_f)
    chi = tuple((v + nf[d] + G) // 2 - 1 for d, v in enumerate(lo_f))
    orc.prolong(Pc, (0, 0, 0), Pf, lo_f, clo, chi)
    Nf = [v + 2 * G for v in nf]
    div = ((stf[5, :Nf[2], :Nf[1], 1:Nf[0] + 1] - stf[5, :Nf[2], :Nf[1], :Nf[0]])
           + (stf[6, :Nf[2], 1:Nf[1] + 1, :Nf[0]] - stf[6, :Nf[2], :Nf[1], :Nf[0]])
           + (stf[7, 1:Nf[2] + 1, :Nf[1], :Nf[0]] - stf[7, :Nf[2], :Nf[1], :Nf[0]]))
    mask = np.ones_like(div, dtype=bool)
    mask[G - 1:G + nf[2] + 1, G - 1:G + nf[1] + 1, G - 1:G + nf[0] + 1] = False  # cells touching interior faces
    assert np.abs(div[mask]).max() < 1e-12 * np.abs(stc[5:8]).max()
    # restriction of the prolonged ghost zone reproduces the coarse data
    back = stc.copy()
    for pass_ in (0, 1):
        orc.restrict(Pf, lo_f, Pc, (0, 0, 0), (0, 0, 0), (1, 7, 7), pass_)  # coarse x in [0,1]: fine ghosts only
    # compare the coarse cells x in [0,1] and their faces except the x-face at
    # x = 2 (it is the fine patch's own, unset, boundary face)
    cs = (slice(G, G + 8), slice(G, G + 8), slice(G, G + 2))
    # rho and M are prolonged conservatively; E through the thermal energy
    assert np.abs(stc[(slice(0, 4),) + cs] - back[(slice(0, 4),) + cs]).max() < 1e-13 * np.abs(back[:4]).max()
    fx = (slice(G, G + 8), slice(G, G + 8), slice(G, G + 2))
    fy = (slice(G, G + 8), slice(G, G + 9), slice(G, G + 2))
    fz = (slice(G, G + 9), slice(G, G + 8), slice(G, G + 2))
    for a, sl in ((0, fx), (1, fy), (2, fz)):
        assert np.abs(stc[(5 + a,) + sl] - back[(5 + a,) + sl]).max() < 1e-13 * np.abs(back[5:8]).max()


def _hierarchy(orc, n0=16, levels=3, split=1, emf=1, p_in=10.0):
    from oracle.amr import OHierarchy
    H = SA.shell_hierarchy(n0=n0, levels=levels, size_min=4, size_max=8, level0_split=split)
    SA.check_hierarchy(H, n0)
    states = [[SA.blast_patch(lo, hi, l, n0, G, p_in=p_in)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, states, (1.0 / n0,) * 3, g=G, prm=orc.params(emf=emf))
    oh.initialise()
    oh.fill(0)
    return oh


def _shared_face_mismatch(oh, l):
    worst = 0.0
    pats = oh.levels[l]
    for P in pats:
        for Q in pats:
            for a in range(3):
                if P.hi[a] + 1 != Q.lo[a]:
                    continue
                lo = [max(P.lo[e], Q.lo[e]) for e in range(3)]
                hi = [min(P.hi[e], Q.hi[e]) for e in range(3)]
                lo[a] = hi[a] = Q.lo[a]
                if any(lo[e] > hi[e] for e in range(3)):
                    continue
                sp = P.state[5 + a, lo[2] - P.glo[2]:hi[2] - P.glo[2] + 1, lo[1] - P.glo[1]:hi[1] - P.glo[1] + 1,
                             lo[0] - P.glo[0]:hi[0] - P.glo[0] + 1]
                sq = Q.state[5 + a, lo[2] - Q.glo[2]:hi[2] - Q.glo[2] + 1, lo[1] - Q.glo[1]:hi[1] - Q.glo[1] + 1,
                             lo[0] - Q.glo[0]:hi[0] - Q.glo[0] + 1]
                worst = max(worst, float(np.abs(sp - sq).max()))
    return worst


@pytest.mark.parametrize("emf,p_in", [(1, 10.0), (0, 1.0)])
def test_amr_conservation_divb_and_single_valued_faces(orc, emf, p_in):
    """Arithmetic edge EMFs on the strong blast; Gardiner-Stone EMFs on a
    milder one (pressure ratio 10)."""
    oh = _hierarchy(orc, emf=emf, p_in=p_in)
    assert [len(l) for l in oh.levels] == [1, 47, 42]
    s0 = oh.sums()
    dv = (1.0 / 16) ** 3
    scale = np.abs(oh.levels[0][0].state[:, G:G + 16, G:G + 16, G:G + 16]).reshape(8, -1).sum(1) * dv
    for _ in range(3):
        oh.coarse_step()
        # same-level shared faces are computed from identical data: single-valued
        for l in range(3):
            assert _shared_face_mismatch(oh, l) == 0.0
    s1 = oh.sums()
    assert np.all(np.abs(s1 - s0) <= 1e-12 * np.maximum(scale, scale[0])), (s1 - s0)
    assert oh.divb_max() * (1.0 / 64) < 1e-12


def test_amr_level0_decomposition_invariance(orc):
    """The base level split into 8 patches gives the same bits as one patch."""
    a = _hierarchy(orc, split=1)
    b = _hierarchy(orc, split=2)
    for _ in range(2):
        a.coarse_step()
        b.coarse_step()
    for l in (1, 2):
        for Pa, Pb in zip(a.levels[l], b.levels[l]):
            assert Pa.lo == Pb.lo and np.array_equal(Pa.state, Pb.state)
    A0 = a.levels[0][0]
    for Pb in b.levels[0]:
        sl = tuple(slice(Pb.lo[2 - d] + G, Pb.hi[2 - d] + G + 1) for d in range(3))
        nb = tuple(Pb.n[2 - d] for d in range(3))
        assert np.array_equal(A0.state[(slice(0, 5),) + sl], Pb.state[(slice(0, 5),) + tuple(slice(G, G + v) for v in nb)])


def test_prolongation_uses_pre_advance_parent_data(orc):
    """Sec. 2.2: children are prolonged from the parent's data before its
    advance; perturbing the parent's advance leaves the children's two substeps
    unchanged."""
    ref = _hierarchy(orc, levels=2)
    per = _hierarchy(orc, levels=2)
    for oh, bump in ((ref, False), (per, True)):
        dt = oh.cfl_dt0()
        oh.fill(0)
        oh.prolong(0)
        oh.fill(1)
        oh.advance(0, 0, dt, True)
        if bump:
            oh.levels[0][0].state[0] *= 1.5
        oh.step(1, 2, 0.5 * dt, True)
        oh.fill(1)
        oh.step(1, 0, 0.5 * dt, False)
    for Pa, Pb in zip(ref.levels[1], per.levels[1]):
        assert np.array_equal(Pa.state[:, G:-G - 1, G:-G - 1, G:G + Pa.n[0]], Pb.state[:, G:-G - 1, G:-G - 1, G:G + Pb.n[0]])


def test_copy_lists_cover_each_ghost_element_once(orc):
    """Brute force over the cells of every destination's grown extended box:
    each cell is in at most one copy box, and in one exactly when some
    same-level interior image contains it."""
    oh = _hierarchy(orc)
    for l in (1, 2):
        n = 16 * 2 ** l
        for D in oh.levels[l]:
            lo = [v - G - 1 for v in D.lo]
            hi = [v + G + 1 for v in D.hi]
            shape = tuple(hi[d] - lo[d] + 1 for d in range(3))
            hits = np.zeros(shape, dtype=int)
            for (s, d, b, off) in oh.copy_lists[l]:
                if d != D.idx:
                    continue
                hits[b[0][0] - lo[0]:b[1][0] - lo[0] + 1, b[0][1] - lo[1]:b[1][1] - lo[1] + 1,
                     b[0][2] - lo[2]:b[1][2] - lo[2] + 1] += 1
            want = np.zeros(shape, dtype=int)
            for S in oh.levels[l]:
                for sh in [(x, y, z) for x in (-n, 0, n) for y in (-n, 0, n) for z in (-n, 0, n)]:
                    if S is D and sh == (0, 0, 0):
                        continue
                    a = [max(S.lo[d] + sh[d], lo[d]) for d in range(3)]
                    b = [min(S.hi[d] + sh[d], hi[d]) for d in range(3)]
                    if all(a[d] <= b[d] for d in range(3)):
                        want[a[0] - lo[0]:b[0] - lo[0] + 1, a[1] - lo[1]:b[1] - lo[1] + 1, a[2] - lo[2]:b[2] - lo[2] + 1] += 1
            assert hits.max() <= 1 and np.array_equal(hits, want)
