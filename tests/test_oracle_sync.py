"""Pins of the oracle's synchronisation of fluxes on faces shared by two
patches of one level (Sec. 2.2 S step; reading R14) -- no GPU.

A periodic 16^3 Alfven-wave state is cut at x = 8 into two patches A and B
whose ghosts hold each other's cells.  B's lower x-ghosts (A's cells) are
then perturbed, so that the two patches compute different fluxes and EMFs on
their shared faces at x = 8.  After the advance, each patch is corrected
towards the mean of the two registers.  Pins:
  * the totals of rho, M, E over both interiors are conserved to rounding
    with the synchronisation and not without it (the shared faces then carry
    one flux, and the periodic faces x = 0 / 16 already agree);
  * the face field B_x on the shared faces is single-valued to rounding with
    it (the EMFs of the shared edges are then one) and two-valued without it;
  * div B stays at rounding in both patches;
  * with unperturbed ghosts the two registers agree bit for bit (R14) and the
    synchronisation leaves both patches unchanged, bit for bit."""
import numpy as np

import synth

G = 2
AT = 8


def setup(orc, perturb):
    pr, _, _ = synth.alfven_wave(16, ndim=3, amp=0.1)
    P = orc.patch(pr.state, pr.n, G, pr.dx)
    orc.fill_periodic(P)
    dt = orc.cfl_dt(P, orc.params(emf=1))
    A, na, B, nb = synth.split_x(pr, AT)
    if perturb:
        B[0:5, :, :, 0:G] *= 1.05
    return pr, dt, (A, na, (0, 0, 0)), (B, nb, (AT, 0, 0))


def boxes(n, glo, side):
    """Array-index boxes (capture layout) of one patch's shared x face and of
    its shared y- and z-edges on that face; side 0: the lower x boundary."""
    xi = G if side == 0 else G + n[0]
    face = ((xi, G, G), (xi, G + n[1] - 1, G + n[2] - 1))
    ey = ((xi, G, G), (xi, G + n[1] - 1, G + n[2]))      # along y, z edge index up to hi + 1
    ez = ((xi, G, G), (xi, G + n[1], G + n[2] - 1))
    return face, ey, ez


def vol(b):
    return int(np.prod(np.array(b[1]) - np.array(b[0]) + 1))


def step(orc, pr, dt, parts, sync):
    prm = orc.params(emf=1)
    regs = []
    for (st, n, glo), side in zip(parts, (1, 0)):
        P = orc.patch(st, n, G, pr.dx)
        face, ey, ez = boxes(n, glo, side)
        rf = np.zeros(5 * vol(face))
        r1 = np.zeros(vol(ey))
        r2 = np.zeros(vol(ez))
        cap = orc.captures([(0, face[0], face[1], 0, rf)])
        ecap = orc.captures([(1, ey[0], ey[1], 0, r1), (2, ez[0], ez[1], 0, r2)])
        assert orc.advance(P, prm, dt, 0, cap=cap, ecap=ecap) == 0
        regs.append((P, n, glo, face, ey, ez, rf, r1, r2))
    if sync:
        for me, other in ((0, 1), (1, 0)):
            P, n, glo, face, ey, ez, rf, r1, r2 = regs[me]
            o = regs[other]
            corr = np.zeros((18,) + parts[me][0].shape[1:])

            def gbox(b):
                return (tuple(b[0][d] - G + glo[d] for d in range(3)), tuple(b[1][d] - G + glo[d] for d in range(3)))
            lo, hi = gbox(face)
            orc.sync_faces(P, glo, corr, 0, lo, hi, o[6], rf)
            lo, hi = gbox(ey)
            orc.sync_edges(P, glo, corr, 1, lo, hi, o[7], r1)
            lo, hi = gbox(ez)
            orc.sync_edges(P, glo, corr, 2, lo, hi, o[8], r2)
            orc.correct(P, corr)
    return regs


def totals(parts):
    t = np.zeros(5)
    for st, n, _ in parts:
        t += st[:5, G:G + n[2], G:G + n[1], G:G + n[0]].reshape(5, -1).sum(1)
    return t


def shared_face_gap(parts):
    (A, na, _), (B, nb, _) = parts
    fa = A[5, G:G + na[2], G:G + na[1], G + na[0]]
    fb = B[5, G:G + nb[2], G:G + nb[1], G]
    return float(np.abs(fa - fb).max())


def run(orc, perturb, sync):
    pr, dt, pa, pb = setup(orc, perturb)
    parts = [pa, pb]
    t0 = totals(parts)
    regs = step(orc, pr, dt, parts, sync)
    return parts, t0, regs


def test_sync_conserves_and_makes_shared_faces_single_valued(orc):
    parts, t0, regs = run(orc, True, True)
    drift = np.abs(totals(parts) - t0) / np.abs(t0).max()
    assert drift.max() <= 1e-14, drift
    assert shared_face_gap(parts) <= 1e-14
    for P, *_ in regs:
        assert orc.divb_max(P) <= 1e-12
    # without the synchronisation the same perturbed step is not conservative
    parts_u, t0_u, regs_u = run(orc, True, False)
    drift_u = np.abs(totals(parts_u) - t0_u) / np.abs(t0_u).max()
    assert drift_u.max() > 1e-8, drift_u
    assert shared_face_gap(parts_u) > 1e-8
    # the two registers differ at the shared face
    assert np.abs(regs_u[0][6] - regs_u[1][6]).max() > 1e-8


def test_sync_is_a_no_op_when_registers_agree(orc):
    parts_s, _, regs_s = run(orc, False, True)
    parts_u, _, regs_u = run(orc, False, False)
    for k in (6, 7, 8):
        assert np.array_equal(regs_u[0][k], regs_u[1][k])   # R14: one face, one value
    for (a, _, _), (b, _, _) in zip(parts_s, parts_u):
        assert np.array_equal(a, b)
