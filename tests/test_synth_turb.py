"""The deep-AMR input generator: spectrum, Mach number, nesting -- no GPU."""
import numpy as np

import synth.turb as ST


def test_kminus4_field_spectrum_and_mach():
    v = ST.kminus4_velocity(m=32, kmax=8, mach=5.0, seed=5)
    assert abs(np.sqrt((v * v).sum(0).mean()) - 5.0) < 1e-12
    # shell-summed power ~ 4 pi k^2 |v(k)|^2 ~ k^-2 within the band, nothing outside
    vh = np.fft.fftn(v[0])
    k = np.fft.fftfreq(32, d=1.0 / 32)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    assert np.abs(vh[(kk > 8.0) | (kk < 1.0)]).max() < 1e-9 * np.abs(vh).max()
    e = [np.sum(np.abs(vh[(kk >= s - 0.5) & (kk < s + 0.5)]) ** 2) for s in (2, 4, 8)]
    slope = np.polyfit(np.log([2, 4, 8]), np.log(e), 1)[0]
    assert -2.6 < slope < -1.4


def test_deep_hierarchy_nesting_and_sizes():
    H, v, ind = ST.deep_hierarchy(n0=16, levels=4, m=32, size_min=4, size_max=12)
    assert len(H) >= 3
    for lev in range(1, len(H)):
        n = 16 * 2 ** lev
        par = H[lev - 1]
        for (lo, hi) in H[lev]:
            ext = [hi[d] - lo[d] + 1 for d in range(3)]
            assert all(e % 2 == 0 and 4 <= e <= 12 for e in ext) and all(x % 2 == 0 for x in lo)
            # coarsened and grown by the margin: inside one parent, inside the domain
            glo = [lo[d] // 2 - 3 for d in range(3)]
            ghi = [hi[d] // 2 + 3 for d in range(3)]
            assert min(glo) >= 0 and max(ghi) <= n // 2 - 1
            assert any(all(p[0][d] <= glo[d] and ghi[d] <= p[1][d] for d in range(3)) for p in par)
        # disjoint
        boxes = H[lev]
        for i in range(len(boxes)):
            for j in range(i + 1, len(boxes)):
                a, b = boxes[i], boxes[j]
                assert any(a[1][d] < b[0][d] or b[1][d] < a[0][d] for d in range(3))


def test_turb_patch_state():
    v = ST.kminus4_velocity(m=16, kmax=4, mach=5.0, seed=1)
    st, dx = ST.turb_patch((4, 6, 8), (11, 13, 15), 1, 16, 4, v)
    g = 4
    rho = st[0, g:g + 8, g:g + 8, g:g + 8]
    assert np.all(rho == 1.0) and dx == (1.0 / 32,) * 3
    vx = st[1, g:g + 8, g:g + 8, g:g + 8] / rho
    # trilinear sampling: cell (4, 6, 8) of a 32^3 level sits at field coordinates
    # (2.25, 3.25, 4.25) - 0.5 in cell units, i.e. a quarter of the way from
    # field cell (1, 2, 3) to (2, 3, 4) along each axis
    w = (0.25, 0.75)
    want = sum(w[a] * w[b] * w[c] * v[0][3 + c, 2 + b, 1 + a] for a in (0, 1) for b in (0, 1) for c in (0, 1))
    assert abs(vx[0, 0, 0] - want) < 1e-12 * abs(want)
    # a linear field is reproduced exactly away from the periodic seam
    lin = np.zeros((3, 16, 16, 16))
    lin[0] = np.arange(16)[None, None, :] * 0.5
    st2, _ = ST.turb_patch((4, 6, 8), (11, 13, 15), 1, 16, 4, lin)
    x = (np.arange(4, 12) + 0.5) / 32 * 16 - 0.5
    assert np.allclose(st2[1, g, g, g:g + 8], 0.5 * x, atol=1e-12)
    p = (5.0 / 3.0 - 1.0) * (st[4, g:g + 8, g:g + 8, g:g + 8] - 0.5 * (st[1] ** 2 + st[2] ** 2 + st[3] ** 2)[
        g:g + 8, g:g + 8, g:g + 8] - 0.5 * st[5, g:g + 8, g:g + 8, g:g + 8] ** 2)
    assert np.allclose(p, 0.6, rtol=1e-12)
    assert np.allclose(st[5, g:g + 8, g:g + 8, g:g + 9], np.sqrt(1.2))
