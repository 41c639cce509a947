"""Pins of the oracle's regridding step of a finest level (oracle/regrid.py,
Sec. 2.1 and the O step of Sec. 2.2): the grown and nested flag masks
against a cell-by-cell brute force, and on a blast-shell hierarchy after one
coarse step: the new grids are aligned, disjoint, each inside one parent
grid, properly nested, and cover every kept flag; the new patches hold the
old iteration's data where they meet it; a threshold that flags nothing
drops the level."""
import itertools

import numpy as np
import pytest

import synth
import synth.amr as SA

G = 4


def _brute_grow(m, r):
    out = np.zeros_like(m)
    for z, y, x in itertools.product(*[range(s) for s in m.shape]):
        out[z, y, x] = m[max(0, z - r):z + r + 1, max(0, y - r):y + r + 1, max(0, x - r):x + r + 1].any()
    return out


def _brute_inner(m, r):
    out = np.zeros_like(m)
    nz, ny, nx = m.shape
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if z - r < 0 or y - r < 0 or x - r < 0 or z + r >= nz or y + r >= ny or x + r >= nx:
            continue
        out[z, y, x] = m[z - r:z + r + 1, y - r:y + r + 1, x - r:x + r + 1].all()
    return out


def test_cube_masks_equal_brute_force():
    from oracle import regrid as R
    rng = np.random.default_rng(5)
    for shape, r in (((7, 9, 11), 1), ((8, 6, 10), 2), ((12, 12, 12), 3)):
        m = rng.random(shape) < 0.15
        assert np.array_equal(R._cube_or(m, r), _brute_grow(m, r))
        m2 = rng.random(shape) < 0.9
        m2[2:-2, 2:-2, 2:-2] = True
        assert np.array_equal(R._cube_and(m2, r), _brute_inner(m2, r))


@pytest.fixture(scope="module")
def stepped(orc):
    from oracle.amr import OHierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=2, size_min=4, size_max=8)
    st = [[SA.blast_patch(lo, hi, l, n0, G, p_in=10.0)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
    oh.initialise()
    oh.coarse_step()
    return oh, H


def _empty(n, g):
    return synth.empty_patch(n, g)


def test_regrid_grids_nested_and_cover_the_flags(orc, stepped):
    from oracle import regrid as R
    oh, H = stepped
    n0, margin, buf = 16, 3, 1
    old = [(P.lo, P.hi, P.state.copy()) for P in oh.levels[1]]
    flags = R.flags_of_parent(oh, 0.05)
    boxes, states, nfall = R.regrid_finest(oh, 0.05, buffer=buf, margin=margin, empty=_empty)
    assert boxes[0] == H[0] and len(boxes) == 2 and len(boxes[1]) > 0 and nfall == 0
    new = boxes[1]
    # kept flags at the parent resolution, from a brute force of the rules
    f = np.zeros((n0,) * 3, dtype=bool)
    f[:, :, :] = flags[0].astype(bool)                 # the one base grid covers the domain
    kept = _brute_grow(f, buf) & _brute_inner(np.ones_like(f), margin)
    assert kept.any() and not kept.all()
    cover = np.zeros((2 * n0,) * 3, dtype=np.int32)
    for lo, hi in new:
        assert all(lo[d] % 2 == 0 and hi[d] % 2 == 1 for d in range(3))
        # properly nested: margin parent cells inside the domain
        assert all(lo[d] // 2 >= margin and hi[d] // 2 <= n0 - 1 - margin for d in range(3))
        cover[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += 1
    assert cover.max() == 1                           # disjoint
    # every kept flag is covered (at the fine resolution, all 8 children)
    kz, ky, kx = np.nonzero(kept)
    assert np.all(cover[2 * kz, 2 * ky, 2 * kx] == 1) and np.all(cover[2 * kz + 1, 2 * ky + 1, 2 * kx + 1] == 1)
    # where a new patch meets an old one, it holds the old cells
    met = 0
    for (lo, hi), st in zip(new, states[1]):
        for olo, ohi, ost in old:
            a = [max(lo[d], olo[d]) for d in range(3)]
            b = [min(hi[d], ohi[d]) for d in range(3)]
            if any(a[d] > b[d] for d in range(3)):
                continue
            met += 1
            sl_n = tuple(slice(a[d] - lo[d] + G, b[d] - lo[d] + G + 1) for d in (2, 1, 0))
            sl_o = tuple(slice(a[d] - olo[d] + G, b[d] - olo[d] + G + 1) for d in (2, 1, 0))
            for q in range(5):
                assert np.array_equal(st[q][sl_n], ost[q][sl_o])
    assert met > 0


def test_regrid_without_flags_drops_the_level(orc, stepped):
    from oracle import regrid as R
    oh, H = stepped
    boxes, states, nfall = R.regrid_finest(oh, 2.0, empty=_empty)   # a normalised difference never exceeds 1
    assert len(boxes) == 1 and boxes[0] == H[0] and nfall == 0


def test_regrid_levels_nest_each_new_level(orc):
    """Regridding levels 1 and 2 of a 3-level hierarchy: level 1 from the
    base's flags, then level 2 from the new level 1's; every new level-2
    grid lies at least `margin` level-1 cells inside the new level 1."""
    from oracle import regrid as R
    from oracle.amr import OHierarchy
    n0, margin = 16, 3
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    st = [[SA.blast_patch(lo, hi, l, n0, G, p_in=10.0)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
    oh.initialise()
    oh.coarse_step()
    boxes, states, nfall = R.regrid_levels(oh, 0.02, first=1, margin=margin, empty=_empty)
    assert len(boxes) == 3 and boxes[0] == H[0] and nfall == 0
    assert all(len(b) > 0 for b in boxes)
    n1 = 2 * n0
    inside = np.zeros((n1,) * 3, dtype=bool)
    for lo, hi in boxes[1]:
        inside[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
    ok = _brute_inner(inside, margin)
    for lo, hi in boxes[2]:
        c = [(lo[d] // 2, hi[d] // 2) for d in range(3)]
        assert ok[c[2][0]:c[2][1] + 1, c[1][0]:c[1][1] + 1, c[0][0]:c[0][1] + 1].all()
