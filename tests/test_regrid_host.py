"""The library's grid generation for regridding (mhd_cluster_flags, Sec.
2.1) and the overlap lists against the oracle, box for box -- host code
only, no GPU."""
import numpy as np
import pytest

from oracle import cluster as K


@pytest.fixture(scope="module")
def R():
    from paper_1112_1710_gb300 import _build
    _build.build()
    from paper_1112_1710_gb300 import regrid
    return regrid


def _flags(rng, nd):
    shape = tuple(int(v) for v in rng.integers(1, 16 if nd == 3 else 30, nd))
    f = np.zeros(shape, bool)
    for _ in range(rng.integers(0, 5)):
        c = [rng.integers(0, s) for s in shape]
        r = [rng.integers(1, 6) for _ in shape]
        f[tuple(slice(max(0, c[d] - r[d]), min(shape[d], c[d] + r[d])) for d in range(nd))] = True
    return f | (rng.random(shape) < rng.choice([0.0, 0.02, 0.2]))


def test_clustering_equals_oracle(R):
    rng = np.random.default_rng(1112)
    for t in range(300):
        f = _flags(rng, 2 + t % 2)
        eff = float(rng.choice([0.5, 0.7, 0.9, 1.0]))
        ms = int(rng.integers(1, 4))
        assert R.cluster(f, eff, ms) == K.cluster(f, eff, ms)


def test_overlaps_equal_oracle(R):
    rng = np.random.default_rng(5)
    for t in range(60):
        f = _flags(rng, 2 + t % 2)
        new = K.cluster(f)
        old = K.cluster(np.roll(f, int(rng.integers(1, 4)), axis=0))
        for g in (0, 2, 4):
            assert R.overlaps(new, old, g) == K.overlaps(new, old, g)


def test_pins_through_the_library(R):
    f = np.zeros((12, 12), bool)
    f[0:12, 0:4] = True
    f[0:4, 4:12] = True
    assert R.cluster(f) == [((0, 0), (3, 11)), ((4, 0), (11, 3))]
    g = np.zeros((20, 8), bool)
    g[1:5, 2:6] = True
    g[12:18, 1:7] = True
    assert R.cluster(g) == [((1, 2), (4, 5)), ((12, 1), (17, 6))]
    assert R.cluster(np.zeros((4, 4, 4), bool)) == []


def test_cluster_rejects_bad_arguments(R):
    from paper_1112_1710_gb300 import capi
    with pytest.raises(capi.MHDError):
        R.cluster(np.ones((4, 4)), eff=0.0)
    with pytest.raises(capi.MHDError):
        R.cluster(np.ones((4, 4)), min_size=0)
    with pytest.raises(capi.MHDError):
        R.cluster(np.ones(4))


def test_children_are_the_refined_flagged_parent_cells(R):
    # the fine cells are exactly {R c + r : c in (cluster boxes) and in (grids)},
    # each covered once, each child inside one parent grid
    import itertools
    rng = np.random.default_rng(9)
    for t in range(40):
        nd = 2 + t % 2
        shape = (16, 14) if nd == 2 else (10, 9, 8)
        f = rng.random(shape) < 0.15
        clusters = K.cluster(f)
        grids = K.cluster(rng.random(shape) < 0.6, eff=0.6)
        kids = R.children(clusters, grids, 2)
        cells = lambda b: set(itertools.product(*[range(b[0][d], b[1][d] + 1) for d in range(nd)]))
        parents = set().union(*[cells(b) for b in clusters]) & set().union(*[cells(b) for b in grids]) \
            if clusters and grids else set()
        want = {tuple(2 * c[d] + r[d] for d in range(nd)) for c in parents for r in itertools.product((0, 1), repeat=nd)}
        got = set()
        for k in kids:
            ck = cells(k)
            assert not (got & ck)
            got |= ck
            assert any(all(2 * g[0][d] <= k[0][d] and k[1][d] <= 2 * g[1][d] + 1 for d in range(nd)) for g in grids)
        assert got == want


def test_transfer_items_and_masks_equal_oracle():
    """The library's host lists of the data transfer into a new iteration
    (copies of the previous iteration's cells and faces, and the
    prolongation masks) equal the oracle's brute-force ones on random
    coarse-aligned boxes."""
    from oracle import transfer as OT
    from paper_1112_1710_gb300 import regrid
    rng = np.random.default_rng(9)

    def box():
        lo = 2 * rng.integers(0, 12, 3)
        hi = lo + 2 * rng.integers(1, 6, 3) - 1
        return tuple(int(v) for v in lo), tuple(int(v) for v in hi)

    for _ in range(40):
        old = [box() for _ in range(rng.integers(0, 4))]
        new = box()
        got = sorted((it.src, it.kind, tuple(it.box.lo), tuple(it.box.hi)) for it in regrid.transfer_items([new], old))
        want = sorted((j, k, tuple(lo), tuple(hi)) for j, k, lo, hi in OT.copy_items(new, old))
        assert got == want
        m, mlo = regrid.transfer_mask(new, old)
        om, omlo = OT.mask(new, old)
        assert tuple(mlo) == tuple(omlo) and np.array_equal(m, om)


def test_fit_boxes_equals_oracle_and_nests():
    """regrid.fit_boxes (cluster boxes halved until they lie in the nested
    region) against the oracle's fit on random flag fields inside random
    L-shaped regions: the same boxes, each inside the region, together
    covering every flag once."""
    from oracle import cluster as OC
    from oracle import regrid as OR
    from paper_1112_1710_gb300 import regrid
    rng = np.random.default_rng(11)
    for t in range(40):
        shape = tuple(int(v) for v in rng.integers(6, 16, size=3))
        allowed = np.zeros(shape, dtype=bool)
        for _ in range(2):
            lo = [int(rng.integers(0, s // 2)) for s in shape]
            hi = [int(rng.integers(lo[d] + 1, shape[d])) for d in range(3)]
            allowed[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1] = True
        flags = (rng.random(shape) < 0.3) & allowed
        if not flags.any():
            continue
        boxes = OC.cluster(flags, 0.7, 2)
        got = regrid.fit_boxes(boxes, flags, allowed)
        want = OR.fit(boxes, flags, allowed)
        assert [tuple(map(tuple, b)) for b in got] == [tuple(map(tuple, b)) for b in want], t
        cover = np.zeros(shape, dtype=np.int32)
        for lo, hi in got:
            sl = tuple(slice(lo[d], hi[d] + 1) for d in range(3))
            assert allowed[sl].all()
            cover[sl] += 1
        assert cover.max() <= 1 and np.all(cover[flags] == 1)


def test_transfer_masks_of_many_patches_equal_oracle():
    """regrid.transfer_masks (the masks of all new patches read off old
    interiors and face sets painted once) equal the oracle's brute-force
    mask of each new patch."""
    from oracle import transfer as OT
    from paper_1112_1710_gb300 import regrid
    rng = np.random.default_rng(13)

    def box():
        lo = 2 * rng.integers(0, 12, 3)
        hi = lo + 2 * rng.integers(1, 6, 3) - 1
        return tuple(int(v) for v in lo), tuple(int(v) for v in hi)

    for _ in range(30):
        old = [box() for _ in range(rng.integers(0, 6))]
        new = [box() for _ in range(rng.integers(1, 5))]
        got = regrid.transfer_masks(new, old)
        for nb, (m, mlo) in zip(new, got):
            om, omlo = OT.mask(nb, old)
            assert tuple(mlo) == tuple(omlo) and np.array_equal(m, om)
