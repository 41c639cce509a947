"""The clustering oracle (grid generation of Sec. 2.1 regridding, by the
Berger-Rigoutsos point clustering the paper's citations lead to) pinned to
what the algorithm must produce -- no GPU."""
import itertools

import numpy as np
import pytest

from oracle import cluster as K


def _cells(b):
    lo, hi = b
    return set(itertools.product(*[range(lo[d], hi[d] + 1) for d in range(len(lo))]))


def _check(flags, boxes, eff, min_size):
    fl = {tuple(int(v) for v in c) for c in np.argwhere(flags)}
    got = set()
    for b in boxes:
        c = _cells(b)
        assert not (got & c), "boxes overlap"
        got |= c
        n = sum(1 for x in c if x in fl)
        ext = [b[1][d] - b[0][d] + 1 for d in range(len(b[0]))]
        assert n >= eff * len(c) or max(ext) < 2 * min_size, (b, n, len(c))
        # shrunk to the flags: every face of the box touches a flagged cell
        for d in range(len(ext)):
            for side in (b[0][d], b[1][d]):
                assert any(x[d] == side for x in c if x in fl)
    assert fl <= got


def test_empty_and_solid_blocks():
    f = np.zeros((12, 10), bool)
    assert K.cluster(f) == []
    f[3:9, 2:7] = True
    assert K.cluster(f) == [((3, 2), (8, 6))]
    g = np.zeros((8, 9, 10), bool)
    g[1:4, 2:9, 5:6] = True
    assert K.cluster(g) == [((1, 2, 5), (3, 8, 5))]


def test_separated_blocks_are_cut_at_the_gap():
    f = np.zeros((20, 8), bool)
    f[1:5, 2:6] = True
    f[12:18, 1:7] = True
    assert K.cluster(f) == [((1, 2), (4, 5)), ((12, 1), (17, 6))]


def test_l_shape_is_cut_at_its_corner():
    # two blocks forming an L, 80 flags in a 12 x 12 bounding box (0.56 < 0.7):
    # the signatures' second differences change sign at the corner
    f = np.zeros((12, 12), bool)
    f[0:12, 0:4] = True
    f[0:4, 4:12] = True
    sig = K.signature(f, (0, 0), (11, 11), 0)
    assert sig == [12] * 4 + [4] * 8
    boxes = K.cluster(f)
    assert boxes == [((0, 0), (3, 11)), ((4, 0), (11, 3))]
    _check(f, boxes, 0.7, 2)


def test_efficiency_threshold_controls_the_cut():
    f = np.zeros((12, 12), bool)
    f[0:12, 0:4] = True
    f[0:4, 4:12] = True
    assert K.cluster(f, eff=0.5) == [((0, 0), (11, 11))]


@pytest.mark.parametrize("nd", [2, 3])
def test_random_flags_are_covered_by_disjoint_efficient_boxes(nd):
    rng = np.random.default_rng(11 + nd)
    shape = (24, 20) if nd == 2 else (14, 12, 10)
    for trial in range(8):
        # blobs of flags plus sparse noise
        f = np.zeros(shape, bool)
        for _ in range(rng.integers(1, 5)):
            c = [rng.integers(0, s) for s in shape]
            r = [rng.integers(1, 5) for _ in shape]
            sl = tuple(slice(max(0, c[d] - r[d]), min(shape[d], c[d] + r[d])) for d in range(nd))
            f[sl] = True
        f |= rng.random(shape) < 0.01
        for eff, ms in [(0.7, 2), (0.9, 1), (0.5, 3)]:
            _check(f, K.cluster(f, eff=eff, min_size=ms), eff, ms)


def test_overlaps_between_iterations():
    old = [((0, 0), (7, 7)), ((8, 0), (15, 7))]
    new = [((4, 2), (11, 5)), ((20, 20), (23, 23))]
    assert K.overlaps(new, old) == [(0, 0, ((4, 2), (7, 5))), (0, 1, ((8, 2), (11, 5)))]
    # with the new grid's ghost region
    assert K.overlaps(new, old, grow=2)[0] == (0, 0, ((2, 0), (7, 7)))
    assert K.overlaps(new, old, grow=4)[-1][0] == 0
