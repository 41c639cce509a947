"""The Hilbert ordering and splitting oracle (Sec. 5.1, 5.2) pinned to the
curve's defining properties and to the paper's claims about the splitting:
no GPU."""
import itertools
import random

import pytest

from oracle import hilbert as H


def _adjacent(a, b):
    return sum(abs(a[d] - b[d]) for d in range(len(a))) == 1


@pytest.mark.parametrize("n,bits", [(2, 1), (2, 2), (2, 3), (2, 5), (3, 1), (3, 2), (3, 3)])
def test_index_is_a_curve_through_face_neighbours(n, bits):
    seen = {}
    for c in itertools.product(range(1 << bits), repeat=n):
        h = H.hilbert_index(c, bits)
        assert 0 <= h < 1 << (n * bits)
        assert h not in seen
        seen[h] = c
    assert len(seen) == 1 << (n * bits)
    order = [seen[h] for h in range(1 << (n * bits))]
    for a, b in zip(order, order[1:]):
        assert _adjacent(a, b), (a, b)


@pytest.mark.parametrize("n,bits", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_children_follow_their_parents(n, bits):
    # Sec. 5.1: the 2^n children of a cell take one contiguous block of
    # indices, and the blocks in order visit the parents along a curve of
    # face neighbours, so child order follows parent order
    block = {}
    for c in itertools.product(range(1 << bits), repeat=n):
        parent = tuple(v >> 1 for v in c)
        blk = H.hilbert_index(c, bits) >> n
        assert block.setdefault(parent, blk) == blk
    assert sorted(block.values()) == list(range(1 << (n * (bits - 1))))
    parents = sorted(block, key=block.get)
    for a, b in zip(parents, parents[1:]):
        assert _adjacent(a, b)


def test_start_cell_and_one_bit_curve():
    # the curve starts at the origin; on the 2 x 2 square it is the U through
    # the four cells
    assert H.hilbert_index((0, 0), 3) == 0
    assert H.hilbert_index((0, 0, 0), 3) == 0
    assert [H.curve(2, 1)[k] for k in range(4)][0] == (0, 0)
    assert _adjacent(H.curve(2, 1)[0], H.curve(2, 1)[3])


def test_weight_list_split_of_the_paper():
    # Sec. 5.2 step 1: [.1 .2 .1 .3 .3] -> [.1 .2 .1] and [.3 .3]
    assert H.split_weights([.1, .2, .1, .3, .3]) == ([.1, .2, .1], [.3, .3])
    assert H.split_weights([1, 1, 1, 1, 1]) == ([1, 1], [1, 1, 1])


def _cells(box):
    lo, hi = box
    return set(itertools.product(*[range(lo[d], hi[d] + 1) for d in range(len(lo))]))


def _check_partition(box, pieces):
    allc = _cells(box)
    got = set()
    for p in pieces:
        c = _cells(p)
        assert not (got & c)
        got |= c
    assert got == allc


def test_sixteen_by_sixteen_on_five():
    # Sec. 6: a 16 x 16 grid over five equal shares leaves one piece with 55
    # cells, 93% of the ideal 51.2
    box = ((0, 0), (15, 15))
    pieces = H.hilbert_split(box[0], box[1], [1.0] * 5, bits=4)
    _check_partition(box, pieces)
    sizes = [len(_cells(p)) for p in pieces]
    assert max(sizes) == 55
    assert sorted(sizes) == [48, 48, 50, 55, 55]
    assert abs(256 / 5 / max(sizes) - 0.93) < 0.005


@pytest.mark.parametrize("n,bits,levels", [(2, 4, 1), (2, 4, 2), (2, 4, 3), (2, 5, 2), (3, 3, 1), (3, 3, 2)])
def test_equal_shares_trace_the_hilbert_curve(n, bits, levels):
    # Sec. 5.2: a square (cube) over 4^k (8^k) equal shares yields a
    # distribution that traces a level-k Hilbert curve: piece j is the j-th
    # block of 2^(n (bits - k)) consecutive curve indices
    side = 1 << bits
    box = ((0,) * n, (side - 1,) * n)
    P = 1 << (n * levels)
    pieces = H.hilbert_split(box[0], box[1], [1.0] * P, bits=bits)
    _check_partition(box, pieces)
    per = 1 << (n * (bits - levels))
    for j, p in enumerate(pieces):
        idx = {H.hilbert_index(c, bits) for c in _cells(p)}
        assert idx == set(range(j * per, (j + 1) * per)), j


def test_random_boxes_are_partitioned_in_proportion():
    rnd = random.Random(1112)
    for _ in range(30):
        n = rnd.choice((2, 3))
        ext = [rnd.randint(2, 12) for _ in range(n)]
        lo = tuple(rnd.randint(0, 3) for _ in range(n))
        hi = tuple(lo[d] + ext[d] - 1 for d in range(n))
        k = rnd.randint(1, min(6, ext[0] * ext[1]))
        w = [rnd.uniform(0.2, 1.0) for _ in range(k)]
        pieces = H.hilbert_split(lo, hi, w, bits=H.bits_for(max(hi) + 1))
        assert len(pieces) == k
        _check_partition((lo, hi), pieces)


def test_order_boxes_and_global_index():
    boxes = [((8, 8), (15, 15)), ((0, 0), (7, 7)), ((0, 8), (7, 15)), ((8, 0), (15, 7))]
    order = H.order_boxes(boxes, 4)
    keys = [H.box_distance(*boxes[i], 4) for i in order]
    assert keys == sorted(keys)
    # quadrant blocks of the 16 x 16 curve: the order is the curve's
    first = [H.hilbert_index(boxes[i][0], 4) >> 6 for i in order]
    assert first == [0, 1, 2, 3]
    # strict grouping: items sorted by key and dealt to holders in runs get
    # global index = local index + the counts of lower holders
    keys = sorted(random.Random(5).sample(range(1000), 40))
    counts = [7, 0, 13, 20]
    off = H.global_index(counts)
    assert off == [0, 7, 7, 20]
    pos = 0
    for hdr, c in enumerate(counts):
        for li in range(c):
            assert off[hdr] + li == pos
            pos += 1
