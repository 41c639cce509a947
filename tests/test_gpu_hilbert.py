"""Hilbert keys and grid distances on the device (mhd_hilbert_keys,
mhd_box_distances; Sec. 5.1) against the oracle, bit for bit, and the
curve's properties at full size."""
import itertools
import random

import pytest
import torch

from oracle import hilbert as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def PH():
    from paper_1112_1710_gb300 import _build
    _build.build()
    from paper_1112_1710_gb300 import hilbert
    return hilbert


def _u64(t):
    return [int(v) & ((1 << 64) - 1) for v in t.cpu().tolist()]


@pytest.mark.parametrize("n,bits", [(2, 5), (3, 3), (2, 0), (3, 1)])
def test_keys_of_every_cell_equal_oracle(PH, n, bits):
    cells = list(itertools.product(range(1 << bits), repeat=n))
    pts = torch.tensor(cells, dtype=torch.int32, device="cuda")
    got = _u64(PH.keys(pts, bits))
    assert got == [H.hilbert_index(c, bits) for c in cells]


@pytest.mark.parametrize("n,bits", [(2, 30), (3, 20), (3, 11), (2, 17)])
def test_keys_of_random_points_equal_oracle(PH, n, bits):
    rnd = random.Random(bits * 10 + n)
    pts = [tuple(rnd.randrange(1 << bits) for _ in range(n)) for _ in range(3000)]
    # corners of the domain and points just outside it
    pts += [(0,) * n, ((1 << bits) - 1,) * n]
    bad = [(-1,) + (0,) * (n - 1), (1 << bits,) + (0,) * (n - 1)]
    got = _u64(PH.keys(torch.tensor(pts + bad, dtype=torch.int32, device="cuda"), bits))
    assert got[:len(pts)] == [H.hilbert_index(p, bits) for p in pts]
    assert got[len(pts):] == [(1 << 64) - 1] * 2


def test_box_distances_equal_oracle(PH):
    rnd = random.Random(3)
    for n, bits in [(2, 6), (3, 5), (3, 20)]:
        boxes = []
        for _ in range(500):
            lo = [rnd.randrange(1 << bits) for _ in range(n)]
            hi = [min((1 << bits) - 1, v + rnd.randrange(1 << min(bits, 6))) for v in lo]
            boxes.append((tuple(lo), tuple(hi)))
        boxes.append(((2,) * n, (1,) * n))  # empty
        boxes.append(((0,) * n, (1 << bits,) * n))  # leaves the domain
        lo = torch.tensor([b[0] for b in boxes], dtype=torch.int32, device="cuda")
        hi = torch.tensor([b[1] for b in boxes], dtype=torch.int32, device="cuda")
        got = PH.box_distances(lo, hi, bits).cpu().tolist()
        assert got[:-2] == [H.box_distance(a, b, bits) for a, b in boxes[:-2]]
        assert got[-2:] == [2 ** 63 - 1] * 2


def test_order_of_the_amr_hierarchy_equals_oracle(PH):
    import synth.amr as SA
    Hh = SA.shell_hierarchy(n0=64, levels=4, seed=42, size_min=8, size_max=64)
    perms = PH.hilbert_order_hierarchy(Hh, 64)
    for l, bl in enumerate(Hh):
        assert list(perms[l]) == H.order_boxes(bl, H.bits_for(64 << l))


def test_full_grid_keys_are_a_face_neighbour_curve(PH):
    # every cell of a 256^3 grid (16.8 M points): the keys are a permutation
    # of [0, 2^24) and consecutive keys sit on face neighbours
    bits, side = 8, 256
    ax = torch.arange(side, dtype=torch.int32, device="cuda")
    z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
    pts = torch.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], 1).contiguous()
    k = PH.keys(pts, bits)
    order = torch.argsort(k)
    assert torch.equal(k[order], torch.arange(side ** 3, dtype=torch.int64, device="cuda"))
    steps = (pts[order[1:]].to(torch.int64) - pts[order[:-1]].to(torch.int64)).abs().sum(1)
    assert bool((steps == 1).all())
