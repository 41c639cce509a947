"""The library's host-side Hilbert splitting (mhd_hilbert_split, Sec. 5.2)
against the oracle, element by element, and against the paper's claims --
host code only, no GPU."""
import itertools
import random

import numpy as np
import pytest

from oracle import hilbert as H


@pytest.fixture(scope="module")
def PH():
    from paper_1112_1710_gb300 import _build
    _build.build()
    from paper_1112_1710_gb300 import hilbert
    return hilbert


def test_split_equals_oracle_on_random_boxes(PH):
    rnd = random.Random(1710)
    for _ in range(400):
        n = rnd.choice((2, 3))
        ext = [rnd.randint(1, 24) for _ in range(n)]
        lo = tuple(rnd.randint(0, 9) for _ in range(n))
        hi = tuple(lo[d] + ext[d] - 1 for d in range(n))
        k = rnd.randint(1, min(9, int(np.prod(ext))))
        w = [rnd.choice([1.0, rnd.uniform(0.05, 3.0)]) for _ in range(k)]
        g = rnd.choice((0, 2, 4))
        bits = H.bits_for(max(hi) + 1)
        try:
            want = H.hilbert_split(lo, hi, w, bits, g)
        except ValueError:
            want = None
        if want is None:
            with pytest.raises(Exception):
                PH.split(lo, hi, w, bits, g)
        else:
            assert PH.split(lo, hi, w, bits, g) == want, (lo, hi, w, g)


def test_paper_claims_through_the_library(PH):
    pieces = PH.split((0, 0), (15, 15), [1.0] * 5, 4)
    sizes = sorted((b[0] - a[0] + 1) * (b[1] - a[1] + 1) for a, b in pieces)
    assert sizes == [48, 48, 50, 55, 55]
    for n, bits, lev in [(2, 5, 2), (3, 3, 2), (3, 4, 1)]:
        side = 1 << bits
        pieces = PH.split((0,) * n, (side - 1,) * n, [1.0] * (1 << (n * lev)), bits)
        per = 1 << (n * (bits - lev))
        for j, (a, b) in enumerate(pieces):
            idx = {H.hilbert_index(c, bits) for c in itertools.product(*[range(a[d], b[d] + 1) for d in range(n)])}
            assert idx == set(range(j * per, (j + 1) * per))


def test_split_rejects_bad_arguments(PH):
    from paper_1112_1710_gb300 import capi
    for args in [((0, 0), (3, 3), [1.0, -1.0], 2), ((0, 0), (3, 3), [1.0, float("nan")], 2),
                 ((0, 0), (0, 0), [1.0, 1.0], 2), ((0, 0), (3, 3), [1.0], 1), ((2, 0), (1, 3), [1.0], 2)]:
        with pytest.raises(capi.MHDError):
            PH.split(*args)
    assert PH.split((0, 0), (0, 0), [1.0], 0) == [((0, 0), (0, 0))]


def test_global_offsets():
    from paper_1112_1710_gb300.hilbert import global_offsets
    assert list(global_offsets([7, 0, 13, 20])) == H.global_index([7, 0, 13, 20])
