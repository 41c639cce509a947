"""Oracle of the space-filling-curve ordering and the Hilbert splitting of
grids (Sec. 5.1 grid assignments, Sec. 5.2 Hilbert splitting).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's baseline legs, never by the product.  Plain Python integers and
floats, one cell or one candidate at a time.

Hilbert index.  The index of a cell (x_0, ..., x_{n-1}), each coordinate
below 2^b, is Skilling's transposed-axes construction (J. Skilling,
"Programming the Hilbert curve", AIP Conf. Proc. 707, 381 (2004)), restated
here: undo the excess work of the rotations from the top bit down (at bit Q,
a set bit of x_i inverts the lower bits of x_0, a clear one exchanges the
lower bits of x_0 and x_i), Gray-encode across the axes, fix the parity, then
read the index off the transposed bits, top bit of x_0 first.  Pinned by the
curve's own properties: every index taken once, consecutive indices on
face-adjacent cells, and the nesting of Sec. 5.1 (the children of a cell
occupy one contiguous block of 2^n indices, so that child order follows
parent order).

Distance of a grid along the curve (Sec. 5.1 lets a grid's position on the
curve be taken from a sample of its cells, its corners for instance): the
sum of the indices of its 2^n corner cells (the mean times 2^n; only
differences and order are used).

Hilbert splitting (Sec. 5.2), readings where the text leaves the detail
open (each also listed with the design notes):
  1. the weight list is cut into a prefix and a suffix whose sums (added
     in list order) differ least; ties go to the shorter prefix;
  2. a candidate split cuts one axis of extent >= 2 at an integer position
     next to the proportional point (floor and ceiling of share * extent,
     kept inside [1, extent - 1]), with the prefix's piece on the low side or
     on the high side;
  3. its cost is the slower piece's advance time per unit of weight: max
     over the two pieces of cells(piece grown by g ghost layers) / share,
     the share being the piece's part of the weight sum;
  4. candidates within a factor 1 + COMPARABLE of the least cost are
     comparable; among them the one whose suffix piece lies furthest ahead of
     the prefix piece along the curve (largest corner-sum difference) wins,
     then the first in enumeration order (axis, prefix side low before
     high, cut position ascending);
  5. the two pieces are split again with their weight lists until every
     list has one weight.
The pieces come back in weight-list order.  Pinned by the paper's claims: a
square (cube) split over 4^n (8^n) equal weights traces a level-n Hilbert
curve, and the 16 x 16 grid on five equal weights leaves at most 55 cells on
one piece (Sec. 6).
"""
from __future__ import annotations

import itertools

COMPARABLE = 0.01


def hilbert_index(x, bits):
    """Hilbert index of the cell with integer coordinates x (a sequence of n
    values in [0, 2^bits)), in [0, 2^(n bits))."""
    X = [int(v) for v in x]
    n = len(X)
    if bits == 0:
        return 0
    for v in X:
        if v < 0 or v >= (1 << bits):
            raise ValueError("coordinate outside [0, 2^bits)")
    M = 1 << (bits - 1)
    Q = M
    while Q > 1:
        P = Q - 1
        for i in range(n):
            if X[i] & Q:
                X[0] ^= P
            else:
                t = (X[0] ^ X[i]) & P
                X[0] ^= t
                X[i] ^= t
        Q >>= 1
    for i in range(1, n):
        X[i] ^= X[i - 1]
    t = 0
    Q = M
    while Q > 1:
        if X[n - 1] & Q:
            t ^= Q - 1
        Q >>= 1
    for i in range(n):
        X[i] ^= t
    h = 0
    for j in range(bits - 1, -1, -1):
        for i in range(n):
            h = (h << 1) | ((X[i] >> j) & 1)
    return h


def bits_for(extent):
    """Smallest b with 2^b >= extent (the curve resolution of a domain)."""
    b = 0
    while (1 << b) < extent:
        b += 1
    return b


def box_corners(lo, hi):
    """The 2^n corner cells of the inclusive box [lo, hi]."""
    return [tuple(hi[d] if (k >> d) & 1 else lo[d] for d in range(len(lo))) for k in range(1 << len(lo))]


def box_distance(lo, hi, bits):
    """Distance of a grid along the curve: the sum of its corner cells'
    indices (Sec. 5.1)."""
    return sum(hilbert_index(c, bits) for c in box_corners(lo, hi))


def order_boxes(boxes, bits):
    """Indices of `boxes` ((lo, hi) pairs) sorted by their distance along the
    curve, ties by position in the list (Sec. 5.1)."""
    keys = [box_distance(lo, hi, bits) for lo, hi in boxes]
    return sorted(range(len(boxes)), key=lambda i: (keys[i], i))


def global_index(local_counts):
    """Sec. 5.1: the global sort index of an item is its local index plus the
    item counts of all lower-numbered holders.  Returns the offsets (the
    exclusive prefix sums of local_counts)."""
    out, acc = [], 0
    for c in local_counts:
        out.append(acc)
        acc += int(c)
    return out


def wsum(ws):
    """Sum of a weight list added in list order, one rounding per addition
    (Python's built-in sum() compensates the rounding of float sums)."""
    s = 0.0
    for v in ws:
        s = s + v
    return s


def split_weights(weights):
    """Step 1: (prefix, suffix) of the weight list with the least difference
    of sums, ties to the shorter prefix."""
    best, cut = None, 1
    for k in range(1, len(weights)):
        a = wsum(weights[:k])
        b = wsum(weights[k:])
        dif = abs(a - b)
        if best is None or dif < best:
            best, cut = dif, k
    return list(weights[:cut]), list(weights[cut:])


def advance_cost(lo, hi, g):
    """Cells of the box grown by g ghost layers on every side."""
    c = 1
    for d in range(len(lo)):
        c *= hi[d] - lo[d] + 1 + 2 * g
    return c


def split_candidates(lo, hi, wa, wb):
    """Step 2: (axis, prefix piece on the high side?, cut) in enumeration
    order; the cut is the extent of the low piece along the axis."""
    tot = wsum(wa) + wsum(wb)
    out = []
    for d in range(len(lo)):
        L = hi[d] - lo[d] + 1
        if L < 2:
            continue
        for high in (False, True):
            share_low = (wsum(wb) if high else wsum(wa)) / tot
            pos = share_low * L
            cuts = sorted({min(max(int(pos // 1), 1), L - 1), min(max(-int((-pos) // 1), 1), L - 1)})
            for c in cuts:
                out.append((d, high, c))
    return out


def cut_box(lo, hi, d, c):
    """Low and high pieces of the box cut after c cells along axis d."""
    lo_hi = list(hi)
    lo_hi[d] = lo[d] + c - 1
    hi_lo = list(lo)
    hi_lo[d] = lo[d] + c
    return (tuple(lo), tuple(lo_hi)), (tuple(hi_lo), tuple(hi))


def hilbert_split(lo, hi, weights, bits, g=2):
    """Steps 1-5: boxes (lo, hi), one per weight, in weight order."""
    lo, hi = tuple(lo), tuple(hi)
    if len(weights) == 1:
        return [(lo, hi)]
    wa, wb = split_weights(weights)
    tot = wsum(wa) + wsum(wb)
    sa, sb = wsum(wa) / tot, wsum(wb) / tot
    cands = []
    for d, high, c in split_candidates(lo, hi, wa, wb):
        low_box, high_box = cut_box(lo, hi, d, c)
        pa, pb = (high_box, low_box) if high else (low_box, high_box)
        cost = max(advance_cost(pa[0], pa[1], g) / sa, advance_cost(pb[0], pb[1], g) / sb)
        gain = box_distance(pb[0], pb[1], bits) - box_distance(pa[0], pa[1], bits)
        cands.append((cost, gain, pa, pb))
    if not cands:
        raise ValueError("box of one cell cannot be split over %d weights" % len(weights))
    least = min(c[0] for c in cands)
    best = None
    for cost, gain, pa, pb in cands:
        if cost <= least * (1.0 + COMPARABLE) and (best is None or gain > best[1]):
            best = (cost, gain, pa, pb)
    _, _, pa, pb = best
    return hilbert_split(pa[0], pa[1], wa, bits, g) + hilbert_split(pb[0], pb[1], wb, bits, g)


def curve(n, bits):
    """All cells of [0, 2^bits)^n in curve order (brute force)."""
    cells = list(itertools.product(range(1 << bits), repeat=n))
    return sorted(cells, key=lambda c: hilbert_index(c, bits))
