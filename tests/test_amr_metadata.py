"""The product's AMR metadata (ghost copies, prolongation and restriction
items, flux-register captures and deposits) equals the oracle's, which is
generated independently by brute-force box intersection -- no GPU."""
import pytest

import synth.amr as SA

G = 4


@pytest.mark.parametrize("split", [1, 2])
def test_amr_metadata_equals_oracle(orc, split):
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8, level0_split=split)
    states = [[SA.blast_patch(lo, hi, l, n0, G)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, states, (1.0 / n0,) * 3, g=G)
    ph = Hierarchy(H, n0, states, (1.0 / n0,) * 3, g=G, dtype="f64", device="cpu")
    tup = lambda b: (tuple(int(v) for v in b.lo), tuple(int(v) for v in b.hi))
    for l in range(3):
        mine = sorted((c.src, c.dst, tup(c.box), tuple(c.offset)) for c in ph.copy_lists[l])
        theirs = sorted((s, d, (tuple(b[0]), tuple(b[1])), tuple(o)) for (s, d, b, o) in oh.copy_lists[l])
        assert mine == theirs
    for l in range(2):
        mine = sorted((p.coarse, p.fine, tup(p.box)) for p in ph.prolong_lists[l])
        theirs = sorted((c, f, (tuple(b[0]), tuple(b[1]))) for (c, f, b) in oh.prolong_lists[l])
        assert mine == theirs
        mine = sorted((r.fine, r.coarse, tup(r.box)) for r in ph.restrict_lists[l])
        theirs = sorted((f, c, (tuple(b[0]), tuple(b[1]))) for (f, c, b) in oh.restrict_lists[l])
        assert mine == theirs
    # captures: (level, patch, kind, axis, box)
    kinds = {"face": 0, "edge": 1}
    for l in range(3):
        mine = sorted((int(p), k, a, tuple(int(v) for v in lo), tuple(int(v) for v in hi))
                      for (p, k, a, lo, hi, r) in ph.fine_caps[l] + ph.coarse_caps[l])
        theirs = sorted((pi, kinds[k], a, tuple(b[0]), tuple(b[1]))
                        for pi, lst in oh.cap[l].items() for (k, a, b, key) in lst)
        assert mine == theirs
    for l in range(2):
        mine = sorted((int(c), k, a, tuple(int(v) for v in lo), tuple(int(v) for v in hi),
                       tuple(int(v) for v in flo), tuple(int(v) for v in fhi))
                      for (c, k, a, lo, hi, rf, flo, fhi, rc) in ph.deposit_list[l])
        theirs = sorted((c, kinds[k], a, tuple(b[0]), tuple(b[1]), tuple(oh.reg[fk]["lo"]), tuple(oh.reg[fk]["hi"]))
                        for (k, c, a, b, fk, ck) in oh.dep[l])
        assert mine == theirs
