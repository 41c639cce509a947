"""The AMR tree on the device (Sec. 3.1: the neighbours of a node's children
are children of the node's neighbours).  The interactions it inherits level
by level equal a brute-force search over every pair of patches and every
periodic shift, and the metadata built from it (ghost copies, prolongation
and restriction items, flux-register captures and deposits) equals the
metadata built by testing every pair, element by element and in the same
order; on the small hierarchy both equal the oracle's lists."""
import itertools

import numpy as np
import pytest

import synth.amr as SA
import synth.turb as ST

pytestmark = pytest.mark.gpu
G = 4


def brute_interactions(boxes, n0, l, r):
    """{(c, c2, shift)}: box(c2) shifted by shift periodic lengths meets box(c)
    grown by r (numpy over all pairs and shifts)."""
    lo = np.array([b[0] for b in boxes[l]], np.int64)
    hi = np.array([b[1] for b in boxes[l]], np.int64)
    n = n0 * 2 ** l
    out = set()
    for s in itertools.product((-1, 0, 1), repeat=3):
        sh = np.array(s) * n
        meet = np.all((lo[None, :, :] + sh <= hi[:, None, :] + r) & (hi[None, :, :] + sh >= lo[:, None, :] - r), axis=2)
        for c, c2 in zip(*np.nonzero(meet)):
            out.add((int(c), int(c2), s))
    return out


def hierarchies():
    yield "shell 16^3, 3 levels", SA.shell_hierarchy(n0=16, levels=3, size_min=4, size_max=8), 16
    yield "shell 16^3 split 2, 3 levels", SA.shell_hierarchy(n0=16, levels=3, size_min=4, size_max=8,
                                                             level0_split=2), 16
    H, _, _ = ST.deep_hierarchy(n0=16, levels=4, m=32, size_min=4, size_max=12)
    yield "turbulence 16^3, 4 levels", H, 16
    yield "shell 64^3, 4 levels (the AMR bench workload)", SA.shell_hierarchy(n0=64, levels=4, seed=42,
                                                                              size_min=8, size_max=64), 64


@pytest.mark.parametrize("case", range(4))
def test_inherited_interactions_equal_brute_force(case):
    from paper_1112_1710_gb300.tree import DeviceTree
    name, H, n0 = list(hierarchies())[case]
    t = DeviceTree(H, n0, G + 1, device="cuda")
    for l in range(len(H)):
        off, idx, s = t.inter[l]
        mine = [(c, int(idx[k]), tuple(int(v) for v in s[k])) for c in range(len(H[l])) for k in range(off[c], off[c + 1])]
        assert len(mine) == len(set(mine)), (name, l)
        assert set(mine) == brute_interactions(H, n0, l, G + 1), (name, l)
        # canonical order: per patch by (shift rank, partner)
        for c in range(len(H[l])):
            keys = [((sv[0] + 1) * 9 + (sv[1] + 1) * 3 + sv[2] + 1, int(p))
                    for p, sv in zip(idx[off[c]:off[c + 1]], s[off[c]:off[c + 1]])]
            assert keys == sorted(keys)
        if l:
            po, pi = t.parents[l]
            clo = np.array([b[0] for b in H[l - 1]])
            chi = np.array([b[1] for b in H[l - 1]])
            for f, (lo, hi) in enumerate(H[l]):
                cl, ch = np.array(lo) // 2, np.array(hi) // 2
                want = np.nonzero(np.all((clo <= ch) & (chi >= cl), axis=1))[0]
                assert list(pi[po[f]:po[f + 1]]) == list(want)


def _meta(h):
    tup = lambda b: (tuple(int(v) for v in b.lo), tuple(int(v) for v in b.hi))
    arr = lambda a: tuple(int(v) for v in a)
    out = {"copies": [[(c.src, c.dst, tup(c.box), tuple(c.offset)) for c in cl] for cl in h.copy_lists],
           "prolong": [[(p.coarse, p.fine, tup(p.box)) for p in pl] for pl in h.prolong_lists],
           "restrict": [[(r.fine, r.coarse, tup(r.box)) for r in rl] for rl in h.restrict_lists]}
    out["fine_caps"] = {l: [(int(p), k, a, arr(lo), arr(hi), r) for (p, k, a, lo, hi, r) in v]
                        for l, v in h.fine_caps.items()}
    out["coarse_caps"] = {l: [(int(p), k, a, arr(lo), arr(hi), r) for (p, k, a, lo, hi, r) in v]
                          for l, v in h.coarse_caps.items()}
    out["deposits"] = {l: [(int(c), k, a, arr(lo), arr(hi), rf, arr(flo), arr(fhi), rc)
                           for (c, k, a, lo, hi, rf, flo, fhi, rc) in v] for l, v in h.deposit_list.items()}
    return out


@pytest.mark.parametrize("case", range(4))
def test_tree_metadata_equals_all_pairs_metadata(case):
    from paper_1112_1710_gb300.amr import Hierarchy
    from paper_1112_1710_gb300.tree import DeviceTree
    name, H, n0 = list(hierarchies())[case]
    kw = dict(g=G, dtype="f32", device="cpu")  # metadata only: patch arrays stay on the host
    tree = DeviceTree(H, n0, G + 1, device="cuda")
    a = _meta(Hierarchy(H, n0, _fake_states(H, n0), (1.0 / n0,) * 3, tree=False, **kw))
    b = _meta(Hierarchy(H, n0, _fake_states(H, n0), (1.0 / n0,) * 3, tree=tree, **kw))
    for k in a:
        assert a[k] == b[k], (name, k)


def _fake_states(H, n0):
    """Zero patch arrays of the right shapes (the metadata does not read them)."""
    import synth
    out = []
    for bl in H:
        out.append([synth.empty_patch(tuple(hi[d] - lo[d] + 1 for d in range(3)), G) for lo, hi in bl])
    return out


def test_tree_metadata_equals_oracle(orc):
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300.amr import Hierarchy
    from paper_1112_1710_gb300.tree import DeviceTree
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8, level0_split=2)
    states = [[SA.blast_patch(lo, hi, l, n0, G)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, states, (1.0 / n0,) * 3, g=G)
    ph = Hierarchy(H, n0, states, (1.0 / n0,) * 3, g=G, dtype="f64", device="cpu",
                   tree=DeviceTree(H, n0, G + 1, device="cuda"))
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
