"""CPU checks of the boundary and of the host logic (no GPU calls)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mhd_gpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhd_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_header_function():
    from paper_1112_1710_gb300 import _build, capi
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    names = header_functions()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(names) == set(capi.EXPORTS)


def test_binding_struct_layouts_match_header():
    from paper_1112_1710_gb300 import capi
    # mhd_patch_desc: 4 int32 + box (6 int32) + 8 pointers + 3 int64 + 3 double
    assert ctypes.sizeof(capi.mhd_box) == 24
    assert ctypes.sizeof(capi.mhd_patch_desc) == 16 + 24 + 64 + 24 + 24
    # mhd_params: 2 double + 2 int32 + double + 4 int32 + 2 double (floors)
    assert ctypes.sizeof(capi.mhd_params) == 64
    assert ctypes.sizeof(capi.mhd_deposit) == 16 + 48 + 16
    assert ctypes.sizeof(capi.mhd_transfer_item) == 16 + 24
    assert ctypes.sizeof(capi.mhd_prolong_new_item) == 8 + 24 + 8 + 24
    assert ctypes.sizeof(capi.mhd_copy) == 8 + 24 + 12
    assert ctypes.sizeof(capi.mhd_level_item) == ctypes.sizeof(capi.mhd_prolong_item) == 8 + 24


@pytest.mark.parametrize("n,g", [((8, 6, 5), 2), ((128, 128, 1), 2), ((3, 5, 2), 4), ((1, 1, 1), 2), ((13, 7, 9), 4)])
def test_periodic_copy_list_partitions_ghosts_like_the_wrap(n, g):
    """Every cell of the ghost-extended box grown by one, except the interior,
    is in exactly one copy box, and its source is its periodic image inside
    the interior."""
    from paper_1112_1710_gb300.patch import periodic_copies
    cop = periodic_copies(n, g)
    N = [n[d] + 2 * g + 2 for d in range(3)]
    hits = np.zeros(N[::-1], dtype=int)
    for c in cop:
        lo, hi, off = list(c.box.lo), list(c.box.hi), list(c.offset)
        for k in range(lo[2], hi[2] + 1):
            for j in range(lo[1], hi[1] + 1):
                for i in range(lo[0], hi[0] + 1):
                    hits[k + g + 1, j + g + 1, i + g + 1] += 1
                    src = (i + off[0], j + off[1], k + off[2])
                    for d, s in enumerate(src):
                        assert 0 <= s < n[d]
                        assert (s - (i, j, k)[d]) % n[d] == 0
    inter = np.zeros_like(hits)
    inter[g + 1:g + 1 + n[2], g + 1:g + 1 + n[1], g + 1:g + 1 + n[0]] = 1
    assert np.array_equal(hits, 1 - inter)


def test_extended_ghost_cell_update_accounting():
    """Sec. 4 worked example: an isolated 4x4 grid, R = 2, n_ghost = 4 updates
    12x12 then 4x4 cells (160); split into four 2x2 pieces it updates
    4 x (10x10 + 2x2) = 416, an efficiency of at most 160/416."""
    from paper_1112_1710_gb300.patch import update_box_schedule
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "extended_ghost_accounting.json")))
    ex = gold["isolated_grid"]
    sched = update_box_schedule(ex["n"], ex["R"], ex["n_ghost"])
    assert [c for _, c in sched] == ex["updates_per_substep"]
    assert sum(c for _, c in sched) == ex["total_updates"]
    sp = gold["split_grid"]
    piece = update_box_schedule(sp["piece_n"], ex["R"], ex["n_ghost"])
    assert sum(c for _, c in piece) == sp["updates_per_piece"]
    assert sp["pieces"] * sum(c for _, c in piece) == sp["total_updates"]
    assert round(100 * ex["total_updates"] / sp["total_updates"]) == sp["efficiency_percent"]
    # the build's own schedule: n_ghost = 2 per step and R = 2 give the 4 ghost layers
    assert [k for k, _ in update_box_schedule((16, 16, 16), 2, 2)] == [2, 0]


def apply_copies_numpy(st, n, g, copies):
    """The copy semantics documented for mhd_copy in include/mhd_gpu.h, written
    out on a numpy patch (single patch, src = dst): pass 0 cells and lower
    faces, pass 1 upper faces of each box's top layer; only elements that exist
    in the destination arrays; never the destination's interior faces."""
    N = [v + 2 * g for v in n]
    src = st.copy()

    def interior_face(d, a):
        return all(g <= d[b] <= (g + n[b] if b == a else g + n[b] - 1) for b in range(3))

    def face_exists(d, a):
        return all(0 <= d[b] <= (N[b] if b == a else N[b] - 1) for b in range(3))

    for pass_ in (0, 1):
        for c in copies:
            lo, hi, off = list(c.box.lo), list(c.box.hi), list(c.offset)
            for k in range(lo[2], hi[2] + 1):
                for j in range(lo[1], hi[1] + 1):
                    for i in range(lo[0], hi[0] + 1):
                        gl = (i, j, k)
                        d = (i + g, j + g, k + g)
                        s = (i + off[0] + g, j + off[1] + g, k + off[2] + g)
                        if pass_ == 0:
                            if all(0 <= d[b] < N[b] for b in range(3)):
                                st[:5, d[2], d[1], d[0]] = src[:5, s[2], s[1], s[0]]
                            for a in range(3):
                                if face_exists(d, a) and not interior_face(d, a):
                                    st[5 + a, d[2], d[1], d[0]] = src[5 + a, s[2], s[1], s[0]]
                        else:
                            for a in range(3):
                                if gl[a] != hi[a]:
                                    continue
                                du, su = list(d), list(s)
                                du[a] += 1
                                su[a] += 1
                                if face_exists(du, a) and not interior_face(du, a):
                                    st[5 + a, du[2], du[1], du[0]] = src[5 + a, su[2], su[1], su[0]]


@pytest.mark.parametrize("n,g", [((6, 5, 4), 2), ((7, 3, 1), 2), ((2, 3, 2), 4), ((1, 1, 1), 2)])
def test_copy_list_semantics_equal_oracle_periodic_fill(orc, n, g):
    import synth
    from paper_1112_1710_gb300.patch import periodic_copies
    rng = np.random.default_rng(9)
    st = rng.normal(size=synth.patch_shape(n, g))
    a = st.copy()
    apply_copies_numpy(a, n, g, periodic_copies(n, g))
    b = st.copy()
    orc.fill_periodic(orc.patch(b, n, g, (1.0, 1.0, 1.0)))
    N = [v + 2 * g for v in n]
    assert np.array_equal(a[:5, :N[2], :N[1], :N[0]], b[:5, :N[2], :N[1], :N[0]])
    for q in range(3):
        ext = list(N)
        ext[q] += 1
        assert np.array_equal(a[5 + q, :ext[2], :ext[1], :ext[0]], b[5 + q, :ext[2], :ext[1], :ext[0]])


def apply_copies_one_launch(st, n, g, copies, order):
    """The rule of the one-launch ghost fill, on a numpy patch: every copy
    writes its cells, the lower faces of its cells and the upper faces of its
    top layer, in one pass over the copies in any `order`, except the lower
    faces of its bottom layer along an axis over the transverse extent it
    shares with another copy whose top layer lies directly below (that
    copy's upper faces): the rectangles the library lists per copy."""
    N = [v + 2 * g for v in n]
    src = st.copy()

    def interior_face(d, a):
        return all(g <= d[b] <= (g + n[b] if b == a else g + n[b] - 1) for b in range(3))

    def face_exists(d, a):
        return all(0 <= d[b] <= (N[b] if b == a else N[b] - 1) for b in range(3))

    boxes = [(list(c.box.lo), list(c.box.hi)) for c in copies]
    rects = []
    for t, (lo, hi) in enumerate(boxes):
        r = []
        for u, (ulo, uhi) in enumerate(boxes):
            for a in range(3):
                if u == t or uhi[a] + 1 != lo[a]:
                    continue
                tr = [e for e in range(3) if e != a]
                x = [(max(ulo[e], lo[e]), min(uhi[e], hi[e])) for e in tr]
                if all(x0 <= x1 for x0, x1 in x):
                    r.append((a, tr, x))
        rects.append(r)
    for t in order:
        c = copies[t]
        lo, hi, off = boxes[t][0], boxes[t][1], list(c.offset)
        for k in range(lo[2], hi[2] + 1):
            for j in range(lo[1], hi[1] + 1):
                for i in range(lo[0], hi[0] + 1):
                    gl = (i, j, k)
                    d = (i + g, j + g, k + g)
                    s = (i + off[0] + g, j + off[1] + g, k + off[2] + g)
                    if all(0 <= d[b] < N[b] for b in range(3)):
                        st[:5, d[2], d[1], d[0]] = src[:5, s[2], s[1], s[0]]
                    for a in range(3):
                        skip = gl[a] == lo[a] and any(
                            ra == a and all(x0 <= gl[e] <= x1 for e, (x0, x1) in zip(tr, x))
                            for ra, tr, x in rects[t])
                        if face_exists(d, a) and not interior_face(d, a) and not skip:
                            st[5 + a, d[2], d[1], d[0]] = src[5 + a, s[2], s[1], s[0]]
                        if gl[a] == hi[a]:
                            du, su = list(d), list(s)
                            du[a] += 1
                            su[a] += 1
                            if face_exists(du, a) and not interior_face(du, a):
                                st[5 + a, du[2], du[1], du[0]] = src[5 + a, su[2], su[1], su[0]]


@pytest.mark.parametrize("n,g", [((6, 5, 4), 2), ((7, 3, 1), 2), ((2, 3, 2), 4), ((1, 1, 1), 2)])
def test_one_launch_copy_rule_equals_oracle_periodic_fill(orc, n, g):
    """On random data (faces shared by two copies differ), the one-launch rule
    gives the two-pass result in any order of the copies: no element is
    written twice with different values."""
    import synth
    from paper_1112_1710_gb300.patch import periodic_copies
    rng = np.random.default_rng(10)
    st = rng.normal(size=synth.patch_shape(n, g))
    b = st.copy()
    orc.fill_periodic(orc.patch(b, n, g, (1.0, 1.0, 1.0)))
    N = [v + 2 * g for v in n]
    copies = periodic_copies(n, g)
    for order in (range(len(copies)), range(len(copies) - 1, -1, -1), rng.permutation(len(copies))):
        a = st.copy()
        apply_copies_one_launch(a, n, g, copies, list(order))
        assert np.array_equal(a[:5, :N[2], :N[1], :N[0]], b[:5, :N[2], :N[1], :N[0]])
        for q in range(3):
            ext = list(N)
            ext[q] += 1
            assert np.array_equal(a[5 + q, :ext[2], :ext[1], :ext[0]], b[5 + q, :ext[2], :ext[1], :ext[0]])
