"""AMR level operations and the subcycled coarse step: GPU (sm_103a) vs the
FP64 oracle through the C ABI.  FP64 results are expected bit-identical (bar
1e-11); the FP32 run reports its conservation drift and div B."""
import numpy as np
import pytest
import torch

import synth
import synth.amr as SA
from gpu_util import random_state, to_patch

pytestmark = pytest.mark.gpu
G = 4
TOL = 1e-11


@pytest.fixture(scope="module")
def capi():
    from paper_1112_1710_gb300 import _build, capi as C
    _build.build()
    C.load()
    return C


def _states(H, n0, p_in=10.0):
    return [[SA.blast_patch(lo, hi, l, n0, G, p_in=p_in)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]


def test_prolong_and_restrict_random_data(capi, orc):
    """Prolongation of random coarse data into a fine patch's ghost zone and the
    restriction of random fine data, against the oracle."""
    ctx = capi.mhd_ctx_create()
    try:
        nc, lo_c = (12, 12, 12), (0, 0, 0)
        stc = random_state(nc, G, seed=31)
        nf, lo_f = (8, 6, 10), (6, 8, 4)
        stf = random_state(nf, G, seed=32)
        pc = to_patch(stc, nc, G, (0.1,) * 3, lo=lo_c)
        pf = to_patch(stf, nf, G, (0.05,) * 3, lo=lo_f, level=1)
        clo = tuple((v - G) // 2 for v in lo_f)
        chi = tuple((v + nf[d] + G) // 2 - 1 for d, v in enumerate(lo_f))
        it = capi.mhd_prolong_item()
        it.coarse, it.fine = 0, 0
        it.box = capi.box(clo, chi)
        capi.mhd_prolong(ctx, [pc.desc()], [pf.desc()], [it])
        Pc = orc.patch(stc, nc, G, (0.1,) * 3)
        a = stf.copy()
        Pf = orc.patch(a, nf, G, (0.05,) * 3)
        orc.prolong(Pc, lo_c, Pf, lo_f, clo, chi)
        assert np.array_equal(pf.state.cpu().numpy(), a)
        # restriction onto the coarse patch (box grown by one around the interior)
        b = stc.copy()
        Pc2 = orc.patch(b, nc, G, (0.1,) * 3)
        rlo = tuple(v // 2 for v in lo_f)
        rhi = tuple((v + nf[d]) // 2 - 1 for d, v in enumerate(lo_f))
        for pass_ in (0, 1):
            orc.restrict(Pf, lo_f, Pc2, lo_c, rlo, rhi, pass_)
        ri = capi.mhd_restrict_item()
        ri.fine, ri.coarse = 0, 0
        ri.box = capi.box(rlo, rhi)
        capi.mhd_restrict(ctx, [pf.desc()], [pc.desc()], [ri])
        assert np.array_equal(pc.state.cpu().numpy(), b)
        # the combined entry point gives the same bits in both modes
        pc2 = to_patch(stc, nc, G, (0.1,) * 3, lo=lo_c)
        pf2 = to_patch(stf, nf, G, (0.05,) * 3, lo=lo_f, level=1)
        li = capi.mhd_level_item()
        li.fine, li.coarse = 0, 0
        li.box = capi.box(clo, chi)
        capi.mhd_restrict_prolong(ctx, capi.MHD_PROLONG, [pf2.desc()], [pc2.desc()], [li])
        assert torch.equal(pf2.state, pf.state)
        li.box = capi.box(rlo, rhi)
        capi.mhd_restrict_prolong(ctx, capi.MHD_RESTRICT, [pf2.desc()], [pc2.desc()], [li])
        assert torch.equal(pc2.state, pc.state)
        with pytest.raises(capi.MHDError) as ei:
            capi.mhd_restrict_prolong(ctx, 2, [pf2.desc()], [pc2.desc()], [li])
        assert ei.value.status == capi.MHD_EINVAL
    finally:
        capi.mhd_ctx_destroy(ctx)


@pytest.mark.parametrize("split,kernel", [(1, 1), (2, 1), (1, 2), (1, 4)])
def test_amr_coarse_steps_fp64_parity(capi, orc, split, kernel):
    """Three subcycled coarse steps of a 3-level shell hierarchy (1 + 47 + 42
    patches of 4^3-8^3 cells, 4 ghost layers): every patch array equals the
    oracle's, with the staged advance (1), the fused one (2), whose
    flux-register captures come from the fluxes it stores, and the fused pass
    (4)."""
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8, level0_split=split)
    st = _states(H, n0)
    oh = OHierarchy(H, n0, [[s.copy() for s in l] for l in st], (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
    ctx = capi.mhd_ctx_create(emf=1, advance_kernel=kernel)
    ph = None
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        oh.initialise()
        oh.fill(0)
        ph.initialise()
        for _ in range(3):
            odt = oh.coarse_step()
            ph.coarse_step()
            assert ph.d_dt.item() == odt
        assert ph.device_status() == 0
        worst = 0.0
        for l in range(3):
            for P, Q in zip(oh.levels[l], ph.levels[l]):
                got = Q.state.cpu().numpy()
                n = P.n
                for q in range(8):
                    ext = list(n)
                    if q >= 5:
                        ext[q - 5] += 1
                    a = got[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                    b = P.state[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                    worst = max(worst, float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)))
        assert worst <= TOL, worst
    finally:
        if ph is not None:
            ph.close()
        capi.mhd_ctx_destroy(ctx)


def test_amr_fp32_conservation_and_divb(capi, capsys):
    """FP32 state with FP64 flux registers and sums: composite totals and the
    face divergence after five coarse steps (reported)."""
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    ctx = capi.mhd_ctx_create(emf=1)
    try:
        ph = Hierarchy(H, n0, _states(H, n0), (1.0 / n0,) * 3, g=G, dtype="f32", ctx=ctx)
        ph.initialise()
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s0 = out.cpu().numpy().copy()
        for _ in range(5):
            ph.coarse_step()
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s1 = out.cpu().numpy()
        divb = 0.0
        for l, pats in enumerate(ph.levels):
            for p in pats:
                s = p.state.double().cpu().numpy()
                nx, ny, nz = p.n
                d = ((s[5, G:G + nz, G:G + ny, G + 1:G + nx + 1] - s[5, G:G + nz, G:G + ny, G:G + nx])
                     + (s[6, G:G + nz, G + 1:G + ny + 1, G:G + nx] - s[6, G:G + nz, G:G + ny, G:G + nx])
                     + (s[7, G + 1:G + nz + 1, G:G + ny, G:G + nx] - s[7, G:G + nz, G:G + ny, G:G + nx]))
                divb = max(divb, float(np.abs(d).max()))
        rel = np.abs(s1 - s0) / np.maximum(np.abs(s0), 1e-12)
        with capsys.disabled():
            print("\nFP32 AMR, 5 coarse steps: relative drift of (rho, E, Bx, By):",
                  " ".join("%.2e" % v for v in rel[[0, 4, 5, 6]]), " max |div B| dx:", "%.2e" % divb)
        assert rel[0] < 1e-5 and rel[4] < 1e-5 and divb < 1e-4
        assert ph.device_status() == 0
    finally:
        ph.close()
        capi.mhd_ctx_destroy(ctx)


@pytest.mark.parametrize("kernel", [0, 4])
def test_amr_graph_replay_and_per_patch_path_equal_eager_batched(capi, kernel):
    """A captured coarse-step graph, and the plain one-call-per-patch advance,
    give the same bits as the eager batched path (the batched paths here
    advance the coarser levels on side streams, concurrently with the finer
    substeps, Sec. 4; the per-patch path runs every level on one stream)."""
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    st = _states(H, n0)
    ctx = capi.mhd_ctx_create(emf=1, advance_kernel=kernel)
    ctx2 = capi.mhd_ctx_create(emf=1, advance_kernel=kernel)  # one context (scratch arena) per stream
    a = b = c = None
    try:
        a = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx, concurrent=True)
        b = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx2, stream=torch.cuda.Stream(),
                      concurrent=True)
        c = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        c.batched = False
        for h in (a, b, c):
            h.initialise()
        b.capture_graph()          # runs one eager step, then captures
        a.coarse_step()
        c.coarse_step()
        for _ in range(2):
            a.coarse_step()
            b.replay()
            c.coarse_step()
        torch.cuda.synchronize()
        for l in range(3):
            for pa, pb, pc in zip(a.levels[l], b.levels[l], c.levels[l]):
                sa = pa.state.cpu().numpy()
                assert np.array_equal(sa, pb.state.cpu().numpy())
                assert np.array_equal(sa, pc.state.cpu().numpy())
    finally:
        for h in (a, b, c):
            if h is not None:
                h.close()
        capi.mhd_ctx_destroy(ctx)
        capi.mhd_ctx_destroy(ctx2)


@pytest.mark.parametrize("kernel", [0, 4])
def test_turbulent_deep_hierarchy_fp64_parity(capi, orc, kernel):
    """The deep-AMR workload's generator downscaled (base 16^3, 3 levels,
    k^-4 velocity field at Mach 5, plasma beta 1): three subcycled coarse
    steps of the FP64 parity build equal the oracle's on every patch."""
    import synth.turb as ST
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H, v, _ = ST.deep_hierarchy(n0=n0, levels=3, m=32, size_min=4, size_max=8)
    assert len(H) == 3 and all(len(l) > 0 for l in H)
    st = [[ST.turb_patch(lo, hi, l, n0, G, v)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, [[s.copy() for s in l] for l in st], (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
    ctx = capi.mhd_ctx_create(emf=1, advance_kernel=kernel)
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        oh.initialise()
        oh.fill(0)
        ph.initialise()
        for _ in range(3):
            odt = oh.coarse_step()
            ph.coarse_step()
            assert ph.d_dt.item() == odt
        assert ph.device_status() == 0
        for l in range(3):
            for P, Q in zip(oh.levels[l], ph.levels[l]):
                got = Q.state.cpu().numpy()
                n = P.n
                for q in range(8):
                    ext = list(n)
                    if q >= 5:
                        ext[q - 5] += 1
                    a = got[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                    b = P.state[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                    assert np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-300), (l, q)
        ph.close()
    finally:
        capi.mhd_ctx_destroy(ctx)


def test_blast_shell_full_size_fp64_properties(capi, capsys):
    """The AMR workload at its full size (base 64^3 + 3 levels, 2,720 patches
    of 8^3-48^3, 4 ghost layers; the oracle is too slow here): one subcycled
    FP64 coarse step conserves the composite totals of rho, M, E to rounding
    and keeps every patch's face divergence at rounding."""
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 64
    H = SA.shell_hierarchy(n0=n0, levels=4, seed=1112, size_min=8, size_max=48)
    assert [len(l) for l in H] == [1, 153, 594, 1972]
    st = [[SA.blast_patch(lo, hi, l, n0, G)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    ctx = capi.mhd_ctx_create(emf=1)
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        del st
        ph.initialise()
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s0 = out.cpu().numpy().copy()
        ph.coarse_step()
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s1 = out.cpu().numpy()
        assert ph.device_status() == 0
        rel = np.abs(s1 - s0) / np.maximum(np.abs(s0), 1e-300)
        divb = 0.0
        for l, pats in enumerate(ph.levels):
            for p in pats:
                s = p.state
                nx, ny, nz = p.n
                d = ((s[5, G:G + nz, G:G + ny, G + 1:G + nx + 1] - s[5, G:G + nz, G:G + ny, G:G + nx])
                     + (s[6, G:G + nz, G + 1:G + ny + 1, G:G + nx] - s[6, G:G + nz, G:G + ny, G:G + nx])
                     + (s[7, G + 1:G + nz + 1, G:G + ny, G:G + nx] - s[7, G:G + nz, G:G + ny, G:G + nx]))
                divb = max(divb, float(d.abs().max()))
        with capsys.disabled():
            print("\nFP64 AMR full size, one coarse step: relative drift (rho, E) %.1e %.1e, max |div B| dx %.1e"
                  % (rel[0], rel[4], divb))
        assert rel[0] < 1e-12 and rel[4] < 1e-12 and divb < 1e-12
        ph.close()
    finally:
        capi.mhd_ctx_destroy(ctx)


def test_deep_hierarchy_full_size_fp32_properties(capi, capsys):
    """The deep-AMR workload at its full size (base 32^3 + 7 levels, 1,800
    patches, 108 M cells on the k^-4 Mach-5 field, beta 1; the oracle runs it
    only downscaled): one subcycled FP32 coarse step with FP64 flux registers
    and sums keeps the composite totals of rho and E to the FP32 budget,
    every face divergence at FP32 rounding, and the device status clean (no
    non-positive density or pressure)."""
    import synth.turb as ST
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 32
    H, v, _ = ST.deep_hierarchy(n0=n0, levels=8, m=256)
    assert len(H) == 8 and sum(len(l) for l in H) == 1800
    ctx = capi.mhd_ctx_create(emf=1)
    ph = None
    try:
        st = [[ST.turb_patch(lo, hi, l, n0, G, v)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f32", ctx=ctx)
        del st
        ph.initialise()
        out = torch.zeros(8, dtype=torch.float64, device="cuda")
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s0 = out.cpu().numpy().copy()
        ph.coarse_step()
        capi.mhd_conservation_sums(ctx, ph.descs[0], out.data_ptr())
        s1 = out.cpu().numpy()
        assert ph.device_status() == 0
        rel = np.abs(s1 - s0) / np.maximum(np.abs(s0), 1e-300)
        divb = 0.0
        for l, pats in enumerate(ph.levels):
            for p in pats:
                s = p.state
                nx, ny, nz = p.n
                d = ((s[5, G:G + nz, G:G + ny, G + 1:G + nx + 1] - s[5, G:G + nz, G:G + ny, G:G + nx])
                     + (s[6, G:G + nz, G + 1:G + ny + 1, G:G + nx] - s[6, G:G + nz, G:G + ny, G:G + nx])
                     + (s[7, G + 1:G + nz + 1, G:G + ny, G:G + nx] - s[7, G:G + nz, G:G + ny, G:G + nx]))
                bmax = max(float(s[5].abs().max()), float(s[6].abs().max()), float(s[7].abs().max()))
                divb = max(divb, float(d.abs().max()) / bmax)
        with capsys.disabled():
            print("\nFP32 deep AMR full size, one coarse step: relative drift (rho, E) %.1e %.1e, "
                  "max |div B| dx / max|B| %.1e" % (rel[0], rel[4], divb))
        assert rel[0] < 1e-6 and rel[4] < 1e-6 and divb < 1e-4
    finally:
        if ph is not None:
            ph.close()
        capi.mhd_ctx_destroy(ctx)


@pytest.mark.parametrize("levels,split", [(2, 2), (3, 1)])
def test_ghost_fill_random_faces_equals_oracle(capi, orc, levels, split):
    """Same-level ghost copies of every level of a shell hierarchy on random
    data, whose faces shared by two patches differ: where the top layer of
    one copy box lies on the bottom layer of another, the two sources give
    different values, so the one-launch fill must reproduce the two-pass
    rule element for element (every array of every patch, ghosts included)."""
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300.amr import Hierarchy
    n0 = 16
    H = SA.shell_hierarchy(n0=n0, levels=levels, size_min=4, size_max=8, level0_split=split)
    st = []
    for l, bl in enumerate(H):
        lv = []
        for i, (lo, hi) in enumerate(bl):
            n = tuple(hi[d] - lo[d] + 1 for d in range(3))
            lv.append(random_state(n, G, seed=1000 * l + i))
        st.append(lv)
    oh = OHierarchy(H, n0, [[s.copy() for s in l] for l in st], (1.0 / n0,) * 3, g=G, prm=orc.params())
    ctx = capi.mhd_ctx_create()
    ph = None
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        shared = 0
        for l in range(levels):
            oh.fill(l)
            ph.fill(l)
            shared += len(ph.copy_lists[l])
        assert shared > 0
        torch.cuda.synchronize()
        for l in range(levels):
            for P, Q in zip(oh.levels[l], ph.levels[l]):
                assert np.array_equal(Q.state.cpu().numpy(), P.state), (l, P.idx)
    finally:
        if ph is not None:
            ph.close()
        capi.mhd_ctx_destroy(ctx)
