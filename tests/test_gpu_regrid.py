"""Regridding's device work (Sec. 2.1) against the oracle: the error flags
of a level (mhd_flag_cells) bit for bit in FP64 and FP32 (the oracle reading
the FP32 state), on several patches of uneven size in one call; and the
chain flags -> Berger-Rigoutsos clustering -> grids equal to the oracle's."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import to_patch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1112_1710_gb300 import _build, capi as C
    _build.build()
    C.load()
    return C


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("theta", [0.01, 0.05, 0.2])
def test_flags_bitexact(capi, orc, dtype, theta):
    from paper_1112_1710_gb300 import regrid
    probs = [synth.blast(n, noise=0.01, seed=7 + n) for n in (16, 24, 13)]
    ctx = capi.mhd_ctx_create()
    try:
        pats = []
        for pr in probs:
            P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
            orc.fill_periodic(P)
            pats.append(to_patch(pr.state, pr.n, pr.g, pr.dx, dtype=dtype))
        got = regrid.flag(ctx, pats, theta)
        torch.cuda.synchronize()
        for pr, p, f in zip(probs, pats, got):
            st = p.state.cpu().numpy().astype(np.float64)     # the state the GPU read
            want = orc.flag(orc.patch(np.ascontiguousarray(st), pr.n, pr.g, pr.dx), orc.params(), theta)
            assert np.array_equal(f.cpu().numpy(), want)
            if theta == 0.05:
                assert 0 < want.sum() < want.size
    finally:
        capi.mhd_ctx_destroy(ctx)


def test_flag_cluster_chain_equals_oracle(capi, orc):
    from oracle import cluster as OC
    from paper_1112_1710_gb300 import regrid
    pr = synth.blast(32, noise=0.0)
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    for _ in range(6):
        orc.fill_periodic(P)
        orc.advance(P, orc.params(emf=1), orc.cfl_dt(P, orc.params(emf=1)), 0)
    orc.fill_periodic(P)
    ctx = capi.mhd_ctx_create(emf=1)
    try:
        p = to_patch(pr.state, pr.n, pr.g, pr.dx)
        f = regrid.flag(ctx, [p], 0.05)[0].cpu().numpy()
    finally:
        capi.mhd_ctx_destroy(ctx)
    want = orc.flag(P, orc.params(), 0.05)
    assert np.array_equal(f, want) and want.sum() > 0
    # flags are (z, y, x); clustering works in (x, y, z) axis order
    fx = np.ascontiguousarray(f.transpose(2, 1, 0))
    assert regrid.cluster(fx) == OC.cluster(fx)


@pytest.mark.parametrize("kind", ["smooth", "linear"])
@pytest.mark.parametrize("energy_mode", [0, 1])
def test_transfer_equals_oracle(capi, orc, kind, energy_mode):
    """Data transfer into a new iteration (mhd_transfer_copy, then
    mhd_prolong_new under the seam masks) equals the oracle
    (tests/test_oracle_transfer.py pins it) in FP64, on a new patch that
    overlaps two old patches; in FP32 it stays within FP32 rounding of it
    and keeps every fine cell divergence-free to FP32 rounding."""
    import test_oracle_transfer as T
    from paper_1112_1710_gb300 import regrid
    from paper_1112_1710_gb300.patch import Patch
    gst, cst, want, n, dxf, nfall = T.run(orc, kind, energy_mode)
    dxc = tuple(2 * v for v in dxf)
    for dtype in ("f64", "f32"):
        ctx = capi.mhd_ctx_create()
        try:
            old = [Patch.from_array(T.sub_patch(gst, lo, hi), lo, tuple(hi[d] - lo[d] + 1 for d in range(3)), T.G,
                                    dxf, dtype=dtype) for lo, hi in T.OLD]
            coarse = [Patch.from_array(cst, (0, 0, 0), (16, 16, 16), T.G, dxc, dtype=dtype)]
            fresh = [Patch.from_array(synth.empty_patch(n, T.G), T.NEW[0], n, T.G, dxf, dtype=dtype, patch_id=0)]
            nf = regrid.transfer(ctx, old, fresh, coarse, energy_mode)
            torch.cuda.synchronize()
            got = fresh[0].state.cpu().numpy().astype(np.float64)
            assert int(nf.item()) == nfall
        finally:
            capi.mhd_ctx_destroy(ctx)
        G_ = T.G
        for q in range(8):
            ext = list(n)
            if q >= 5:
                ext[q - 5] += 1
            a = got[q, G_:G_ + ext[2], G_:G_ + ext[1], G_:G_ + ext[0]]
            b = want[q, G_:G_ + ext[2], G_:G_ + ext[1], G_:G_ + ext[0]]
            tol = 1e-11 if dtype == "f64" else 2e-6
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), (dtype, q, np.abs(a - b).max() / np.abs(b).max())
        if dtype == "f32":
            P = orc.patch(np.ascontiguousarray(got), n, T.G, dxf)
            assert orc.divb_max(P) * dxf[0] <= 1e-5 * np.abs(got[5:8]).max()


def _interiors_equal(oh, ph, G=4):
    for l in range(len(oh.levels)):
        for P, Q in zip(oh.levels[l], ph.levels[l]):
            got = Q.state.cpu().numpy()
            for q in range(8):
                ext = list(P.n)
                if q >= 5:
                    ext[q - 5] += 1
                a = got[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                b = P.state[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
                if not np.array_equal(a, b):
                    return (l, q, float(np.abs(a - b).max()))
    return None


@pytest.mark.parametrize("theta,first", [(0.03, None), (0.1, None), (0.02, 1)])
def test_regrid_fp64_equals_oracle_and_steps_on(capi, orc, theta, first):
    """One regridding (regrid.regrid_levels: of the finest level, or of
    levels 1 and 2 with level 2 made from the new level 1; each from the
    parent level's flags on the device, grown, nested, clustered, fitted to
    the nested region, cut by the parent grids, and the data transfer) in
    the FP64 parity build: the same grids and the same new patch data as the
    oracle's regridding, and two more coarse steps of the regridded
    hierarchies agree bit for bit."""
    import synth.amr as SA
    from oracle import regrid as OR
    from oracle.amr import OHierarchy
    from paper_1112_1710_gb300 import regrid
    from paper_1112_1710_gb300.amr import Hierarchy
    n0, G = 16, 4
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    st = [[SA.blast_patch(lo, hi, l, n0, G, p_in=10.0)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    oh = OHierarchy(H, n0, [[s.copy() for s in l] for l in st], (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
    ctx = capi.mhd_ctx_create(emf=1)
    ph = ph2 = None
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        oh.initialise()
        ph.initialise()
        assert oh.coarse_step() == (ph.coarse_step() or ph.d_dt.item())
        boxes, states, nfall = regrid.regrid_levels(ph, theta, first=first)
        oboxes, ostates, onfall = OR.regrid_levels(oh, theta, first=first, empty=synth.empty_patch)
        torch.cuda.synchronize()
        assert boxes == oboxes and len(boxes) == 3 and len(boxes[2]) > 0
        assert int(nfall.item()) == onfall
        for l in range(1 if first == 1 else 2, 3):
            for s_gpu, s_orc in zip(states[l], ostates[l]):
                a = s_gpu.cpu().numpy()
                assert np.array_equal(a[:, :s_orc.shape[1], :s_orc.shape[2], :s_orc.shape[3]], s_orc)
        ph.close()
        ph = None
        ph2 = Hierarchy(boxes, n0, states, (1.0 / n0,) * 3, g=G, dtype="f64", ctx=ctx)
        oh2 = OHierarchy(oboxes, n0, ostates, (1.0 / n0,) * 3, g=G, prm=orc.params(emf=1))
        oh2.initialise()
        ph2.initialise()
        for _ in range(2):
            ph2.coarse_step()
            assert oh2.coarse_step() == ph2.d_dt.item()
        torch.cuda.synchronize()
        assert ph2.device_status() == 0
        assert _interiors_equal(oh2, ph2) is None
    finally:
        for h in (ph, ph2):
            if h is not None:
                h.close()
        capi.mhd_ctx_destroy(ctx)


def test_regrid_finest_fp32_runs_on(capi):
    """The same regridding on an FP32 hierarchy: the regridded hierarchy
    steps on with a healthy status and divergence-free new patches."""
    import synth.amr as SA
    from paper_1112_1710_gb300 import regrid
    from paper_1112_1710_gb300.amr import Hierarchy
    n0, G = 16, 4
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    st = [[SA.blast_patch(lo, hi, l, n0, G, p_in=10.0)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    ctx = capi.mhd_ctx_create(emf=1)
    ph = ph2 = None
    try:
        ph = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f32", ctx=ctx)
        ph.initialise()
        ph.coarse_step()
        boxes, states, nfall = regrid.regrid_finest(ph, 0.05)
        assert len(boxes) == 3 and len(boxes[2]) > 0 and int(nfall.item()) == 0
        ph.close()
        ph = None
        ph2 = Hierarchy(boxes, n0, states, (1.0 / n0,) * 3, g=G, dtype="f32", ctx=ctx)
        ph2.initialise()
        for _ in range(2):
            ph2.coarse_step()
        torch.cuda.synchronize()
        assert ph2.device_status() == 0
        dx = 1.0 / (n0 * 4)
        worst = 0.0
        for P in ph2.levels[2]:
            s = P.state.cpu().numpy().astype(np.float64)
            nx, ny, nz = P.n
            bx = s[5, G:G + nz, G:G + ny, G:G + nx + 1]
            by = s[6, G:G + nz, G:G + ny + 1, G:G + nx]
            bz = s[7, G:G + nz + 1, G:G + ny, G:G + nx]
            div = (np.diff(bx, axis=2) + np.diff(by, axis=1) + np.diff(bz, axis=0)) / dx
            worst = max(worst, float(np.abs(div).max()))
        assert worst < 1e-3, worst
    finally:
        for h in (ph, ph2):
            if h is not None:
                h.close()
        capi.mhd_ctx_destroy(ctx)


def test_hierarchy_regrid_method(capi):
    """Hierarchy.regrid: the new hierarchy keeps the context, has the
    regridded finest level and steps on."""
    import synth.amr as SA
    from paper_1112_1710_gb300.amr import Hierarchy
    n0, G = 16, 4
    H = SA.shell_hierarchy(n0=n0, levels=3, size_min=4, size_max=8)
    st = [[SA.blast_patch(lo, hi, l, n0, G, p_in=10.0)[0] for (lo, hi) in bl] for l, bl in enumerate(H)]
    h = Hierarchy(H, n0, st, (1.0 / n0,) * 3, g=G, dtype="f32", concurrent=True)
    ctx = h.ctx
    try:
        h.initialise()
        h.coarse_step()
        h2 = h.regrid(0.05)
        h = h2
        assert h.ctx == ctx and h.own_ctx and len(h.side) == 2
        assert h.regrid_info["new_patches"] == len(h.levels[2]) > 0
        h.coarse_step()
        torch.cuda.synchronize()
        assert h.device_status() == 0
    finally:
        h.close()
