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
