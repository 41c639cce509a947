"""Synchronisation of fluxes on faces shared by two patches of one level
(mhd_reflux deposits in mode MHD_SYNC, Sec. 2.2) with library-owned FP64
registers (mhd_fluxreg_create), against the oracle (tests/test_oracle_sync.py
pins the oracle): FP64 bit for bit, on the perturbed two-patch step whose
shared-face fluxes differ and on the unperturbed one where the
synchronisation changes nothing."""
import numpy as np
import pytest
import torch

import test_oracle_sync as S
from gpu_util import to_patch

pytestmark = pytest.mark.gpu
G = S.G


@pytest.fixture(scope="module")
def capi():
    from paper_1112_1710_gb300 import _build, capi as C
    _build.build()
    C.load()
    return C


def gpu_step(capi, orc, perturb, sync):
    pr, dt, (A, na, gla), (B, nb, glb) = S.setup(orc, perturb)
    ctx = capi.mhd_ctx_create(emf=1)
    reg = None
    try:
        pa = to_patch(A, na, G, pr.dx, lo=gla, pid=0)
        pb = to_patch(B, nb, G, pr.dx, lo=glb, pid=1)
        descs = [pa.desc(), pb.desc()]
        reg = capi.mhd_fluxreg_create(ctx, descs)
        d_dt = torch.full((1,), dt, dtype=torch.float64, device="cuda")
        # A's shared face is its upper x side, B's its lower x side
        mine = {}
        for pi, side in ((0, 1), (1, 0)):
            fptr, fbox = capi.mhd_fluxreg_face(reg, pi, 0, side)
            yptr, ybox = capi.mhd_fluxreg_edge(reg, pi, 0, side, 1)
            zptr, zbox = capi.mhd_fluxreg_edge(reg, pi, 0, side, 2)
            caps = []
            for kind, axis, (lo, hi), ptr in ((capi.MHD_CAP_FACE, 0, fbox, fptr), (capi.MHD_CAP_EDGE, 1, ybox, yptr),
                                              (capi.MHD_CAP_EDGE, 2, zbox, zptr)):
                c = capi.mhd_capture()
                c.patch, c.kind, c.axis, c.mode = 0, kind, axis, 0
                c.box = capi.box(lo, hi)
                c.dst = ptr
                caps.append(c)
            capi.mhd_patch_advance(ctx, [descs[pi]], d_dt.data_ptr(), caps=caps)
            mine[pi] = ((fptr, fbox), (yptr, ybox), (zptr, zbox))
        if sync:
            corr = [torch.zeros((18,) + tuple(p.state.shape[1:]), dtype=torch.float64, device="cuda") for p in (pa, pb)]
            deps = []
            for me, other in ((0, 1), (1, 0)):
                for (kind, axis), (ptr, (lo, hi)), (optr, _) in zip(
                        ((capi.MHD_CAP_FACE, 0), (capi.MHD_CAP_EDGE, 1), (capi.MHD_CAP_EDGE, 2)), mine[me], mine[other]):
                    dp = capi.mhd_deposit()
                    dp.coarse, dp.kind, dp.axis, dp.mode = me, kind, axis, capi.MHD_SYNC
                    dp.box = capi.box(lo, hi)
                    dp.fine_box = capi.box(lo, hi)
                    dp.fine = optr
                    dp.coarse_reg = ptr
                    deps.append(dp)
            capi.mhd_reflux(ctx, descs, [c.data_ptr() for c in corr], deps)
        torch.cuda.synchronize()
        assert capi.mhd_get_device_status(ctx) == 0
        out = (pa.state.cpu().numpy(), pb.state.cpu().numpy())
    finally:
        if reg:
            capi.mhd_fluxreg_destroy(reg)
        capi.mhd_ctx_destroy(ctx)
    return out


@pytest.mark.parametrize("perturb", [True, False])
def test_sync_equals_oracle(capi, orc, perturb):
    ga, gb = gpu_step(capi, orc, perturb, True)
    parts, _, _ = S.run(orc, perturb, True)
    (A, na, _), (B, nb, _) = parts
    for got, want, n in ((ga, A, na), (gb, B, nb)):
        for q in range(8):
            ext = list(n)
            if q >= 5:
                ext[q - 5] += 1
            a = got[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
            b = want[q, G:G + ext[2], G:G + ext[1], G:G + ext[0]]
            assert np.abs(a - b).max() <= 1e-11 * max(np.abs(b).max(), 1e-300), q
    if perturb:
        # and the synchronisation did something: the unsynchronised step differs
        ua, _ = gpu_step(capi, orc, True, False)
        assert np.abs(ua - ga).max() > 1e-8


def test_fluxreg_layout(capi):
    """Register boxes of library-owned registers follow the header's layout."""
    from paper_1112_1710_gb300.patch import Patch
    st = np.zeros((8, 10, 12, 16))
    p = Patch.from_array(np.ascontiguousarray(st), (4, 6, 8), (5, 7, 5), 2, (1.0, 1.0, 1.0), dtype="f64")
    ctx = capi.mhd_ctx_create()
    reg = capi.mhd_fluxreg_create(ctx, [p.desc()])
    try:
        _, (lo, hi) = capi.mhd_fluxreg_face(reg, 0, 1, 1)
        assert lo == (4, 13, 8) and hi == (8, 13, 12)
        _, (lo, hi) = capi.mhd_fluxreg_edge(reg, 0, 2, 0, 0)     # x-edges in the lower z face
        assert lo == (4, 6, 8) and hi == (8, 13, 8)
        _, (lo, hi) = capi.mhd_fluxreg_edge(reg, 0, 2, 0, 1)     # y-edges in the lower z face
        assert lo == (4, 6, 8) and hi == (9, 12, 8)
        with pytest.raises(Exception):
            capi.mhd_fluxreg_edge(reg, 0, 2, 0, 2)
        with pytest.raises(Exception):
            capi.mhd_fluxreg_face(reg, 1, 0, 0)
        capi.mhd_fluxreg_zero(reg)
        torch.cuda.synchronize()
    finally:
        capi.mhd_fluxreg_destroy(reg)
        capi.mhd_ctx_destroy(ctx)
