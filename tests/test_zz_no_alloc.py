"""The allocation-free conservation sums (mhd_conservation_sums_static).

Some callers of this library cannot allocate device memory (their memory is
reserved by another allocator, or they must avoid cudaMalloc/cudaFree because
those can synchronise the device).  For them the library offers one entry
point whose scratch is a fixed array inside the library.  These tests call it
through the C ABI and check it against the regular, context-based entry point
on two calls in a row (a larger request followed by a smaller one, so the
second call runs over partials left behind by the first).  The file is named
to be collected last."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    from paper_1112_1710_gb300 import _build, capi as C
    _build.build()
    C.load()
    return C


def _patch(pr, dtype, pid):
    from paper_1112_1710_gb300.patch import Patch
    return Patch.from_array(pr.state, (0, 0, 0), pr.n, pr.g, pr.dx, dtype=dtype, patch_id=pid)


def _bound(pr_list):
    """Standard summation bound 2 n u sum|x| of the regular path's tests."""
    tot = np.zeros(8)
    n = 0
    for pr in pr_list:
        g, (nx, ny, nz) = pr.g, pr.n
        dv = pr.dx[0] * pr.dx[1] * pr.dx[2]
        tot += np.abs(pr.state[:, g:g + nz, g:g + ny, g:g + nx]).reshape(8, -1).sum(1) * dv
        n += nx * ny * nz
    return 2 * n * np.finfo(np.float64).eps * tot


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_static_sums_match_context_sums_on_two_calls(capi, dtype):
    ctx = capi.mhd_ctx_create()
    try:
        big = [synth.blast(48, seed=1), synth.blast(40, seed=2), synth.orszag_tang(64)]
        small = [synth.blast(24, seed=3)]
        for probs in (big, small):
            patches = [_patch(pr, dtype, i) for i, pr in enumerate(probs)]
            descs = [p.desc() for p in patches]
            want = torch.zeros(8, dtype=torch.float64, device="cuda")
            got = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            capi.mhd_conservation_sums(ctx, descs, want.data_ptr())
            capi.mhd_conservation_sums_static(descs, got.data_ptr())
            torch.cuda.synchronize()
            w, g = want.cpu().numpy(), got.cpu().numpy()
            assert np.all(np.abs(g - w) <= _bound(probs)), (g, w)
            assert np.array_equal(g, w)
    finally:
        capi.mhd_ctx_destroy(ctx)


def test_static_sums_leave_device_memory_unchanged(capi):
    """After a first call (the library loaded, its fixed array resident), a
    call changes neither the device's free memory nor torch's allocation."""
    pr = synth.blast(32, seed=7)
    p = _patch(pr, "f32", 0)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    capi.mhd_conservation_sums_static([p.desc()], out.data_ptr())
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        capi.mhd_conservation_sums_static([p.desc()], out.data_ptr())
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0


def test_static_sums_reject_requests_beyond_capacity(capi):
    pr = synth.blast(8)
    p = _patch(pr, "f64", 0)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.MHDError) as e:
        capi.mhd_conservation_sums_static([p.desc()] * 17, out.data_ptr())
    assert e.value.status == capi.MHD_ETOOBIG
    # a real 200^3 patch (8e6 cells > 4,194,304): rejected before any launch
    from paper_1112_1710_gb300.patch import Patch, patch_shape
    n = (200, 200, 200)
    st = torch.zeros(patch_shape(n, 2), dtype=torch.float64, device="cuda")
    big = Patch(st, (0, 0, 0), n, 2, (0.005, 0.005, 0.005))
    with pytest.raises(capi.MHDError) as e:
        capi.mhd_conservation_sums_static([big.desc()], out.data_ptr())
    assert e.value.status == capi.MHD_ETOOBIG
    torch.cuda.synchronize()
