"""GPU (sm_103a) vs FP64 oracle parity through the C ABI.

FP64: the GPU build has no multiply-add contraction and evaluates every
expression in the oracle's order, so results are expected to be identical;
the bar is L-infinity relative error <= 1e-11 per variable after 10 steps.
Integer metadata and copies are bit-exact."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import random_state, rel_l1, rel_linf, to_patch

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module")
def capi():
    from paper_1112_1710_gb300 import _build, capi as C
    _build.build()
    C.load()
    return C


@pytest.fixture
def ctx(capi):
    c = capi.mhd_ctx_create()
    yield c
    capi.mhd_ctx_destroy(c)


@pytest.mark.parametrize("n,g", [((8, 6, 5), 2), ((128, 128, 1), 2), ((3, 5, 2), 4), ((1, 1, 1), 2),
                                 ((37, 29, 23), 4)])
def test_periodic_ghost_fill_bitexact(capi, ctx, orc, n, g):
    from paper_1112_1710_gb300.patch import periodic_copies
    st = random_state(n, g, seed=11)
    p = to_patch(st, n, g, (1.0, 1.0, 1.0))
    capi.mhd_ghost_fill(ctx, [p.desc()], periodic_copies(n, g))
    P = orc.patch(st, n, g, (1.0, 1.0, 1.0))
    orc.fill_periodic(P)
    got = p.state.cpu().numpy()
    # every cell array element and every face element the fill defines
    assert np.array_equal(got[:5, :n[2] + 2 * g, :n[1] + 2 * g, :n[0] + 2 * g],
                          st[:5, :n[2] + 2 * g, :n[1] + 2 * g, :n[0] + 2 * g])
    N = [v + 2 * g for v in n]
    for a in range(3):
        ext = list(N)
        ext[a] += 1
        assert np.array_equal(got[5 + a, :ext[2], :ext[1], :ext[0]], st[5 + a, :ext[2], :ext[1], :ext[0]])


@pytest.mark.parametrize("problem", ["blast", "ot", "random"])
def test_cfl_dt_bitexact(capi, ctx, orc, problem):
    if problem == "blast":
        pr = synth.blast(24)
        st, n, g, dx = pr.state, pr.n, pr.g, pr.dx
    elif problem == "ot":
        pr = synth.orszag_tang(40)
        st, n, g, dx = pr.state, pr.n, pr.g, pr.dx
    else:
        n, g, dx = (21, 17, 13), 2, (0.1, 0.07, 0.13)
        st = random_state(n, g, seed=3)
    P = orc.patch(st, n, g, dx)
    orc.fill_periodic(P)
    want = orc.cfl_dt(P, orc.params())
    p = to_patch(st, n, g, dx)
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    capi.mhd_cfl_dt(ctx, [p.desc()], d.data_ptr())
    assert d.item() == want
    # the scale factor of a hierarchy level is an exact power of two
    capi.mhd_cfl_dt(ctx, [p.desc()], d.data_ptr(), scale=[4.0])
    assert d.item() == 4.0 * want


@pytest.mark.parametrize("emf,lim", [(0, 0), (1, 0), (0, 1), (0, 2)])
@pytest.mark.parametrize("k", [0, 2])
@pytest.mark.parametrize("kernel,chunk", [(1, 0), (2, 0), (2, 4), (4, 0), (4, 3)])
def test_one_step_random_state_ragged(capi, orc, emf, lim, k, kernel, chunk):
    """One step on a ragged patch (several blocks, partial tail) from random
    data, including the extended update box (k = 2, g = 4), with the staged
    kernels (1), the fused kernel (2: 8 x 8 tiles in FP64, ragged in x and
    y; z in one chunk or in chunks of 4 planes with a ragged last one) and the
    fused pass (4: 8 x 8 tiles, z in chunks of 16 or 3 planes).  The
    tiled predictor of the staged path is checked by the autotuner test and
    test_tiled_predictor_fp64_bitexact."""
    n, g, dx = (19, 13, 11), 4, (0.05, 0.07, 0.06)
    st = random_state(n, g, seed=5 + k)
    ctx = capi.mhd_ctx_create(limiter=lim, emf=emf, advance_kernel=kernel, fused_chunk=chunk)
    try:
        p = to_patch(st, n, g, dx)
        d = torch.full((1,), 1.3e-3, dtype=torch.float64, device="cuda")
        capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr(), grow=[k])
        assert capi.mhd_get_device_status(ctx) == 0
        got = p.state.cpu().numpy()
    finally:
        capi.mhd_ctx_destroy(ctx)
    P = orc.patch(st, n, g, dx)
    assert orc.advance(P, orc.params(limiter=lim, emf=emf), 1.3e-3, k) == 0
    # compare the update box and its faces
    lo, hi = g - k, g + np.array(n) - 1 + k
    for q in range(8):
        ext_hi = hi.copy()
        if q >= 5:
            ext_hi[q - 5] += 1
        a = got[q, lo:ext_hi[2] + 1, lo:ext_hi[1] + 1, lo:ext_hi[0] + 1]
        b = st[q, lo:ext_hi[2] + 1, lo:ext_hi[1] + 1, lo:ext_hi[0] + 1]
        assert np.abs(a - b).max() <= TOL * np.abs(b).max(), (q, np.abs(a - b).max())
    # outside the update box nothing changed
    untouched = got.copy()
    untouched[:, lo:hi[2] + 2, lo:hi[1] + 2, lo:hi[0] + 2] = 0
    ref = st.copy()
    ref[:, lo:hi[2] + 2, lo:hi[1] + 2, lo:hi[0] + 2] = 0
    assert np.array_equal(untouched, ref)


def _run_both(capi, ctx, orc, pr, steps, dtype="f64", dt=None, emf=0):
    from paper_1112_1710_gb300.runner import PeriodicRunner
    st0 = pr.state.copy()
    p = to_patch(st0, pr.n, pr.g, pr.dx, dtype=dtype)
    run = PeriodicRunner(p, ctx)
    gdts = run.run(steps, dt=dt, record_dt=True)
    got = p.state.cpu().numpy()
    odts = orc.run_periodic(pr.state, pr.n, pr.g, pr.dx, orc.params(emf=emf), steps, dt=dt)
    return got, pr.state, gdts, odts


@pytest.fixture
def ctx_blast(capi):
    """The blast workloads use the arithmetic edge-EMF average."""
    c = capi.mhd_ctx_create(emf=1)
    yield c
    capi.mhd_ctx_destroy(c)


def test_orszag_tang_128_fp64_10_steps(capi, ctx, orc):
    """2D Orszag-Tang, 128^2 + 2 ghosts, FP64, CFL 0.4 (the full-size 2D case)."""
    pr = synth.orszag_tang(128)
    got, want, gdts, odts = _run_both(capi, ctx, orc, pr, 10)
    assert gdts == odts
    err = rel_linf(got, want, pr.n, pr.g)
    assert np.all(err <= TOL), err
    assert capi.mhd_get_device_status(ctx) == 0


@pytest.mark.parametrize("kernel", [2, 4])
def test_orszag_tang_fused_paths_equal_staged(capi, kernel):
    """The 2D Orszag-Tang patch (one cell along z, periodic z) through the
    fused kernel (2) and the fused pass (4) in the FP64 parity build: the
    staged kernels' bits after 5 steps with the CFL dt of each step."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    pr = synth.orszag_tang(64)
    out = []
    for k in (1, kernel):
        ctx = capi.mhd_ctx_create(advance_kernel=k)
        try:
            p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx)
            r = PeriodicRunner(p, ctx)
            for _ in range(5):
                r.step()
            assert capi.mhd_get_device_status(ctx) == 0
            out.append(p.state.cpu().numpy())
        finally:
            capi.mhd_ctx_destroy(ctx)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 1), (3, 1, 2), (17, 1, 5)])
def test_tiny_patches_every_advance_equals_staged(capi, n):
    """Patches down to one cell (update boxes thinner than a tile, a block's
    lower column and row outside the region): the fused kernel (2) and the
    fused pass (4) give the staged bits in the FP64 parity build, k = 0 and
    2."""
    g = 4
    for k in (0, 2):
        st = random_state(n, g, seed=90 + k + sum(n))
        out = []
        for kernel in (1, 2, 4):
            ctx = capi.mhd_ctx_create(advance_kernel=kernel)
            try:
                p = to_patch(st, n, g, (0.05, 0.06, 0.07))
                d = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
                capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr(), grow=[k])
                assert capi.mhd_get_device_status(ctx) == 0
                out.append(p.state.cpu().numpy())
            finally:
                capi.mhd_ctx_destroy(ctx)
        assert np.array_equal(out[0], out[1]), (k, "fused kernel")
        assert np.array_equal(out[0], out[2]), (k, "fused pass")


def test_blast_128_fp64_10_steps(capi, ctx_blast, orc):
    """3D blast, 128^3 + 2 ghosts, FP64 (the full-size 3D case, same launch
    configuration as the bench)."""
    pr = synth.blast(128)
    got, want, gdts, odts = _run_both(capi, ctx_blast, orc, pr, 10, emf=1)
    assert gdts == odts
    err = rel_linf(got, want, pr.n, pr.g)
    assert np.all(err <= TOL), err
    assert capi.mhd_get_device_status(ctx_blast) == 0


@pytest.mark.parametrize("case", ["orszag_tang", "blast"])
def test_contracted_fp64_within_tolerance(capi, orc, case, capsys):
    """The FP64 build with fused multiply-adds (fp64_contract = 1) against the
    oracle after 10 steps at full size, on the oracle's dt sequence: relative
    L-infinity error <= 1e-11 per variable (rounding differences only)."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    emf = 1 if case == "blast" else 0
    pr = synth.blast(128) if case == "blast" else synth.orszag_tang(128)
    ctx = capi.mhd_ctx_create(emf=emf, fp64_contract=1)
    try:
        p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx)
        run = PeriodicRunner(p, ctx)
        want = pr.state
        P = orc.patch(want, pr.n, pr.g, pr.dx)
        prm = orc.params(emf=emf)
        for _ in range(10):
            orc.fill_periodic(P)
            dt = orc.cfl_dt(P, prm)
            assert orc.advance(P, prm, dt, 0) == 0
            run.step(dt)
        got = p.state.cpu().numpy()
        err = rel_linf(got, want, pr.n, pr.g)
        with capsys.disabled():
            print("\ncontracted FP64 vs oracle, %s, 10 steps: max rel Linf %.2e" % (case, err.max()))
        assert np.all(err <= TOL), err
        assert capi.mhd_get_device_status(ctx) == 0
    finally:
        capi.mhd_ctx_destroy(ctx)


def _interior_totals(st, n, g):
    """FP64 totals of rho, M, E over the interior cells and of each face
    field over the faces of the interior (lower faces, plus the top face)."""
    nx, ny, nz = n
    a = st.astype(np.float64)
    cells = a[:5, g:g + nz, g:g + ny, g:g + nx].reshape(5, -1).sum(axis=1)
    bx = a[5, g:g + nz, g:g + ny, g:g + nx + 1].sum()
    by = a[6, g:g + nz, g:g + ny + 1, g:g + nx].sum()
    bz = a[7, g:g + nz + 1, g:g + ny, g:g + nx].sum()
    return np.concatenate([cells, [bx, by, bz]])


def _max_divb(st, n, g, dx):
    """max over interior cells of |div B| dx / max|B| (the CT invariant)."""
    nx, ny, nz = n
    a = st.astype(np.float64)
    bx = a[5, g:g + nz, g:g + ny, g:g + nx + 1]
    by = a[6, g:g + nz, g:g + ny + 1, g:g + nx]
    bz = a[7, g:g + nz + 1, g:g + ny, g:g + nx]
    div = (bx[:, :, 1:] - bx[:, :, :-1]) / dx[0] + (by[:, 1:, :] - by[:, :-1, :]) / dx[1] + \
        (bz[1:, :, :] - bz[:-1, :, :]) / dx[2]
    bmax = max(np.abs(bx).max(), np.abs(by).max(), np.abs(bz).max())
    return float(np.abs(div).max() * min(dx) / bmax)


@pytest.mark.parametrize("case", ["orszag_tang", "blast"])
def test_fp32_error_report(capi, orc, case, capsys):
    """FP32 bulk arithmetic against the FP64 oracle on the two single-patch
    workloads at full size (Orszag-Tang 128^2, blast 128^3), on the oracle's
    dt sequence: the error is reported per variable at steps 10 and 50 (L1
    and L-infinity, relative), with the FP32 run's relative drift of the
    totals and its max |div B| dx / max|B|.  No parity bar: loose sanity
    bounds only."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    emf = 1 if case == "blast" else 0
    pr = synth.blast(128) if case == "blast" else synth.orszag_tang(128)
    ctx = capi.mhd_ctx_create(emf=emf)
    try:
        p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx, dtype="f32")
        run = PeriodicRunner(p, ctx)
        want = pr.state
        P = orc.patch(want, pr.n, pr.g, pr.dx)
        prm = orc.params(emf=emf)
        tot0 = _interior_totals(p.state.cpu().numpy(), pr.n, pr.g)
        rows = []
        for step in range(1, 51):
            orc.fill_periodic(P)
            dt = orc.cfl_dt(P, prm)
            assert orc.advance(P, prm, dt, 0) == 0
            run.step(dt)
            if step in (10, 50):
                run.fill()
                orc.fill_periodic(P)
                got = p.state.cpu().numpy()
                tot = _interior_totals(got, pr.n, pr.g)
                scale = np.maximum(np.abs(tot0), np.abs(_interior_totals(np.abs(got), pr.n, pr.g)))
                drift = np.abs(tot - tot0) / np.maximum(scale, 1e-300)
                rows.append((step, rel_linf(got, want, pr.n, pr.g), rel_l1(got, want, pr.n, pr.g), drift,
                             _max_divb(got, pr.n, pr.g, pr.dx)))
        assert capi.mhd_get_device_status(ctx) == 0
    finally:
        capi.mhd_ctx_destroy(ctx)
    with capsys.disabled():
        for step, li, l1, drift, divb in rows:
            print("\nFP32 vs FP64 oracle, %s %s, step %d (rho Mx My Mz E Bx By Bz)" %
                  (case, "x".join(str(v) for v in pr.n if v > 1), step))
            print("  Linf rel :", " ".join("%.2e" % v for v in li))
            print("  L1   rel :", " ".join("%.2e" % v for v in l1))
            print("  drift    :", " ".join("%.2e" % v for v in drift), " max|divB|dx/|B|: %.2e" % divb)
    _, li, l1, drift, divb = rows[-1]
    live = [0, 1, 2, 4, 5, 6] + ([3, 7] if case == "blast" else [])
    assert np.all(l1[live] < 1e-3) and np.all(li[[0, 4]] < 5e-2)
    assert np.all(drift[[0, 4]] < 1e-5) and divb < 1e-4


@pytest.mark.parametrize("kernel", [1, 2, 4])
def test_batched_patches_equal_single_and_oracle(capi, orc, kernel):
    """Independent periodic patches of uneven sizes advanced in one call give
    the same bits as one call per patch, and match the oracle (staged and
    fused advance; the fused work queue mixes the patches' tiles)."""
    from paper_1112_1710_gb300.patch import periodic_copies
    ctx = capi.mhd_ctx_create(advance_kernel=kernel)
    sizes = [(8, 8, 8), (13, 9, 7), (24, 16, 12), (5, 5, 5)]
    probs = [random_state(n, 2, seed=20 + i) for i, n in enumerate(sizes)]
    dx = (0.05, 0.05, 0.05)
    batch = [to_patch(s, n, 2, dx, pid=i) for i, (s, n) in enumerate(zip(probs, sizes))]
    alone = [to_patch(s, n, 2, dx, pid=i) for i, (s, n) in enumerate(zip(probs, sizes))]
    d = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    descs = [p.desc() for p in batch]
    copies = []
    for i, n in enumerate(sizes):
        for c in periodic_copies(n, 2):
            c.src = c.dst = i
            copies.append(c)
    for _ in range(3):
        capi.mhd_ghost_fill(ctx, descs, copies)
        capi.mhd_patch_advance(ctx, descs, d.data_ptr())
        for p in alone:
            capi.mhd_ghost_fill(ctx, [p.desc()], periodic_copies(p.n, 2))
            capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr())
    for i, (s, n) in enumerate(zip(probs, sizes)):
        a = batch[i].state.cpu().numpy()
        b = alone[i].state.cpu().numpy()
        assert np.array_equal(a, b)
        orc.run_periodic(s, n, 2, dx, orc.params(), 3, dt=1e-3)
        capi.mhd_ghost_fill(ctx, [batch[i].desc()], periodic_copies(n, 2))
        err = rel_linf(batch[i].state.cpu().numpy(), s, n, 2)
        assert np.all(err <= TOL), (i, err)
    capi.mhd_ctx_destroy(ctx)


@pytest.mark.parametrize("kernel", [2, 4])
def test_fused_fp64_blast_10_steps(capi, orc, kernel):
    """The fused kernel (2) and the fused pass (4) in the FP64 parity build on
    the 3D blast (64^3, several 8 x 8 tiles, CFL dt every step) against the
    oracle after 10 steps."""
    pr = synth.blast(64)
    ctx = capi.mhd_ctx_create(emf=1, advance_kernel=kernel)
    try:
        got, want, gdts, odts = _run_both(capi, ctx, orc, pr, 10, emf=1)
        assert gdts == odts
        err = rel_linf(got, want, pr.n, pr.g)
        assert np.all(err <= TOL), err
        assert capi.mhd_get_device_status(ctx) == 0
    finally:
        capi.mhd_ctx_destroy(ctx)


def test_fused_fp32_chunking_invariant_and_close_to_staged(capi, capsys):
    """FP32: the fused kernel gives the same bits for any z-chunk length (every
    element is computed by the same code whatever the work decomposition), and
    stays within FP32 rounding of the staged kernels after 5 steps."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    pr = synth.blast(72)
    outs = {}
    for key, kernel, chunk in (("auto", 2, 0), ("c5", 2, 5), ("staged", 1, 0), ("pf", 4, 0), ("pf5", 4, 5)):
        ctx = capi.mhd_ctx_create(emf=1, advance_kernel=kernel, fused_chunk=chunk)
        try:
            p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx, dtype="f32")
            run = PeriodicRunner(p, ctx)
            for _ in range(5):
                run.step(2e-4)
            assert capi.mhd_get_device_status(ctx) == 0
            outs[key] = p.state.clone()
        finally:
            capi.mhd_ctx_destroy(ctx)
    assert torch.equal(outs["auto"], outs["c5"])
    assert torch.equal(outs["pf"], outs["pf5"])
    err = rel_linf(outs["auto"].cpu().numpy(), outs["staged"].cpu().numpy().astype(np.float64), pr.n, pr.g)
    errp = rel_linf(outs["pf"].cpu().numpy(), outs["staged"].cpu().numpy().astype(np.float64), pr.n, pr.g)
    with capsys.disabled():
        print("\nfused vs staged FP32, blast 72^3, 5 steps: max rel Linf %.2e (fused pass %.2e)"
              % (err.max(), errp.max()))
    assert err.max() <= 1e-5 and errp.max() <= 1e-5


def test_conservation_sums_within_summation_bound(capi, ctx, orc):
    pr = synth.blast(48)
    P = orc.patch(pr.state, pr.n, pr.g, pr.dx)
    orc.fill_periodic(P)
    want = orc.sums(P)
    p = to_patch(pr.state, pr.n, pr.g, pr.dx)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    capi.mhd_conservation_sums(ctx, [p.desc()], out.data_ptr())
    got = out.cpu().numpy()
    dv = pr.dx[0] * pr.dx[1] * pr.dx[2]
    absum = np.abs(pr.state[:, pr.g:pr.g + 48, pr.g:pr.g + 48, pr.g:pr.g + 48]).reshape(8, -1).sum(1) * dv
    ncell = 48 ** 3
    bound = 2 * ncell * np.finfo(np.float64).eps * absum
    assert np.all(np.abs(got - want) <= bound + 1e-300)
    # reproducible bit for bit
    out2 = torch.zeros(8, dtype=torch.float64, device="cuda")
    capi.mhd_conservation_sums(ctx, [p.desc()], out2.data_ptr())
    assert np.array_equal(out2.cpu().numpy(), got)


def test_negative_pressure_sets_status_without_trapping(capi, ctx):
    pr = synth.blast(16)
    st = pr.state.copy()
    st[4, 5, 6, 7] = -1.0  # total energy below the magnetic energy: p < 0
    p = to_patch(st, pr.n, pr.g, pr.dx)
    d = torch.full((1,), 1e-4, dtype=torch.float64, device="cuda")
    capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr())
    assert capi.mhd_get_device_status(ctx) == capi.MHD_ENEGATIVE
    assert capi.mhd_get_device_status(ctx) == 0  # cleared by the read
    # the context still works
    q = to_patch(pr.state, pr.n, pr.g, pr.dx)
    capi.mhd_patch_advance(ctx, [q.desc()], d.data_ptr())
    torch.cuda.synchronize()


def test_host_checks_reject_without_launch(capi, ctx):
    pr = synth.blast(8)
    p = to_patch(pr.state, pr.n, pr.g, pr.dx)
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    before = capi.mhd_launch_count(ctx)
    with pytest.raises(capi.MHDError) as e:
        capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr(), grow=[1])  # 1 + 2 > g = 2
    assert e.value.status == capi.MHD_EINVAL
    bad = p.desc()
    bad.stride[1] = 3
    with pytest.raises(capi.MHDError):
        capi.mhd_patch_advance(ctx, [bad], d.data_ptr())
    bad = p.desc()
    bad.dtype = 7
    with pytest.raises(capi.MHDError):
        capi.mhd_cfl_dt(ctx, [bad], d.data_ptr())
    assert capi.mhd_launch_count(ctx) == before
    # an empty advance is valid and launches nothing
    capi.mhd_patch_advance(ctx, [], d.data_ptr())
    assert capi.mhd_launch_count(ctx) == before


def test_autotune_keeps_state_and_stores_a_choice(capi):
    """The autotuner times both staged forms and every compiled fused shape
    without touching the patch state, stores the fastest in the context, and
    later advances agree with the staged kernels to FP32 rounding."""
    from paper_1112_1710_gb300.patch import periodic_copies
    pr = synth.blast(64)
    ctx = capi.mhd_ctx_create(emf=1)
    ref = capi.mhd_ctx_create(emf=1, advance_kernel=1)
    try:
        p = to_patch(pr.state, pr.n, pr.g, pr.dx, dtype="f32")
        q = to_patch(pr.state, pr.n, pr.g, pr.dx, dtype="f32")
        capi.mhd_ghost_fill(ctx, [p.desc()], periodic_copies(p.n, p.g))
        capi.mhd_ghost_fill(ctx, [q.desc()], periodic_copies(q.n, q.g))
        before = p.state.clone()
        d = torch.full((1,), 2e-4, dtype=torch.float64, device="cuda")
        v, cz, ms = capi.mhd_autotune_advance(ctx, [p.desc()], d.data_ptr(), reps=2)
        torch.cuda.synchronize()
        assert torch.equal(p.state, before)
        assert -6 <= v < 4 and (cz == 0 if v in (-2, -1) else 1 <= cz <= 66) and ms > 0.0
        capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr())
        capi.mhd_patch_advance(ref, [q.desc()], d.data_ptr())
        err = rel_linf(p.state.cpu().numpy(), q.state.cpu().numpy().astype(np.float64), pr.n, pr.g)
        assert err.max() <= 1e-6, (v, cz, err)
        if v == -2:  # the same kernels as the reference context
            assert torch.equal(p.state, q.state)
        p64 = to_patch(pr.state, pr.n, pr.g, pr.dx)
        capi.mhd_ghost_fill(ctx, [p64.desc()], periodic_copies(p64.n, p64.g))
        before64 = p64.state.clone()
        v64, cz64, _ = capi.mhd_autotune_advance(ctx, [p64.desc()], d.data_ptr(), reps=1)
        torch.cuda.synchronize()
        assert v64 in (-3, -2, -1, 0) and torch.equal(p64.state, before64)
        assert capi.mhd_get_device_status(ctx) == 0
    finally:
        capi.mhd_ctx_destroy(ctx)
        capi.mhd_ctx_destroy(ref)


@pytest.mark.parametrize("k", [0, 2])
def test_tiled_predictor_fp64_bitexact(capi, orc, k):
    """The staged path with the shared-memory-tiled predictor
    (advance_kernel = 3; tiles of 16 x 4 x 4 cells in FP64, ragged in all
    three axes) equals the oracle after one step."""
    n, g, dx = (37, 13, 11), 4, (0.05, 0.07, 0.06)
    st = random_state(n, g, seed=41 + k)
    ctx = capi.mhd_ctx_create(limiter=0, emf=0, advance_kernel=3)
    try:
        p = to_patch(st, n, g, dx)
        d = torch.full((1,), 1.1e-3, dtype=torch.float64, device="cuda")
        capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr(), grow=[k])
        assert capi.mhd_get_device_status(ctx) == 0
        got = p.state.cpu().numpy()
    finally:
        capi.mhd_ctx_destroy(ctx)
    P = orc.patch(st, n, g, dx)
    assert orc.advance(P, orc.params(limiter=0, emf=0), 1.1e-3, k) == 0
    assert np.array_equal(got, st)


@pytest.mark.parametrize("emf", [0, 1])
@pytest.mark.parametrize("k,chunk", [(0, 0), (2, 5), (1, 1)])
def test_fused_pass_fp64_equals_staged_bitexact(capi, k, chunk, emf):
    """The fused pass (advance_kernel = 4) computes every primitive, predicted
    state, half-step face field and flux with the staged kernels'
    expressions: in the FP64 parity build one step gives the staged bits on a
    ragged random patch (tiles ragged in x and y, z chunks of 16, 5 and 1
    planes), the whole array included."""
    n, g, dx = (23, 17, 14), 4, (0.05, 0.07, 0.06)
    st = random_state(n, g, seed=61 + k)
    out = []
    for kernel in (1, 4):
        ctx = capi.mhd_ctx_create(limiter=2, emf=emf, advance_kernel=kernel, fused_chunk=chunk)
        try:
            p = to_patch(st, n, g, dx)
            d = torch.full((1,), 1.2e-3, dtype=torch.float64, device="cuda")
            capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr(), grow=[k])
            assert capi.mhd_get_device_status(ctx) == 0
            out.append(p.state.cpu().numpy())
        finally:
            capi.mhd_ctx_destroy(ctx)
    assert np.array_equal(out[0], out[1])


def test_fused_pass_fp32_shapes(capi, capsys):
    """Every compiled FP32 tile shape of the fused pass (kernel_shape 1-4):
    the same bits for two z-chunk lengths, and within FP32 rounding of the
    staged kernels after 3 steps of the 48^3 blast; a shape outside the FP64
    table is refused at the call."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    pr = synth.blast(48)

    def run(**kw):
        ctx = capi.mhd_ctx_create(emf=1, **kw)
        try:
            p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx, dtype="f32")
            r = PeriodicRunner(p, ctx)
            for _ in range(3):
                r.step(3e-4)
            assert capi.mhd_get_device_status(ctx) == 0
            return p.state.clone()
        finally:
            capi.mhd_ctx_destroy(ctx)
    ref = run(advance_kernel=1).cpu().numpy().astype(np.float64)
    worst = []
    for shape in (1, 2, 3, 4):
        a = run(advance_kernel=4, kernel_shape=shape, fused_chunk=0)
        b = run(advance_kernel=4, kernel_shape=shape, fused_chunk=5)
        assert torch.equal(a, b), shape
        err = rel_linf(a.cpu().numpy(), ref, pr.n, pr.g)
        worst.append(err.max())
        assert err.max() <= 1e-5, (shape, err)
    with capsys.disabled():
        print("\nfused pass FP32 shapes vs staged, blast 48^3, 3 steps: max rel Linf " +
              " ".join("%.2e" % w for w in worst))
    ctx = capi.mhd_ctx_create(advance_kernel=4, kernel_shape=2)
    try:
        p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx)
        d = torch.full((1,), 1e-4, dtype=torch.float64, device="cuda")
        before = p.state.clone()
        with pytest.raises(capi.MHDError):
            capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr())
        torch.cuda.synchronize()
        assert torch.equal(p.state, before)
    finally:
        capi.mhd_ctx_destroy(ctx)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", ["ragged", "blast64"])
def test_cfl_in_primitive_pass_equals_separate_cfl(capi, dtype, case):
    """mhd_patch_step_cfl (the CFL reduction inside k_prim) against
    mhd_cfl_dt + mhd_patch_advance on the same states: the same dt and state
    bit for bit in the FP64 parity build; in FP32 (fast math in k_prim, not in
    the separate reduction) the dt within 1e-6 and the state within 1e-5."""
    from paper_1112_1710_gb300.runner import PeriodicRunner
    if case == "ragged":
        n, g, dx = (37, 29, 23), 2, (1.0 / 37, 1.3 / 29, 0.9 / 23)
        st = random_state(n, g, seed=77)
        ctx = capi.mhd_ctx_create()
    else:
        pr = synth.blast(64)
        n, g, dx, st = pr.n, pr.g, pr.dx, pr.state
        ctx = capi.mhd_ctx_create(emf=1)
    try:
        out = []
        for fused in (True, False):
            p = to_patch(st.copy(), n, g, dx, dtype=dtype)
            run = PeriodicRunner(p, ctx, cfl_in_step=fused)
            dts = run.run(3, record_dt=True)
            out.append((dts, p.state.cpu().numpy()))
        assert capi.mhd_get_device_status(ctx) == 0
    finally:
        capi.mhd_ctx_destroy(ctx)
    (d1, s1), (d2, s2) = out
    if dtype == "f64":
        assert d1 == d2
        assert np.array_equal(s1, s2)
    else:
        assert np.allclose(d1, d2, rtol=1e-6, atol=0)
        err = rel_linf(s1.astype(np.float64), s2.astype(np.float64), n, g)
        assert np.all(err <= 1e-5), err


def _interior_face_energy(s, n, g):
    """Sum of squared interior face fields (the loop's magnetic energy up to
    a constant factor and the face-to-cell averaging)."""
    tot = 0.0
    for a in range(3):
        ext = list(n)
        ext[a] += 1
        tot += float(np.sum(s[5 + a, g:g + ext[2], g:g + ext[1], g:g + ext[0]] ** 2))
    return tot


@pytest.mark.parametrize("normal", [0, 1, 2])
def test_field_loop_gs05_fp64_and_fp32(capi, orc, normal):
    """The field loop that pins the upwinded edge EMF (Gardiner & Stone 2005)
    in each coordinate plane, carried along the diagonal of its plane, 20
    steps with the default (upwinded) EMF: FP64 equals the oracle within
    1e-11 per variable with the same dt sequence; FP32 keeps the pinned
    property (the loop's magnetic energy never rises) and its field stays
    within 1e-4 of the oracle's field strength."""
    t1, t2 = (normal + 1) % 3, (normal + 2) % 3
    v = [0.0, 0.0, 0.0]
    v[t1], v[t2] = 1.0, 0.5
    pr = synth.field_loop(32, normal, tuple(v))
    res = {}
    for dtype in ("f64", "f32"):
        ctx = capi.mhd_ctx_create(emf=0)
        try:
            from paper_1112_1710_gb300.runner import PeriodicRunner
            p = to_patch(pr.state.copy(), pr.n, pr.g, pr.dx, dtype=dtype)
            run = PeriodicRunner(p, ctx)
            eb = []
            dts = []
            for _ in range(20):
                dts += run.run(1, record_dt=True)
                s = p.state.cpu().numpy().astype(np.float64)
                eb.append(_interior_face_energy(s, pr.n, pr.g))
            assert capi.mhd_get_device_status(ctx) == 0
            res[dtype] = (p.state.cpu().numpy(), dts, np.array(eb))
        finally:
            capi.mhd_ctx_destroy(ctx)
    want = pr.state.copy()
    odts = orc.run_periodic(want, pr.n, pr.g, pr.dx, orc.params(emf=0), 20)
    got64, dts64, _ = res["f64"]
    assert dts64 == odts
    err = rel_linf(got64, want, pr.n, pr.g)
    assert np.all(err[5:] <= TOL), err
    assert np.all(err[:5] <= TOL), err
    got32, _, eb32 = res["f32"]
    assert np.all(np.diff(eb32) <= 1e-5 * eb32[0]), eb32
    g = pr.g
    nx, ny, nz = pr.n
    for a in range(3):
        ext = [nx, ny, nz]
        ext[a] += 1
        d = np.abs(got32[5 + a, g:g + ext[2], g:g + ext[1], g:g + ext[0]] -
                   want[5 + a, g:g + ext[2], g:g + ext[1], g:g + ext[0]]).max()
        assert d <= 1e-4 * 1e-3, (a, d)


@pytest.mark.parametrize("kernel", [1, 2, 4])
def test_pressure_floor_equals_oracle(capi, orc, kernel):
    """The optional pressure floor (mhd_params.p_floor) after the staged (1),
    the fused (2) and the fused-pass (4) advance: FP64 equals the oracle bit for bit and raises
    the same number of cells (mhd_floor_count)."""
    pr = synth.blast(12, noise=0.01, seed=4)
    n, g = pr.n, pr.g
    st = pr.state.copy()
    P = orc.patch(st, n, g, pr.dx)
    orc.fill_periodic(P)
    dt = orc.cfl_dt(P, orc.params(emf=1))
    ctx = capi.mhd_ctx_create(emf=1, p_floor=0.099, advance_kernel=kernel)
    try:
        p = to_patch(st, n, g, pr.dx)
        d = torch.full((1,), dt, dtype=torch.float64, device="cuda")
        capi.mhd_patch_advance(ctx, [p.desc()], d.data_ptr())
        nfl = capi.mhd_floor_count(ctx)
        assert capi.mhd_floor_count(ctx) == 0          # the count resets
        got = p.state.cpu().numpy()
    finally:
        capi.mhd_ctx_destroy(ctx)
    assert orc.advance(P, orc.params(emf=1, p_floor=0.099), dt, 0) == 0
    assert nfl == orc.floor_count() > 0
    err = rel_linf(got, st, n, g)
    assert np.all(err <= TOL), err


def test_level_floor_equals_oracle(capi, orc):
    """mhd_floor (the floors over whole interiors, used after refluxing)
    equals orc_floor bit for bit in FP64, cell count included."""
    pr = synth.blast(12, noise=0.01, seed=5)
    n, g = pr.n, pr.g
    st = pr.state.copy()
    P = orc.patch(st, n, g, pr.dx)
    orc.fill_periodic(P)
    st[0, g + 1, g + 2, g + 3] = 1e-6
    ctx = capi.mhd_ctx_create(p_floor=0.2, rho_floor=1e-3)
    try:
        p = to_patch(st, n, g, pr.dx)
        capi.mhd_floor(ctx, [p.desc()])
        nch = capi.mhd_floor_count(ctx)
        got = p.state.cpu().numpy()
    finally:
        capi.mhd_ctx_destroy(ctx)
    want_n = orc.floor(P, orc.params(p_floor=0.2, rho_floor=1e-3))
    assert nch == want_n > 1
    assert np.array_equal(got[:, :n[2] + 2 * g + 1, :n[1] + 2 * g + 1, :n[0] + 2 * g + 1],
                          st[:, :n[2] + 2 * g + 1, :n[1] + 2 * g + 1, :n[0] + 2 * g + 1])
