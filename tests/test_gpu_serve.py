"""The served, continuously batched path on the GPU: every request's result is
the same in the mix as alone (bit-identical, FP32 and FP64), a served FP64
request matches the oracle, and a Poisson stream reports latencies."""
import math

import numpy as np
import pytest
import torch

import synth
from gpu_util import rel_l1, rel_linf

pytestmark = pytest.mark.gpu
G = 4
SOLVER = dict(gamma=5.0 / 3.0, cfl=0.4, limiter=0, emf=1)
SIZES = (16, 18, 24, 32, 40)


@pytest.fixture(scope="module")
def templates():
    from paper_1112_1710_gb300 import _build, capi
    _build.build()
    capi.load()
    from paper_1112_1710_gb300.serve import make_templates
    return make_templates(SIZES, g=G, solver=SOLVER)


def _stream(count, rate, seed):
    from paper_1112_1710_gb300.serve import Request
    rng = np.random.default_rng(seed)
    t = np.zeros(count) if math.isinf(rate) else np.cumsum(rng.exponential(1.0 / rate, count))
    return [Request(i, float(t[i]), int(rng.choice(SIZES)), int(rng.integers(0, 8)),
                    "f32" if rng.random() < 0.5 else "f64") for i in range(count)]


@pytest.mark.parametrize("rate", [math.inf, 2000.0])
def test_mix_equals_alone(templates, rate):
    from paper_1112_1710_gb300 import capi
    from paper_1112_1710_gb300.serve import GpuBackend, Scheduler
    be = GpuBackend(templates, n_slots=3, g=G, solver=SOLVER, keep=True)
    try:
        sch = Scheduler(be, n_slots=3, max_batch_cells=120_000, g=G)
        reqs = sch.run(_stream(48, rate, seed=11), t_limit=120.0)
        torch.cuda.synchronize()
        assert len(sch.batches) >= 4
        assert any(len(rids) > 1 for _, rids in sch.batches)
        by = {r.rid: r for r in reqs}
        assert any(len({by[i].n for i in rids}) > 1 for _, rids in sch.batches)   # uneven sizes in one batch
        for c in be.ctxs:
            assert capi.mhd_get_device_status(c) == 0
        for r in reqs:
            alone = be.alone(r)
            assert torch.equal(r.result, alone), (r.rid, r.n, r.dtype)
    finally:
        be.close()


def test_served_fp64_matches_oracle(templates, orc):
    from paper_1112_1710_gb300.serve import GpuBackend, Request, Scheduler
    be = GpuBackend(templates, n_slots=2, g=G, solver=SOLVER, keep=True)
    try:
        reqs = [Request(0, 0.0, 24, 3, "f64"), Request(1, 0.0, 16, 5, "f64"), Request(2, 0.0, 18, 1, "f32")]
        Scheduler(be, n_slots=2, g=G).run(reqs, t_limit=60.0)
        torch.cuda.synchronize()
        for r in reqs[:2]:
            pr = synth.blast(r.n, g=G, seed=4242 + r.n)
            _, dt = templates[(r.n, "f64")]
            P = orc.patch(pr.state, pr.n, G, pr.dx)
            orc.fill_periodic(P)
            assert orc.advance(P, orc.params(**SOLVER), dt, 0) == 0
            err = rel_linf(r.result.cpu().numpy(), pr.state, pr.n, G)
            assert err.max() <= 1e-11, err
    finally:
        be.close()


def test_poisson_latency_report(templates):
    from paper_1112_1710_gb300.serve import GpuBackend, Scheduler, latency_stats
    be = GpuBackend(templates, n_slots=2, g=G, solver=SOLVER)
    try:
        sch = Scheduler(be, n_slots=2, g=G, max_batch_cells=200_000)
        reqs = sch.run(_stream(200, 4000.0, seed=5), t_limit=120.0)
        st = latency_stats(reqs)
        assert st["count"] == 200 and st["p99_ms"] >= st["p50_ms"] > 0
        assert st["cell_updates_per_s"] > 0
        assert sch.resident == 0
    finally:
        be.close()


def test_served_contracted_fp64_and_fp32_error_vs_oracle(templates, orc, capsys):
    """Served FP64 requests on the contracted build (fused multiply-adds,
    reciprocal HLLD) are within 1e-11 of the oracle per variable; served FP32
    requests report their per-variable error against the FP64 oracle (L1 and
    L-infinity relative), bounded by 1e-5 (one step of FP32 rounding)."""
    from paper_1112_1710_gb300.serve import GpuBackend, Request, Scheduler
    be = GpuBackend(templates, n_slots=2, g=G, solver=dict(SOLVER, fp64_contract=1), keep=True)
    try:
        reqs = [Request(0, 0.0, 24, 3, "f64"), Request(1, 0.0, 40, 5, "f64"), Request(2, 0.0, 32, 1, "f32"),
                Request(3, 0.0, 40, 6, "f32")]
        Scheduler(be, n_slots=2, g=G).run(reqs, t_limit=60.0)
        torch.cuda.synchronize()
        linf32 = np.zeros(8)
        l1_32 = np.zeros(8)
        for r in reqs:
            pr = synth.blast(r.n, g=G, seed=4242 + r.n)
            _, dt = templates[(r.n, "f64")]
            P = orc.patch(pr.state, pr.n, G, pr.dx)
            orc.fill_periodic(P)
            assert orc.advance(P, orc.params(**SOLVER), dt, 0) == 0
            got = r.result.cpu().numpy().astype(np.float64)
            err = rel_linf(got, pr.state, pr.n, G)
            if r.dtype == "f64":
                assert err.max() <= 1e-11, err
            else:
                linf32 = np.maximum(linf32, err)
                l1_32 = np.maximum(l1_32, rel_l1(got, pr.state, pr.n, G))
        with capsys.disabled():
            print("\nserved FP32 requests (32^3, 40^3 blast cubes, one step) vs FP64 oracle "
                  "(rho Mx My Mz E Bx By Bz)")
            print("  Linf rel : " + " ".join("%.2e" % v for v in linf32))
            print("  L1   rel : " + " ".join("%.2e" % v for v in l1_32))
        assert np.all(linf32 <= 1e-5) and np.all(l1_32 <= 1e-6), (linf32, l1_32)
    finally:
        be.close()


def test_balanced_policy_mix_equals_alone(templates):
    """The serving policy that sizes each slot's batch by the distribution
    equation of Sec. 5 (balanced) on the GPU backend: every result equals
    the same request run alone, and the batches' sizes follow the policy."""
    from paper_1112_1710_gb300 import capi
    from paper_1112_1710_gb300.serve import GpuBackend, Scheduler
    be = GpuBackend(templates, n_slots=3, g=G, solver=SOLVER, keep=True)
    try:
        sch = Scheduler(be, n_slots=3, max_batch_cells=200_000, min_batch_cells=4096, g=G, policy="balanced")
        reqs = sch.run(_stream(60, math.inf, seed=21), t_limit=120.0)
        torch.cuda.synchronize()
        assert len(sch.batches) >= 3
        for c in be.ctxs:
            assert capi.mhd_get_device_status(c) == 0
        by = {r.rid: r for r in reqs}
        assert sum(len(rids) for _, rids in sch.batches) == 60
        for _, rids in sch.batches:
            # a batch exceeds its cell budget only when a single request does
            assert len(rids) == 1 or sum(by[i].cells for i in rids) <= 200_000
        for r in reqs:
            assert torch.equal(r.result, be.alone(r)), (r.rid, r.n, r.dtype)
    finally:
        be.close()
