"""Host-side checks of the serving scheduler against a simulated device.

The simulated backend finishes a batch after a time proportional to its
cells on a virtual clock, so the policy (finer levels first, HBM-budget
admission, single-precision batches, overlap of batches on free slots) is
checked without a GPU.
"""
import math
import types

import numpy as np
import pytest

from paper_1112_1710_gb300 import capi
from paper_1112_1710_gb300.patch import periodic_copies
from paper_1112_1710_gb300.serve import (GpuBackend, Request, Scheduler, latency_stats, poisson_requests,
                                         state_bytes)


class Clock:
    """Virtual time: every read advances it by `tick` seconds."""

    def __init__(self, tick=1e-5):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t


class SimBackend:
    def __init__(self, clock, rate=1e9):
        self.clock = clock
        self.rate = rate
        self.launched = []           # (slot, t_start, t_end, [rids])
        self.busy_until = {}

    def launch(self, slot, batch):
        t = self.clock.t
        t_end = t + sum(r.cells for r in batch) / self.rate
        self.launched.append((slot, t, t_end, [r.rid for r in batch]))
        return (t_end, [r.rid for r in batch])

    def ready(self, h):
        return self.clock.t >= h[0]

    def finish(self, h):
        return ["out%d" % rid for rid in h[1]]


def run(reqs, **kw):
    clk = Clock()
    be = SimBackend(clk, rate=kw.pop("rate", 1e9))
    sch = Scheduler(be, **kw)
    out = sch.run(reqs, clock=clk, t_limit=1e6)
    return out, sch, be


def test_poisson_stream_shape():
    reqs = poisson_requests(20000, rate=1000.0, seed=4242)
    n = np.array([r.n for r in reqs])
    assert n.min() >= 16 and n.max() <= 128 and np.all(n % 2 == 0)
    # log-uniform: the median edge is near the geometric mean of the range
    assert abs(np.median(n) - math.sqrt(16 * 128)) < 3
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert abs(gaps.mean() * 1000.0 - 1.0) < 0.03
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05      # exponential gaps
    lev = np.array([r.level for r in reqs])
    assert set(lev.tolist()) == set(range(8))
    f32 = np.mean([r.dtype == "f32" for r in reqs])
    assert abs(f32 - 0.5) < 0.02
    assert all(r.arrival == 0.0 for r in poisson_requests(10, math.inf))


def test_finer_levels_first():
    reqs = [Request(i, 0.0, 16, (i * 5) % 8, "f64") for i in range(40)]
    out, sch, be = run(reqs, n_slots=1, max_batch_cells=1)   # one request per batch
    order = [rid for (_, rids) in sch.batches for rid in rids]
    key = [(-reqs[i].level, i) for i in order]
    assert key == sorted(key)
    assert all(r.done >= r.start >= r.arrival for r in out)


def test_batches_single_precision_and_bounded():
    reqs = poisson_requests(500, rate=2e4, seed=7)
    out, sch, be = run(reqs, n_slots=3, max_batch_cells=1 << 20)
    by = {r.rid: r for r in out}
    seen = []
    for _, rids in sch.batches:
        assert len({by[i].dtype for i in rids}) == 1
        cells = sum(by[i].cells for i in rids)
        assert cells <= 1 << 20 or len(rids) == 1
        seen += rids
    assert sorted(seen) == list(range(500))                  # every request exactly once
    assert all(r.result == "out%d" % r.rid for r in out)


def test_hbm_budget_admission_and_rejection():
    big = state_bytes(128, 4, "f64")
    budget = 3 * big
    reqs = [Request(i, 0.0, 128, 0, "f64") for i in range(10)]
    reqs.append(Request(10, 0.0, 128, 7, "f64"))
    out, sch, be = run(reqs, n_slots=8, budget_bytes=budget, max_batch_cells=1 << 30)
    assert sch.peak_resident <= budget
    assert sch.resident == 0
    assert not any(r.error for r in out)
    # a request that could never fit is rejected without a launch
    r2 = [Request(0, 0.0, 128, 0, "f64"), Request(1, 0.0, 16, 0, "f32")]
    out, sch, be = run(r2, budget_bytes=state_bytes(64, 4, "f64"))
    assert out[0].error and not out[1].error
    assert [rids for _, rids in sch.batches] == [[1]]


def test_continuous_batching_overlaps():
    # a long FP64 batch is running when a short FP32 request arrives; the
    # latter starts on the second slot before the former has finished
    reqs = [Request(0, 0.0, 128, 0, "f64"), Request(1, 1e-4, 16, 0, "f32")]
    out, sch, be = run(reqs, n_slots=2, rate=1e8)
    (s0, t0, e0, r0), (s1, t1, e1, r1) = be.launched
    assert r0 == [0] and r1 == [1] and s0 != s1
    assert t1 < e0 and out[1].done < out[0].done


def test_latency_stats():
    reqs = poisson_requests(300, rate=5e3, seed=3)
    out, sch, be = run(reqs, n_slots=2)
    st = latency_stats(out)
    assert st["count"] == 300 and st["p99_ms"] >= st["p50_ms"] > 0
    assert sum(b["n"] for b in st["by_size"].values()) == 300
    assert set(st["by_size"]) <= {"16-32", "32-64", "64-128"}


def test_batch_copy_list_layout():
    fake = types.SimpleNamespace(capi=capi, g=4, _copies={})
    ns = [16, 30, 16, 128]
    arr, total = GpuBackend.copies(fake, ns)
    expect = []
    for i, n in enumerate(ns):
        expect += [(i, i, tuple(c.box.lo), tuple(c.box.hi), tuple(c.offset)) for c in periodic_copies((n,) * 3, 4)]
    got = [(arr[j].src, arr[j].dst, tuple(arr[j].box.lo), tuple(arr[j].box.hi), tuple(arr[j].offset))
           for j in range(total)]
    assert got == expect


def test_balanced_policy_sizes_batches_by_the_distribution_equation():
    """With one slot busy on a large batch, the balanced policy gives the free
    slot a larger share of the waiting work (equal predicted remaining work),
    never beyond the batch cap, and every request is still served once."""
    from paper_1112_1710_gb300.balance import desired_distribution
    reqs = [Request(i, 0.0, 32, 0, "f32") for i in range(64)]
    out, sch, be = run(reqs, n_slots=2, max_batch_cells=1 << 20, policy="balanced", min_batch_cells=1 << 14)
    assert sorted(r for _, rids in sch.batches for r in rids) == list(range(64))
    assert all(sum(out[i].cells for i in rids) <= 1 << 20 for _, rids in sch.batches)
    # the share of a free slot next to a busy one: gbar + (inflight busy) / 2
    d = desired_distribution(1000.0, [[0, 600]], [[0, 0]], [1, 1], 1)
    assert np.allclose(d, [1300, 700])
    with pytest.raises(ValueError):
        Scheduler(SimBackend(Clock()), policy="other")


class FlakyBackend(SimBackend):
    """Raises on the launches whose index is in `fail` (a host-side failure:
    nothing of that batch reaches the device)."""

    def __init__(self, clock, fail, **kw):
        super().__init__(clock, **kw)
        self.fail = set(fail)
        self.calls = 0

    def launch(self, slot, batch):
        self.calls += 1
        if self.calls in self.fail:
            raise RuntimeError("launch %d rejected" % self.calls)
        return super().launch(slot, batch)


def test_failed_launch_is_requeued_then_reported():
    clk = Clock()
    be = FlakyBackend(clk, fail={1, 3})
    sch = Scheduler(be, n_slots=2, max_batch_cells=1 << 15, max_retries=2)
    reqs = [Request(i, 0.0, 16, i % 3, "f32") for i in range(20)]
    out = sch.run(reqs, clock=clk, t_limit=1e6)
    assert len(sch.failures) == 2
    assert not any(r.error for r in out)                      # every request served after a retry
    assert sorted(r for _, rids in sch.batches for r in rids) == list(range(20))
    assert sch.resident == 0
    # a backend that always fails: requests end as errors, the loop ends
    clk = Clock()
    bad = FlakyBackend(clk, fail=set(range(1, 100)))
    sch = Scheduler(bad, n_slots=2, max_retries=1)
    out = sch.run([Request(i, 0.0, 16, 0, "f64") for i in range(3)], clock=clk, t_limit=1e6)
    assert all(r.error.startswith("failed 2 launches") for r in out)
    assert sch.batches == [] and sch.resident == 0
