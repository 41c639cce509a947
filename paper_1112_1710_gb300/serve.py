"""Continuous-batching server of patch-advance requests on one GPU.

A request asks for one step (ghost fill + advance) of a ghost-celled periodic
patch of a given cube size, refinement level and precision, with the dt it
was given.  The server

  * orders waiting requests finer level first (the paper's scheduler gives the
    threads of finer levels priority over coarser ones, Sec. 4), then by
    arrival;
  * admits a request only when its resident state fits an HBM budget, and
    rejects on arrival one that could never fit;
  * forms a batch of waiting requests of one precision (up to a cell budget)
    whenever one of its slots (a CUDA stream with its own library context,
    i.e. its own scratch arena) is idle, so that requests that arrive while
    other batches are on the GPU start as soon as a slot and memory free up
    and their work overlaps on the device;
  * runs a batch as one ghost fill and one batched advance over all of its
    patches (uneven sizes in one launch), each patch with its own dt passed
    as its dt scale (device dt = 1), so no patch's arithmetic depends on the
    mix;
  * records arrival, start and completion times for p50/p99 latencies;
  * requeues the requests of a launch that raised (a host-side failure: a
    rejected descriptor, an allocation that failed) up to max_retries times,
    then reports them as failed instead of stopping the loop.

The policy (`Scheduler`) is plain host code; the device side is a backend
with `launch(slot, batch)` and `ready(handle)`, so the policy runs unchanged
against a simulated backend on a CPU.
"""
from __future__ import annotations

import ctypes
import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float          # s, relative to the start of the run
    n: int                  # cube edge (cells)
    level: int              # refinement level (priority: finer first)
    dtype: str              # "f32" or "f64"
    start: float = math.nan
    done: float = math.nan
    error: str = ""
    result: object = field(default=None, repr=False)

    @property
    def cells(self) -> int:
        return self.n ** 3


def poisson_requests(count, rate, n_min=16, n_max=128, levels=8, seed=4242):
    """`count` requests with Poisson arrivals at `rate` per second (all at t = 0
    when rate is infinite), cube edges log-uniform in [n_min, n_max] rounded to
    even, levels uniform in [0, levels), precision FP32 or FP64 with equal
    odds."""
    rng = np.random.default_rng(seed)
    if math.isinf(rate):
        t = np.zeros(count)
    else:
        t = np.cumsum(rng.exponential(1.0 / rate, count))
    edge = np.exp(rng.uniform(math.log(n_min), math.log(n_max), count))
    edge = np.clip(2 * np.rint(edge / 2), n_min, n_max).astype(int)
    lev = rng.integers(0, levels, count)
    f32 = rng.random(count) < 0.5
    return [Request(i, float(t[i]), int(edge[i]), int(lev[i]), "f32" if f32[i] else "f64")
            for i in range(count)]


def state_bytes(n, g, dtype):
    """Bytes of one resident patch state of cube edge n with g ghost layers
    (the (8, NZ+1, NY+1, PX) layout with PX padded to 8)."""
    N = n + 2 * g
    px = -(-(N + 1) // 8) * 8
    return 8 * (N + 1) * (N + 1) * px * (4 if dtype == "f32" else 8)


class Scheduler:
    """Finer-first, HBM-budgeted continuous batching over `n_slots` slots."""

    def __init__(self, backend, n_slots=2, budget_bytes=64 << 30, max_batch_cells=8 << 20, g=4,
                 lookahead=64, policy="greedy", min_batch_cells=1 << 16, max_retries=2):
        """policy "greedy": a free slot takes up to max_batch_cells of waiting
        work; "balanced": its share from the distribution equation of Sec. 5
        with the slots as workers (balance.desired_distribution), so that the
        slots' predicted remaining work (in-flight cells plus the new batch)
        evens out, clamped to [min_batch_cells, max_batch_cells]."""
        if policy not in ("greedy", "balanced"):
            raise ValueError("policy must be greedy or balanced")
        self.policy = policy
        self.min_batch_cells = min_batch_cells
        self.max_retries = max_retries
        self.failures = []           # (slot, [rid, ...], error text) of launches that raised
        self.backend = backend
        self.n_slots = n_slots
        self.budget = budget_bytes
        self.max_batch_cells = max_batch_cells
        self.g = g
        self.lookahead = lookahead
        self.resident = 0
        self.peak_resident = 0
        self.batches = []            # (slot, [rid, ...]) in launch order

    def _cell_budget(self, slot, slots, waiting):
        """Cells the next batch of `slot` may take."""
        if self.policy == "greedy":
            return self.max_batch_cells
        from .balance import desired_distribution
        inflight = [sum(r.cells for r in f[1]) if f is not None else 0 for f in slots]
        pending = sum(item[3].cells for item in waiting)
        gbar = pending / self.n_slots
        d = desired_distribution(gbar, [inflight], [[0] * self.n_slots], [1, 1], 1)
        return int(min(self.max_batch_cells, max(self.min_batch_cells, d[slot])))

    def _form_batch(self, waiting, budget=None):
        """Pops the next batch off the waiting heap: the head request fixes the
        precision; the rest join in priority order while the batch stays
        under the cell budget and the resident state under the HBM budget."""
        budget = self.max_batch_cells if budget is None else budget
        dtype = waiting[0][3].dtype
        batch, cells, nbytes, skipped = [], 0, 0, []
        while waiting and len(skipped) <= self.lookahead:
            item = heapq.heappop(waiting)
            r = item[3]
            b = state_bytes(r.n, self.g, r.dtype)
            ok = r.dtype == dtype and self.resident + nbytes + b <= self.budget and (
                not batch or cells + r.cells <= budget)
            if ok:
                batch.append(r)
                cells += r.cells
                nbytes += b
            else:
                skipped.append(item)
        for item in skipped:
            heapq.heappush(waiting, item)
        return batch, nbytes

    def run(self, requests, t_limit=600.0, clock=time.perf_counter):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        waiting = []                             # heap of (-level, arrival, rid, request)
        slots = [None] * self.n_slots            # (handle, batch, bytes)
        nxt = done = 0
        t0 = clock()
        while done < len(reqs):
            now = clock() - t0
            if now > t_limit:
                raise TimeoutError("serving run exceeded %.0f s" % t_limit)
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                r = reqs[nxt]
                nxt += 1
                if state_bytes(r.n, self.g, r.dtype) > self.budget:
                    r.error = "rejected: state larger than the HBM budget"
                    r.start = r.done = now
                    done += 1
                    continue
                heapq.heappush(waiting, (-r.level, r.arrival, r.rid, r))
            for s, f in enumerate(slots):
                if f is not None and self.backend.ready(f[0]):
                    tnow = clock() - t0
                    for r, res in zip(f[1], self.backend.finish(f[0])):
                        r.done = tnow
                        r.result = res
                    self.resident -= f[2]
                    done += len(f[1])
                    slots[s] = None
            for s in range(self.n_slots):
                if slots[s] is not None or not waiting:
                    continue
                batch, nbytes = self._form_batch(waiting, self._cell_budget(s, slots, waiting))
                if not batch:
                    break                        # nothing fits until memory frees up
                tstart = clock() - t0
                for r in batch:
                    r.start = tstart
                try:
                    handle = self.backend.launch(s, batch)
                except Exception as exc:  # a failed launch: nothing of it is in flight
                    self.failures.append((s, [r.rid for r in batch], str(exc)))
                    for r in batch:
                        r.retries = getattr(r, "retries", 0) + 1
                        if r.retries > self.max_retries:
                            r.error = "failed %d launches: %s" % (r.retries, exc)
                            r.done = clock() - t0
                            done += 1
                        else:
                            heapq.heappush(waiting, (-r.level, r.arrival, r.rid, r))
                    continue
                self.resident += nbytes
                self.peak_resident = max(self.peak_resident, self.resident)
                self.batches.append((s, [r.rid for r in batch]))
                slots[s] = (handle, batch, nbytes)
            if all(f is None for f in slots) and not waiting and nxt < len(reqs):
                wait = reqs[nxt].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        return reqs


class GpuBackend:
    """Runs batches through the C ABI, one stream and one context per slot.

    Initial states are copied device-to-device from resident templates, one
    per (cube edge, precision), built from the seeded blast-wave generator.
    With `keep=True` each request's final state stays on the device (for the
    mix-versus-alone check); otherwise it is released when the batch ends.
    """

    def __init__(self, templates, n_slots=2, g=4, solver=None, keep=False, device="cuda"):
        import torch
        from . import capi
        self.torch, self.capi = torch, capi
        self.templates = templates
        self.g = g
        self.keep = keep
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self._solver = dict(solver or {})
        self.ctxs = [capi.mhd_ctx_create(**self._solver) for _ in range(n_slots)]
        self.d_one = torch.ones(1, dtype=torch.float64, device=self.device)
        self._copies = {}
        self.kernel_calls = 0

    def close(self):
        for c in self.ctxs:
            self.capi.mhd_ctx_destroy(c)
        self.ctxs = []

    def copies(self, ns):
        """Ghost-fill copy list of a batch of periodic cubes with edges `ns`
        (patch i copies onto itself), as a (ctypes array, count) pair built
        from one cached list per edge."""
        from .patch import periodic_copies
        C, capi = ctypes, self.capi
        rec = C.sizeof(capi.mhd_copy)
        base = []
        for n in ns:
            b = self._copies.get(n)
            if b is None:
                lst = periodic_copies((n, n, n), self.g)
                b = self._copies[n] = ((capi.mhd_copy * len(lst))(*lst), len(lst))
            base.append(b)
        total = sum(k for _, k in base)
        arr = (capi.mhd_copy * max(1, total))()
        off = 0
        for b, k in base:
            C.memmove(C.addressof(arr) + off * rec, b, k * rec)
            off += k
        ids = np.frombuffer(arr, dtype=np.int32).reshape(max(1, total), rec // 4)
        ids[:total, 0:2] = np.repeat(np.arange(len(ns), dtype=np.int32), [k for _, k in base])[:, None]
        return arr, total

    def launch(self, slot, batch):
        torch, capi = self.torch, self.capi
        from .patch import Patch
        s = self.streams[slot]
        ctx = self.ctxs[slot]
        patches, descs, scales = [], [], []
        with torch.cuda.stream(s):
            for i, r in enumerate(batch):
                tpl, dt = self.templates[(r.n, r.dtype)]
                st = torch.empty_like(tpl.state)
                st.copy_(tpl.state, non_blocking=True)
                p = Patch(st, tpl.lo, tpl.n, tpl.g, tpl.dx, r.level, r.rid)
                patches.append(p)
                descs.append(p.desc())
                scales.append(dt)
        capi.mhd_ghost_fill(ctx, descs, self.copies([r.n for r in batch]), s.cuda_stream)
        capi.mhd_patch_advance(ctx, descs, self.d_one.data_ptr(), s.cuda_stream, dt_scale=scales)
        self.kernel_calls += 2
        ev = torch.cuda.Event()
        ev.record(s)
        return ev, patches

    def ready(self, handle):
        return handle[0].query()

    def finish(self, handle):
        return [p.state for p in handle[1]] if self.keep else [None] * len(handle[1])

    def alone(self, r):
        """The same request run by itself: one patch, one ghost fill, one
        advance, on a fresh context and the current stream; returns its state."""
        torch, capi = self.torch, self.capi
        from .patch import Patch
        tpl, dt = self.templates[(r.n, r.dtype)]
        p = Patch(tpl.state.clone(), tpl.lo, tpl.n, tpl.g, tpl.dx, r.level, r.rid)
        ctx = capi.mhd_ctx_create(**self._solver)
        try:
            sid = torch.cuda.current_stream().cuda_stream
            capi.mhd_ghost_fill(ctx, [p.desc()], self.copies([r.n]), sid)
            capi.mhd_patch_advance(ctx, [p.desc()], self.d_one.data_ptr(), sid, dt_scale=[dt])
            torch.cuda.current_stream().synchronize()
        finally:
            capi.mhd_ctx_destroy(ctx)
        return p.state


def make_templates(sizes, dtypes=("f32", "f64"), g=4, solver=None, device="cuda", seed=4242):
    """One seeded blast-wave patch per (cube edge, precision) on the device,
    ghost-filled, with the CFL dt of its FP64 state (reduced on the GPU) as the
    request dt.  Returns {(n, dtype): (Patch, dt)}."""
    import torch
    import synth
    from . import capi
    from .patch import Patch, periodic_copies
    out = {}
    ctx = capi.mhd_ctx_create(**(solver or {}))
    try:
        d = torch.zeros(1, dtype=torch.float64, device=device)
        for n in sorted(set(int(v) for v in sizes)):
            pr = synth.blast(n, g=g, seed=seed + n)
            p64 = Patch.from_array(pr.state, (0, 0, 0), pr.n, g, pr.dx, dtype="f64", device=device)
            capi.mhd_ghost_fill(ctx, [p64.desc()], periodic_copies(p64.n, g))
            capi.mhd_cfl_dt(ctx, [p64.desc()], d.data_ptr())
            dt = float(d.item())
            for dtype in dtypes:
                p = p64 if dtype == "f64" else Patch.from_array(pr.state, (0, 0, 0), pr.n, g, pr.dx,
                                                                  dtype=dtype, device=device)
                if dtype != "f64":
                    capi.mhd_ghost_fill(ctx, [p.desc()], periodic_copies(p.n, g))
                out[(n, dtype)] = (p, dt)
        torch.cuda.synchronize()
    finally:
        capi.mhd_ctx_destroy(ctx)
    return out


def latency_stats(reqs):
    """p50/p99/mean latency (arrival to completion) overall and per size
    bucket [16, 32), [32, 64), [64, 128]; throughput over the whole run."""
    ok = [r for r in reqs if not r.error]
    lat = np.array([r.done - r.arrival for r in ok])
    span = max(r.done for r in ok) - min(r.arrival for r in ok)
    out = {"count": len(ok), "rejected": len(reqs) - len(ok),
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "span_s": span,
           "cell_updates_per_s": sum(r.cells for r in ok) / span, "requests_per_s": len(ok) / span}
    buckets = {}
    for r in ok:
        lo = 16 * 2 ** min(int(math.log2(r.n / 16)), 2)
        key = "%d-%d" % (lo, min(2 * lo, 128))
        buckets.setdefault(key, []).append(r.done - r.arrival)
    out["by_size"] = {k: {"n": len(v), "p50_ms": float(np.percentile(v, 50) * 1e3),
                          "p99_ms": float(np.percentile(v, 99) * 1e3)}
                      for k, v in sorted(buckets.items(), key=lambda kv: int(kv[0].split("-")[0]))}
    by_lev = {}
    for r in ok:
        by_lev.setdefault(r.level, []).append(r.done - r.arrival)
    out["p50_ms_by_level"] = {int(k): float(np.percentile(v, 50) * 1e3) for k, v in sorted(by_lev.items())}
    return out
