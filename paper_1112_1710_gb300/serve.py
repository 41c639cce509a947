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


# ---------------------------------------------------------------------------
# Serving the level steps of a resident AMR hierarchy.
#
# A hierarchy held on the device (amr.Hierarchy) is advanced by requests: one
# request per operation of a level step of the paper's life cycle (Sec. 2.2;
# extended ghost zones, Sec. 2.3), each a captured CUDA graph of one batched
# launch sequence over all patches of its level:
#   start      CFL dt of every level (device scalar) and the level-0 ghost fill
#   PF(l)      prolongation of level l (pre-advance) into level l+1's ghosts,
#              then level l+1's same-level copies
#   A(l,k)     advance of level l (update box grown by k) with its flux-register
#              captures
#   S(l)       same-level copies of level l between its two substeps
#   RR(l)      refluxing of level l from the registers, restriction of l+1
#              (and the floors on level l, when the hierarchy has them)
# The requests of a coarse step form a dependency graph (a request is issued
# once the requests it reads from are issued; the GPU orders them through
# events).  Among the issuable requests the finer level goes first, as in the
# paper's scheduler (Sec. 4).  The advance of a level that has children runs
# on a slot of its own (stream and library context, so scratch arenas do not
# collide) while the finer levels' requests proceed on the main slot, which
# is created with the higher stream priority.  Every request is bracketed by
# CUDA events, from which its latency (issuable-on-device to done) and the
# per-level p50/p99 follow after the run.
# ---------------------------------------------------------------------------
@dataclass
class LevelRequest:
    tid: int
    kind: str               # "start", "PF", "A", "S", "RR"
    level: int
    k: int = 0
    first: bool = True
    deps: tuple = ()
    step: int = 0           # coarse step
    slot: int = 0


def level_requests(nlev: int, nsteps: int):
    """The requests of `nsteps` coarse steps of an nlev-level hierarchy with
    their dependencies, in the order the recursive step would issue them."""
    out = []

    def add(kind, level, deps, step, k=0, first=True):
        out.append(LevelRequest(len(out), kind, level, k, first, tuple(deps), step))
        return len(out) - 1

    def level_step(l, k, first, deps, step):
        if l + 1 >= nlev:
            return add("A", l, deps, step, k, first)
        pf = add("PF", l, deps, step)
        a = add("A", l, [pf], step, k, first)
        c1 = level_step(l + 1, 2, True, [pf], step)
        s = add("S", l + 1, [c1], step)
        c2 = level_step(l + 1, 0, False, [s], step)
        return add("RR", l, [a, c2], step)

    last = None
    for c in range(nsteps):
        st = add("start", 0, [] if last is None else [last], c)
        last = level_step(0, 0, True, [st], c)
    return out


class AmrLevelServer:
    """Serves the level-step requests of one resident hierarchy (see above).

    budget_bytes: the hierarchy is admitted only if its resident device memory
    (states, flux registers and correction planes, scratch arenas measured
    over a warm-up coarse step) fits; otherwise the constructor raises."""

    def __init__(self, h, budget_bytes=64 << 30):
        import torch
        self.torch = torch
        self.h = h
        dev = h.device
        free0, _ = torch.cuda.mem_get_info(dev)
        h.coarse_step()                      # sizes every arena, uploads every table
        torch.cuda.synchronize(dev)
        free1, _ = torch.cuda.mem_get_info(dev)
        tensors = sum(p.state.numel() * p.state.element_size() for pats in h.levels for p in pats)
        tensors += h.regbuf.numel() * 8 + sum(t.numel() * 8 for t in getattr(h, "_corr_keep", []))
        self.resident_bytes = tensors + max(0, free0 - free1)
        if self.resident_bytes > budget_bytes:
            raise MemoryError("hierarchy needs %.1f GB, budget %.1f GB" % (self.resident_bytes / 2 ** 30,
                                                                           budget_bytes / 2 ** 30))
        # slots: 0 = the main stream and context; 1 + l = the side slot of level l
        self.slots = [(h.ctx, h.stream)] + [(c, s) for c, s in h.side]
        self.graphs = {}
        self._capture()

    def _slot_of(self, r: LevelRequest) -> int:
        if r.kind == "A" and self.h.concurrent and r.level + 1 < self.h.nlev:
            return 1 + r.level
        return 0

    def _body(self, key):
        h = self.h
        kind = key[0]
        if kind == "start":
            h.cfl()
            h.fill(0)
        elif kind == "PF":
            h.prolong(key[1])
            h.fill(key[1] + 1)
        elif kind == "S":
            h.fill(key[1])
        elif kind == "RR":
            h.reflux(key[1])
            h.restrict(key[1])
            if h.floors:
                h.floor(key[1])
        else:
            _, l, k, first, slot = key
            ctx, st = self.slots[slot]
            h.advance(l, k, first, ctx=ctx, stream=st)

    def _key(self, r: LevelRequest):
        if r.kind == "A":
            return ("A", r.level, r.k, r.first, self._slot_of(r))
        return (r.kind, r.level)

    def _capture(self):
        """One CUDA graph per distinct request (kind, level, substep), each
        captured on the stream of the slot that will replay it."""
        torch = self.torch
        from . import capi
        keys = {}
        for r in level_requests(self.h.nlev, 1):
            keys[self._key(r)] = self._slot_of(r)
        for key, slot in keys.items():
            st = self.slots[slot][1]
            n0 = sum(capi.mhd_launch_count(c) for c, _ in self.slots)
            # a request with nothing to launch (a level without same-level
            # neighbours has no copies) keeps no graph
            if not self._launches(key):
                self.graphs[key] = None
                continue
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                self._body(key)
            assert sum(capi.mhd_launch_count(c) for c, _ in self.slots) > n0
            self.graphs[key] = g
        torch.cuda.synchronize(self.h.device)

    def _launches(self, key) -> bool:
        """Whether the request's body enqueues any kernel."""
        h = self.h
        kind = key[0]
        if kind == "S":
            return bool(h._copy_arr[key[1]][1])
        if kind == "PF":
            return bool(h._prolong_arr[key[1]][1]) or bool(h._copy_arr[key[1] + 1][1])
        return True

    def run(self, nsteps: int, timing: bool = True):
        """Serves `nsteps` coarse steps; returns per-request timing records and
        latency statistics (device clock)."""
        torch = self.torch
        reqs = level_requests(self.h.nlev, nsteps)
        for r in reqs:
            r.slot = self._slot_of(r)
        n = len(reqs)
        ndeps = [len(r.deps) for r in reqs]
        users = [[] for _ in range(n)]
        for r in reqs:
            for d in r.deps:
                users[d].append(r.tid)
        ready = []                            # heap: finer level first, then issue order
        for r in reqs:
            if not r.deps:
                heapq.heappush(ready, (-r.level, r.tid))
        ev_end = [None] * n
        ev_start = [None] * n
        base = torch.cuda.Event(enable_timing=True)
        base.record(self.slots[0][1])
        for _, st in self.slots[1:]:
            st.wait_event(base)
        issued = 0
        while ready:
            _, tid = heapq.heappop(ready)
            r = reqs[tid]
            st = self.slots[r.slot][1]
            for d in r.deps:
                if reqs[d].slot != r.slot:
                    st.wait_event(ev_end[d])
            if timing:
                ev_start[tid] = torch.cuda.Event(enable_timing=True)
                ev_start[tid].record(st)
            g = self.graphs[self._key(r)]
            if g is not None:
                with torch.cuda.stream(st):
                    g.replay()
            ev_end[tid] = torch.cuda.Event(enable_timing=timing)
            ev_end[tid].record(st)
            issued += 1
            for u in users[tid]:
                ndeps[u] -= 1
                if ndeps[u] == 0:
                    heapq.heappush(ready, (-reqs[u].level, u))
        if issued != n:
            raise RuntimeError("level-request graph has a cycle")
        main = self.slots[0][1]
        for _, st in self.slots[1:]:
            j = torch.cuda.Event()
            j.record(st)
            main.wait_event(j)
        fin = torch.cuda.Event(enable_timing=True)
        fin.record(main)
        fin.synchronize()
        total_ms = base.elapsed_time(fin)
        out = {"requests": n, "coarse_steps": nsteps, "ms": total_ms}
        if not timing:
            return out
        t0 = [base.elapsed_time(e) for e in ev_start]
        t1 = [base.elapsed_time(e) for e in ev_end]
        lat = []
        per_level = {}
        for r in reqs:
            ready_at = max([t1[d] for d in r.deps], default=0.0)
            ready_at = min(ready_at, t0[r.tid])
            v = t1[r.tid] - ready_at
            lat.append(v)
            per_level.setdefault(r.level, []).append(v)
        lat = np.array(lat)
        out.update({"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                    "max_ms": float(lat.max()),
                    "by_level": {int(l): {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                                          "p99_ms": float(np.percentile(v, 99))}
                                 for l, v in sorted(per_level.items())}})
        return out
