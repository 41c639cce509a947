"""Static AMR hierarchy on the GPU: metadata (ghost copies, prolongation and
restriction items, FP64 flux registers and their deposits) and the subcycled
coarse step of the paper's life cycle (Sec. 2.2) with extended ghost zones
(Sec. 2.3), refinement ratio 2.  Every level operation is one batched call of
``libmhdgpu.so`` over all patches of a level.

One coarse step (AMR(0) of Sec. 2.2):
  dt_0 = min over levels of 2^l * (CFL dt of level l)      (device scalar)
  fill level 0 (periodic images, same-level copies);  step(0, 0)
step(l, k):
  P: prolong level l (pre-advance) into the ghost zones of level l+1, then
     same-level copies on level l+1
  A: advance level l (update box = interior grown by k, dt_l = dt_0 / 2^l),
     capturing dt*F and dt*E on coarse-fine faces and edges (FP64)
  step(l+1, 2); S: same-level copies on l+1; step(l+1, 0)
  reflux level l from the registers; R: restrict l+1 onto l

Level concurrency (Sec. 4, threaded multilevel advance; optional): once P has given
level l+1 its ghost data, nothing in the level l+1 substeps reads level l,
and the advance A of level l touches only level l and its own flux
registers.  With ``concurrent`` set, A of every level that has children
runs on a stream of its own (with a context of its own, so scratch arenas do
not collide) while the finer substeps proceed on the main stream; the main
stream waits for it before refluxing.  The paper gives the finer levels
priority; here the main stream, which carries all finer work, should be the
caller's high-priority stream.
"""
from __future__ import annotations

import ctypes as C
import itertools

import numpy as np
import torch

from . import capi
from .patch import Patch


def _isect(alo, ahi, blo, bhi):
    """Vectorised box intersection: alo/ahi (M, 3) with one box (3,)."""
    lo = np.maximum(alo, blo)
    hi = np.minimum(ahi, bhi)
    ok = np.all(lo <= hi, axis=1)
    return lo, hi, ok


def _vol(lo, hi):
    return (int(hi[0]) - int(lo[0]) + 1) * (int(hi[1]) - int(lo[1]) + 1) * (int(hi[2]) - int(lo[2]) + 1)


def _rows_array(ctype, blocks, width):
    """One ctypes array of `ctype` (int32 fields only, `width` of them) from
    blocks of int rows laid out like its fields; [] when there is no row."""
    blocks = [b for b in blocks if len(b)]
    if not blocks:
        return []
    a = np.ascontiguousarray(np.concatenate(blocks).astype(np.int32))
    assert a.shape[1] == width and a.itemsize * width == C.sizeof(ctype)
    return (ctype * len(a)).from_buffer_copy(a)


# numpy layouts of mhd_capture and mhd_deposit (include/mhd_gpu.h), for
# filling the ctypes arrays of long lists in one copy
_CAP_DT = np.dtype([("patch", "<i4"), ("kind", "<i4"), ("axis", "<i4"), ("mode", "<i4"), ("lo", "<i4", 3),
                    ("hi", "<i4", 3), ("dst", "<u8")])
_DEP_DT = np.dtype([("coarse", "<i4"), ("kind", "<i4"), ("axis", "<i4"), ("mode", "<i4"), ("lo", "<i4", 3),
                    ("hi", "<i4", 3), ("flo", "<i4", 3), ("fhi", "<i4", 3), ("fine", "<u8"), ("creg", "<u8")])


class Hierarchy:
    def __init__(self, boxes, n0, states, dx0, g=4, dtype="f32", ctx=None, stream=None, device="cuda",
                 tree=None, concurrent=None, floors=False):
        """boxes[l] = [(lo, hi)]; states[l][i] = float64 numpy array (synth layout).

        tree: build the metadata from the device AMR tree (neighbour
        inheritance, Sec. 3.1; the default on a GPU; a tree.DeviceTree of the
        same boxes may be passed) instead of testing every pair of patches;
        both give the same lists in the same order.
        concurrent: advance each level that has children on a stream of its
        own alongside the finer substeps (off by default: on one GB300 the
        finer levels' launches already fill the GPU, and the measured coarse
        step is the same within 1%, for a scratch arena per level).
        floors: the context was created with floors (mhd_params.p_floor /
        rho_floor); they are then applied again to a level's interiors after
        its refluxing and restriction, which change cells outside any
        advance (reading R33)."""
        self.floors = bool(floors)
        self.n0, self.g, self.dtype = n0, g, dtype
        self.dx0 = tuple(dx0)
        self.device = torch.device(device)
        self.gpu = self.device.type == "cuda"  # on the CPU only the metadata is built (tests)
        self.ctx = ctx if (ctx is not None or not self.gpu) else capi.mhd_ctx_create()
        self.own_ctx = ctx is None and self.gpu
        self.stream = (stream or torch.cuda.current_stream(self.device)) if self.gpu else None
        self.levels = []
        for l, bl in enumerate(boxes):
            dx = tuple(v / 2 ** l for v in dx0)
            pats = []
            for i, (lo, hi) in enumerate(bl):
                n = tuple(hi[d] - lo[d] + 1 for d in range(3))
                pats.append(Patch.from_array(states[l][i], lo, n, g, dx, dtype=dtype, device=self.device,
                                             level=l, patch_id=i))
            self.levels.append(pats)
        self.descs = [[p.desc() for p in pats] for pats in self.levels] if self.gpu else None
        self.lo = [np.array([p.lo for p in pats], dtype=np.int64) for pats in self.levels]
        self.hi = [np.array([p.hi for p in pats], dtype=np.int64) for pats in self.levels]
        self.d_dt = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.concurrent = bool(concurrent) and self.gpu and len(boxes) > 1
        self.side = []  # (context, stream) per level with children
        if self.concurrent:
            for _ in range(len(boxes) - 1):
                self.side.append((capi.mhd_ctx_clone(self.ctx), torch.cuda.Stream(device=self.device)))
        self.tree = None
        if tree is not None and not isinstance(tree, bool):
            self.tree = tree
        elif tree if tree is not None else self.gpu:
            from .tree import DeviceTree
            self.tree = DeviceTree(boxes, n0, g + 1, device=self.device)
        self._build()

    @property
    def sp(self) -> int:
        return self.stream.cuda_stream

    @property
    def nlev(self) -> int:
        return len(self.levels)

    # ------------------------------------------------------------------ metadata
    def _copies(self, l):
        n = self.n0 * 2 ** l
        g = self.g
        lo, hi = self.lo[l], self.hi[l]
        if self.tree is not None:
            return self._copies_tree(l)
        near = np.any(lo <= g + 1, axis=1) | np.any(hi >= n - g - 2, axis=1)
        shifts = [(0, 0, 0)]
        if near.any():
            shifts = [s for s in itertools.product((-n, 0, n), repeat=3)]
        rows = []   # src, dst, box lo, box hi, offset
        for di in range(len(lo)):
            elo = lo[di] - g - 1
            ehi = hi[di] + g + 1
            for sh in shifts:
                sh = np.array(sh)
                blo, bhi, ok = _isect(lo + sh, hi + sh, elo, ehi)
                if not sh.any():
                    ok[di] = False
                si = np.nonzero(ok)[0]
                if len(si):
                    rows.append(np.column_stack([si, np.full(len(si), di), blo[si], bhi[si],
                                                 np.repeat(-sh[None], len(si), axis=0)]))
        return _rows_array(capi.mhd_copy, rows, 11)

    def _copies_tree(self, l):
        """The same copies from the tree's interactions of each destination,
        already in (shift, source) order."""
        n = self.n0 * 2 ** l
        g = self.g
        lo, hi = self.lo[l], self.hi[l]
        rows = []   # src, dst, box lo, box hi, offset
        for di in range(len(lo)):
            idx, s = self.tree.interactions(l, di)
            keep = (idx != di) | np.any(s != 0, axis=1)
            idx, sh = idx[keep], s[keep].astype(np.int64) * n
            blo = np.maximum(lo[idx] + sh, lo[di] - g - 1)
            bhi = np.minimum(hi[idx] + sh, hi[di] + g + 1)
            if len(idx):
                rows.append(np.column_stack([idx, np.full(len(idx), di), blo, bhi, -sh]))
        return _rows_array(capi.mhd_copy, rows, 11)

    def _coarse(self, l, fi):
        """Level-l patches that can touch fine patch fi of level l+1, ascending:
        all of them, or the tree's candidates."""
        if self.tree is None:
            return np.arange(len(self.lo[l]))
        return self.tree.coarse_candidates(l + 1, fi)

    def _prolongs(self, l):
        g = self.g
        clo, chi = self.lo[l], self.hi[l]
        out = []
        for fi, (flo, fhi) in enumerate(zip(self.lo[l + 1], self.hi[l + 1])):
            cand = self._coarse(l, fi)
            clo, chi = self.lo[l][cand], self.hi[l][cand]
            el, eh = flo - g, fhi + g
            slabs = [((el[0], el[1], el[2]), (eh[0], eh[1], flo[2] - 1)),
                     ((el[0], el[1], fhi[2] + 1), (eh[0], eh[1], eh[2])),
                     ((el[0], el[1], flo[2]), (eh[0], flo[1] - 1, fhi[2])),
                     ((el[0], fhi[1] + 1, flo[2]), (eh[0], eh[1], fhi[2])),
                     ((el[0], flo[1], flo[2]), (flo[0] - 1, fhi[1], fhi[2])),
                     ((fhi[0] + 1, flo[1], flo[2]), (eh[0], fhi[1], fhi[2]))]
            for (slo, shi) in slabs:
                cl = np.array(slo) // 2
                ch = np.array(shi) // 2
                blo, bhi, ok = _isect(clo, chi, cl, ch)
                k = np.nonzero(ok)[0]
                if len(k):
                    out.append(np.column_stack([np.asarray(cand)[k], np.full(len(k), fi), blo[k], bhi[k]]))
        return _rows_array(capi.mhd_prolong_item, out, 8)

    def _restricts(self, l):
        out = []
        for fi, (flo, fhi) in enumerate(zip(self.lo[l + 1], self.hi[l + 1])):
            cand = self._coarse(l, fi)
            clo, chi = self.lo[l][cand], self.hi[l][cand]
            cl, ch = flo // 2, (fhi + 1) // 2 - 1
            blo, bhi, ok = _isect(clo - 1, chi + 1, cl, ch)
            k = np.nonzero(ok)[0]
            if len(k):
                out.append(np.column_stack([np.full(len(k), fi), np.asarray(cand)[k], blo[k], bhi[k]]))
        return _rows_array(capi.mhd_restrict_item, out, 8)

    def _build(self):
        L = self.nlev
        self.copy_lists = [self._copies(l) for l in range(L)]
        self.prolong_lists = [self._prolongs(l) for l in range(L - 1)]
        self.restrict_lists = [self._restricts(l) for l in range(L - 1)]
        # flux registers: (size, owner) records, then one FP64 buffer
        regs = []          # (values,)
        fine_caps = {l: [] for l in range(L)}     # (patch, kind, axis, lo, hi, reg)
        coarse_caps = {l: [] for l in range(L)}
        deposits = {l: [] for l in range(L)}      # (coarse, kind, axis, lo, hi, fine reg, fine lo, fine hi, coarse reg)

        def new_reg(nvals):
            regs.append(nvals)
            return len(regs) - 1

        eye = np.eye(3, dtype=np.int64)
        for l in range(1, L):
            for fi, (flo, fhi) in enumerate(zip(self.lo[l], self.hi[l])):
                cand = self._coarse(l - 1, fi)
                clo_all, chi_all = self.lo[l - 1][cand], self.hi[l - 1][cand]
                # the 6 sides (d, side) and their 12 edge axes, intersected
                # with every candidate at once; the lists are then filled
                # side by side in the order of the registers
                sides = [(d, side) for d in range(3) for side in (0, 1)]
                fidx = np.array([int(flo[d]) if side == 0 else int(fhi[d]) + 1 for d, side in sides], np.int64)
                cidx = fidx // 2
                outc = np.array([c - 1 if side == 0 else c for c, (d, side) in zip(cidx, sides)], np.int64)
                dd = np.array([d for d, _ in sides])
                c0, c1 = flo // 2, (fhi + 1) // 2 - 1
                CL = np.repeat(c0[None], 6, axis=0)
                CH = np.repeat(c1[None], 6, axis=0)
                CL[np.arange(6), dd] = cidx
                CH[np.arange(6), dd] = cidx
                # faces: the coarse patches holding the cells outside the side
                # (coarse index outc along d), cut to the side's coarse faces
                FLO = np.maximum(clo_all[None], CL[:, None])
                FHI = np.minimum(chi_all[None], CH[:, None])
                FLO[np.arange(6), :, dd] = cidx[:, None]
                FHI[np.arange(6), :, dd] = cidx[:, None]
                FOK = ((clo_all[:, dd].T <= outc[:, None]) & (outc[:, None] <= chi_all[:, dd].T) &
                       np.all(FLO <= FHI, axis=2))
                # edges along a != d in the side plane
                edges = [(q, a) for q in range(6) for a in range(3) if a != sides[q][0]]
                ea = np.array([a for _, a in edges])
                eq = np.array([q for q, _ in edges])
                ett = 3 - ea - dd[eq]
                ECL = CL[eq].copy()
                ECH = CH[eq].copy()
                ECH[np.arange(12), ett] = (fhi[ett] + 1) // 2
                top = chi_all[None] + 1 - eye[ea][:, None, :]
                ELO = np.maximum(clo_all[None], ECL[:, None])
                EHI = np.minimum(top, ECH[:, None])
                EOK = np.all(ELO <= EHI, axis=2)
                e = 0
                for q, (d, side) in enumerate(sides):
                    # fine faces of the side
                    rlo, rhi = flo.copy(), fhi.copy()
                    rlo[d] = rhi[d] = fidx[q]
                    rf = new_reg(5 * _vol(rlo, rhi))
                    fine_caps[l].append((fi, 0, d, rlo, rhi, rf))
                    for k in np.nonzero(FOK[q])[0]:
                        ci = int(cand[k])
                        blo, bhi = FLO[q, k].copy(), FHI[q, k].copy()
                        rc = new_reg(5 * _vol(blo, bhi))
                        coarse_caps[l - 1].append((ci, 0, d, blo, bhi, rc))
                        deposits[l - 1].append((ci, 0, d, blo, bhi, rf, rlo, rhi, rc))
                    for a in range(3):
                        if a == d:
                            continue
                        tt = 3 - a - d
                        elo, ehi = flo.copy(), fhi.copy()
                        elo[d] = ehi[d] = fidx[q]
                        ehi[tt] = fhi[tt] + 1
                        re = new_reg(_vol(elo, ehi))
                        fine_caps[l].append((fi, 1, a, elo, ehi, re))
                        for k in np.nonzero(EOK[e])[0]:
                            ci = int(cand[k])
                            blo, bhi = ELO[e, k].copy(), EHI[e, k].copy()
                            rc = new_reg(_vol(blo, bhi))
                            coarse_caps[l - 1].append((ci, 1, a, blo, bhi, rc))
                            deposits[l - 1].append((ci, 1, a, blo, bhi, re, elo, ehi, rc))
                        e += 1
        offs = np.concatenate([[0], np.cumsum(regs)]).astype(np.int64)
        self.regbuf = torch.zeros(max(1, int(offs[-1])), dtype=torch.float64, device=self.device)
        base = self.regbuf.data_ptr()

        def cap_array(items, mode_fine):
            # the ctypes array is filled from a numpy record array of the same layout
            rec = np.zeros(max(1, len(items)), dtype=_CAP_DT)
            if items:
                rec["patch"] = [it[0] for it in items]
                rec["kind"] = [it[1] for it in items]
                rec["axis"] = [it[2] for it in items]
                rec["mode"] = [mode_fine if it[6] else 0 for it in items]
                rec["lo"] = np.array([it[3] for it in items], dtype=np.int64)
                rec["hi"] = np.array([it[4] for it in items], dtype=np.int64)
                rec["dst"] = base + 8 * offs[np.array([it[5] for it in items], dtype=np.int64)]
            return (capi.mhd_capture * len(rec)).from_buffer_copy(rec.tobytes()), len(items)

        self.caps = {}
        for l in range(L):
            items = [c + (True,) for c in fine_caps[l]] + [c + (False,) for c in coarse_caps[l]]
            self.caps[(l, True)] = cap_array(items, 0) if items else None
            self.caps[(l, False)] = cap_array(items, 1) if items else None
        self.deps = {}
        self.corr = {}
        for l in range(L - 1):
            dl = deposits[l]
            arr = (capi.mhd_deposit * max(1, len(dl)))()
            need = sorted({int(x[0]) for x in dl})
            corr = {}
            for ci in need:
                nelem = int(np.prod(self.levels[l][ci].state.shape[1:]))
                corr[ci] = torch.zeros(18 * nelem, dtype=torch.float64, device=self.device)
            if dl:
                rec = np.zeros(len(dl), dtype=_DEP_DT)
                rec["coarse"] = [x[0] for x in dl]
                rec["kind"] = [x[1] for x in dl]
                rec["axis"] = [x[2] for x in dl]
                rec["lo"] = np.array([x[3] for x in dl], dtype=np.int64)
                rec["hi"] = np.array([x[4] for x in dl], dtype=np.int64)
                rec["flo"] = np.array([x[6] for x in dl], dtype=np.int64)
                rec["fhi"] = np.array([x[7] for x in dl], dtype=np.int64)
                rec["fine"] = base + 8 * offs[np.array([x[5] for x in dl], dtype=np.int64)]
                rec["creg"] = base + 8 * offs[np.array([x[8] for x in dl], dtype=np.int64)]
                arr = (capi.mhd_deposit * len(dl)).from_buffer_copy(rec.tobytes())
            self.deps[l] = (arr, len(dl))
            self.corr[l] = [corr[ci].data_ptr() if ci in corr else None for ci in range(len(self.levels[l]))]
            self._corr_keep = getattr(self, "_corr_keep", []) + list(corr.values())
        self.fine_caps, self.coarse_caps, self.deposit_list = fine_caps, coarse_caps, deposits
        # prebuilt ctypes arrays of the static lists
        self._copy_arr = [capi._structs(capi.mhd_copy, cl) for cl in self.copy_lists]
        self._prolong_arr = [capi._structs(capi.mhd_prolong_item, pl) for pl in self.prolong_lists]
        self._restrict_arr = [capi._structs(capi.mhd_restrict_item, rl) for rl in self.restrict_lists]
        if not self.gpu:
            return
        self._desc_arr = [capi._descs(d) for d in self.descs]
        self._all_descs = capi._descs([d for dl in self.descs for d in dl])
        self._all_scale = capi._arr(C.c_double, [2.0 ** l for l, dl in enumerate(self.descs) for _ in dl])
        self._dt_scale = [capi._arr(C.c_double, [0.5 ** l] * len(dl)) for l, dl in enumerate(self.descs)]

    # ------------------------------------------------------------------ operations
    def fill(self, l):
        arr, n = self._desc_arr[l]
        ca, nc = self._copy_arr[l]
        if nc:
            capi._check(self.ctx, capi.load().mhd_ghost_fill(self.ctx, arr, n, ca, nc, self.sp))

    def prolong(self, l):
        capi.mhd_prolong(self.ctx, self.descs[l], self.descs[l + 1], self._prolong_arr[l], self.sp)

    def restrict(self, l):
        capi.mhd_restrict(self.ctx, self.descs[l + 1], self.descs[l], self._restrict_arr[l], self.sp)

    def advance(self, l, k, first, ctx=None, stream=None):
        if not self.batched:
            return self._advance_per_patch(l, k, first)
        ctx = ctx or self.ctx
        arr, n = self._desc_arr[l]
        grow = capi._arr(C.c_int32, [k] * n)
        caps = self.caps[(l, first)]
        ca, nca = caps if caps is not None else (None, 0)
        capi._check(ctx, capi.load().mhd_patch_advance(ctx, arr, n, grow, self.d_dt.data_ptr(), self._dt_scale[l],
                                                       ca, nca, stream.cuda_stream if stream else self.sp))

    batched = True

    def _advance_per_patch(self, l, k, first):
        """The plain path: one advance call (six kernels) per patch."""
        if not hasattr(self, "_pp"):
            self._pp = {}
        key = (l, first)
        if key not in self._pp:
            caps = self.caps[(l, first)]
            per = [[] for _ in self.descs[l]]
            if caps is not None:
                arr, n = caps
                for t in range(n):
                    c = capi.mhd_capture()
                    C.memmove(C.byref(c), C.byref(arr[t]), C.sizeof(c))
                    p = c.patch
                    c.patch = 0
                    per[p].append(c)
            self._pp[key] = [(capi._descs([d]), capi._structs(capi.mhd_capture, cl)) for d, cl in
                             zip(self.descs[l], per)]
        grow = capi._arr(C.c_int32, [k])
        scale = capi._arr(C.c_double, [0.5 ** l])
        for (arr, n), (ca, nca) in self._pp[key]:
            capi._check(self.ctx, capi.load().mhd_patch_advance(self.ctx, arr, n, grow, self.d_dt.data_ptr(),
                                                                scale, ca if nca else None, nca, self.sp))

    def reflux(self, l):
        capi.mhd_reflux(self.ctx, self.descs[l], self.corr[l], self.deps[l], self.sp)

    def cfl(self):
        arr, n = self._all_descs
        capi._check(self.ctx, capi.load().mhd_cfl_dt(self.ctx, arr, n, self._all_scale, self.d_dt.data_ptr(),
                                                     self.sp))

    def step(self, l, k, first=True):
        last = l + 1 >= self.nlev
        if not last:
            self.prolong(l)
            self.fill(l + 1)
        join = None
        if not last and self.concurrent and self.batched:
            ctx, side = self.side[l]
            fork = torch.cuda.Event()
            fork.record(self.stream)
            side.wait_event(fork)
            self.advance(l, k, first, ctx=ctx, stream=side)
            join = torch.cuda.Event()
            join.record(side)
        else:
            self.advance(l, k, first)
        if not last:
            self.step(l + 1, 2, True)
            self.fill(l + 1)
            self.step(l + 1, 0, False)
            if join is not None:
                self.stream.wait_event(join)
            self.reflux(l)
            self.restrict(l)
            if self.floors:
                self.floor(l)

    def floor(self, l):
        capi.mhd_floor(self.ctx, self.descs[l], self.sp)

    def launch_count(self) -> int:
        """Kernel launches of all the hierarchy's contexts so far."""
        return sum(capi.mhd_launch_count(c) for c in [self.ctx] + [c for c, _ in self.side])

    def device_status(self) -> int:
        """The first non-zero device status of the hierarchy's contexts (0: clean)."""
        for c in [self.ctx] + [c for c, _ in self.side]:
            st = capi.mhd_get_device_status(c)
            if st:
                return st
        return 0

    def initialise(self):
        for l in range(self.nlev - 2, -1, -1):
            self.restrict(l)
        self.fill(0)

    def coarse_step(self, dt: float | None = None):
        if dt is None:
            self.cfl()
        else:
            with torch.cuda.stream(self.stream):
                self.d_dt.fill_(float(dt))
        self.fill(0)
        self.step(0, 0)

    def capture_graph(self):
        """Captures one whole coarse step (CFL dt, ghost fills, subcycled
        advances, refluxing, restriction) as a CUDA graph.  dt lives in device
        memory, so the graph stays valid across steps.  One eager step is run
        first so that every descriptor table is already on the device (the
        capture issues no uploads)."""
        self.coarse_step()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self.cfl()
            self.fill(0)
            self.step(0, 0)
        self.graph = g
        return g

    def replay(self):
        # CUDAGraph.replay launches on the current stream
        with torch.cuda.stream(self.stream):
            self.graph.replay()

    def autotune(self, reps: int = 1, dt: float = 1e-7):
        """Lets mhd_autotune_advance choose this hierarchy's advance (staged
        kernels, fused pass or fused kernel, tile shape and z-chunk) for each
        context on the batch it advances: the main context on the finest
        level, and with concurrent levels each level's own slot context on
        that level (without them the main context advances every level and
        is tuned on the finest).  Each batch is timed with its first
        substep's update box (grown by 2 when subcycled), its flux-register
        captures and a small dt; the patch state is unchanged.  Call it after
        a first coarse step (until then the fine levels' ghost zones hold
        whatever the initial states held there) and before any step is
        captured.  Returns the finest level's (choice, chunk, ms); every
        level's is kept in `tuned`."""
        d = torch.full((1,), dt, dtype=torch.float64, device=self.device)

        def tune(ctx, l):
            k = 2 if l > 0 else 0
            return capi.mhd_autotune_advance(ctx, self.descs[l], d.data_ptr(), reps=reps,
                                             grow=[k] * len(self.descs[l]), stream=self.sp,
                                             caps=self.caps[(l, True)])
        self.tuned = {self.nlev - 1: tune(self.ctx, self.nlev - 1)}
        for l, (c, _) in enumerate(self.side):
            self.tuned[l] = tune(c, l)
        return self.tuned[self.nlev - 1]

    def cell_updates_per_coarse_step(self) -> int:
        return sum(p.cells * 2 ** l for l, pats in enumerate(self.levels) for p in pats)

    def regrid(self, theta: float, first: int | None = None, **kw) -> "Hierarchy":
        """The hierarchy with its levels from `first` (default: the finest)
        up replaced by their next iterations (regrid.regrid_levels: each from
        the flags of the new level below on the device, Berger-Rigoutsos
        grids, the data transfer), built with this one's context, stream and
        options; this hierarchy is closed (its kept levels' state tensors
        move to the new one).  The new hierarchy's `regrid_info` holds the
        energy-fallback count (a device tensor) and the old and new patch
        counts of the finest level."""
        from . import regrid as R
        boxes, states, nfall = R.regrid_levels(self, theta, first=first, **kw)
        old = len(self.levels[-1])
        own, self.own_ctx = self.own_ctx, False
        conc = bool(self.side)
        self.close()
        h = Hierarchy(boxes, self.n0, states, self.dx0, g=self.g, dtype=self.dtype, ctx=self.ctx,
                      stream=self.stream, device=self.device, concurrent=conc, floors=self.floors)
        h.own_ctx = own
        h.regrid_info = {"fallbacks": nfall, "old_patches": old,
                         "new_patches": len(boxes[-1]) if len(boxes) == self.nlev else 0}
        return h

    def close(self):
        for c, _ in self.side:
            capi.mhd_ctx_destroy(c)
        self.side = []
        if self.own_ctx and self.ctx:
            capi.mhd_ctx_destroy(self.ctx)
            self.ctx = None
