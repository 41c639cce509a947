"""AMR tree on the device (Sec. 3.1): the parents of every patch and the
same-level interactions of every level, built level by level by inheritance
in ``libmhdgpu.so`` (``mhd_tree_parents``, ``mhd_tree_inherit``).

Level 0 inherits from a virtual root that is the parent of every level-0
patch and interacts with itself under all 27 periodic shifts, so its pairs
are the brute-force ones; level l+1 inherits from level l: the interactions
of a patch's children are children of the patch's interactions (Sec. 3.1).
An interaction (c', s) of patch c means that box(c') shifted by s (in
{-1, 0, 1}^3 periodic domain lengths) meets box(c) grown by r cells; with
r = g + 1 the interactions hold every same-level ghost copy, and the coarse
candidates of a fine patch (its parents and their unshifted interactions)
hold every coarse patch its prolongation, restriction and flux registers
touch.  The kernels emit candidates with repeats; the host side here sorts
them, drops repeats and lays them out as CSR lists.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def _shift_index(s):
    """Rank of a shift (sx, sy, sz) in itertools.product((-1, 0, 1), repeat=3)
    order (x slowest)."""
    return (s[:, 0] + 1) * 9 + (s[:, 1] + 1) * 3 + (s[:, 2] + 1)


def _off(counts, device):
    off = torch.zeros(counts.numel() + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(counts.to(torch.int64), 0)
    return off


class DeviceTree:
    """Parents and interactions of a static hierarchy, computed on the GPU.

    boxes[l] = [(lo, hi)] (inclusive, level-l cells; level l has n0 2^l cells
    per side, periodic).  After construction (host numpy, in canonical order):
      inter[l] = (off, idx, shift): interactions of each level-l patch sorted
                 by (shift rank, idx), (c, 0) itself included;
      parents[l] = (off, idx) for l >= 1: parents of each level-l patch on
                 level l-1, ascending.
    """

    def __init__(self, boxes, n0, r, device="cuda"):
        self.n0, self.r = n0, r
        self.device = torch.device(device)
        dev = self.device
        self.inter, self.parents = [], [None]
        lo_d = [torch.tensor(np.array([b[0] for b in bl], dtype=np.int32).reshape(-1, 3), device=dev) for bl in boxes]
        hi_d = [torch.tensor(np.array([b[1] for b in bl], dtype=np.int32).reshape(-1, 3), device=dev) for bl in boxes]
        i32, i64, i8 = torch.int32, torch.int64, torch.int8
        for l, bl in enumerate(boxes):
            n = len(bl)
            ndom = n0 * 2 ** l
            if l == 0:
                # virtual root: parent of every level-0 patch, interacting with
                # itself under all 27 shifts
                par_off = torch.arange(n + 1, dtype=i64, device=dev)
                par = torch.zeros(n, dtype=i32, device=dev)
                sh = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], np.int8)
                int_off = torch.tensor([0, 27], dtype=i64, device=dev)
                inter = torch.zeros(27, dtype=i32, device=dev)
                ish = torch.tensor(sh.reshape(-1), device=dev)
                kid_off = torch.tensor([0, n], dtype=i64, device=dev)
                kid = torch.arange(n, dtype=i32, device=dev)
            else:
                nc = len(boxes[l - 1])
                cnt = torch.zeros(n, dtype=i32, device=dev)
                self._parents(lo_d[l], hi_d[l], lo_d[l - 1], hi_d[l - 1], None, cnt, None)
                par_off = _off(cnt, dev)
                par = torch.empty(max(1, int(par_off[-1])), dtype=i32, device=dev)
                self._parents(lo_d[l], hi_d[l], lo_d[l - 1], hi_d[l - 1], par_off, None, par)
                # children of each coarse patch: the transpose of the parents
                child = torch.repeat_interleave(torch.arange(n, dtype=i64, device=dev), par_off[1:] - par_off[:-1])
                pk = par[: child.numel()].to(i64)
                order = torch.argsort(pk * n + child)
                kid = child[order].to(i32)
                kid_off = _off(torch.bincount(pk, minlength=nc), dev)
                int_off, inter, ish = self._int_dev
                self.parents.append((par_off.cpu().numpy(), par[: child.numel()].cpu().numpy()))
            cnt = torch.zeros(n, dtype=i32, device=dev)
            args = (lo_d[l], hi_d[l], ndom, r, par_off, par, int_off, inter, ish, kid_off, kid)
            self._inherit(*args, None, cnt, None, None)
            off = _off(cnt, dev)
            m = int(off[-1])
            out = torch.empty(max(1, m), dtype=i32, device=dev)
            osh = torch.empty(max(1, 3 * m), dtype=i8, device=dev)
            self._inherit(*args, off, None, out, osh)
            # canonical order per patch: (shift rank, partner), repeats dropped
            c = torch.repeat_interleave(torch.arange(n, dtype=i64, device=dev), off[1:] - off[:-1])
            s3 = osh[: 3 * m].view(-1, 3).to(i64)
            key = (c * 27 + _shift_index(s3)) * n + out[:m].to(i64)
            key = torch.unique(key)  # sorted
            cc = key // (27 * n)
            rank = (key // n) % 27
            idx = (key % n).to(i32)
            s = torch.stack([rank // 9 - 1, (rank // 3) % 3 - 1, rank % 3 - 1], 1).to(i8)
            ioff = _off(torch.bincount(cc, minlength=n), dev)
            self._int_dev = (ioff, idx.contiguous(), s.reshape(-1).contiguous())
            self.inter.append((ioff.cpu().numpy(), idx.cpu().numpy(), s.cpu().numpy()))

    @staticmethod
    def _ptr(t):
        return t.data_ptr() if t is not None else None

    def _parents(self, flo, fhi, clo, chi, off, count, out):
        """One pass of mhd_tree_parents on the current stream."""
        p = self._ptr
        r = capi.load().mhd_tree_parents(p(flo), p(fhi), flo.shape[0], p(clo), p(chi), clo.shape[0], p(off),
                                         p(count), p(out), torch.cuda.current_stream(self.device).cuda_stream)
        if r != capi.MHD_OK:
            raise capi.MHDError(r, "mhd_tree_parents")

    def _inherit(self, lo, hi, ndom, r, par_off, par, int_off, inter, ish, kid_off, kid, off, count, out, osh):
        """One pass of mhd_tree_inherit on the current stream."""
        p = self._ptr
        st = capi.load().mhd_tree_inherit(p(lo), p(hi), lo.shape[0], ndom, r, p(par_off), p(par), p(int_off),
                                          p(inter), p(ish), p(kid_off), p(kid), p(off), p(count), p(out), p(osh),
                                          torch.cuda.current_stream(self.device).cuda_stream)
        if st != capi.MHD_OK:
            raise capi.MHDError(st, "mhd_tree_inherit")

    def interactions(self, l, i):
        """(partner indices, shifts (k, 3)) of patch i of level l, sorted by
        (shift rank, partner)."""
        off, idx, s = self.inter[l]
        return idx[off[i]:off[i + 1]], s[off[i]:off[i + 1]]

    def coarse_candidates(self, l, f):
        """Ascending level-(l-1) patches near patch f of level l: its parents
        and their unshifted interactions."""
        po, pi = self.parents[l]
        ps = pi[po[f]:po[f + 1]]
        off, idx, s = self.inter[l - 1]
        out = [ps]
        for p in ps:
            a, b = off[p], off[p + 1]
            z = ~np.any(s[a:b] != 0, axis=1)
            out.append(idx[a:b][z])
        return np.unique(np.concatenate(out)) if out else np.zeros(0, np.int32)
