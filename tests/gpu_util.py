"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np

import synth


def to_patch(arr, n, g, dx, dtype="f64", lo=(0, 0, 0), level=0, pid=0):
    from paper_1112_1710_gb300.patch import Patch
    return Patch.from_array(arr, lo, n, g, dx, dtype=dtype, level=level, patch_id=pid)


def rel_linf(a, b, n, g):
    """Per-variable max |a - b| / max |b| over the interior (cells and their faces)."""
    nx, ny, nz = n
    out = []
    for q in range(8):
        ext = [nx, ny, nz]
        if q >= 5:
            ext[q - 5] += 1
        sa = a[q, g:g + ext[2], g:g + ext[1], g:g + ext[0]]
        sb = b[q, g:g + ext[2], g:g + ext[1], g:g + ext[0]]
        den = max(np.abs(sb).max(), 1e-300)
        out.append(float(np.abs(sa.astype(np.float64) - sb).max() / den))
    return np.array(out)


def rel_l1(a, b, n, g):
    nx, ny, nz = n
    out = []
    for q in range(8):
        ext = [nx, ny, nz]
        if q >= 5:
            ext[q - 5] += 1
        sa = a[q, g:g + ext[2], g:g + ext[1], g:g + ext[0]].astype(np.float64)
        sb = b[q, g:g + ext[2], g:g + ext[1], g:g + ext[0]]
        den = max(np.abs(sb).mean(), 1e-300)
        out.append(float(np.abs(sa - sb).mean() / den))
    return np.array(out)


def random_state(n, g, seed, align=8):
    """Positive random cells and random faces over the whole array."""
    rng = np.random.default_rng(seed)
    st = synth.empty_patch(n, g, align=align)
    st[0] = rng.uniform(0.5, 2.0, st.shape[1:])
    st[1:4] = rng.uniform(-0.5, 0.5, (3,) + st.shape[1:])
    st[5:8] = rng.uniform(-0.7, 0.7, (3,) + st.shape[1:])
    st[4] = 3.0 + rng.uniform(0.0, 1.0, st.shape[1:])
    return st
