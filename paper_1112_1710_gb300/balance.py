"""Global load balancing across levels (Sec. 5): the desired distribution of
newly created level-l work over P workers, given what every worker still has
to do on the coarser levels, and the partition of the new child work over
those desired shares.

Notation (Sec. 5, table of variables): g[l'][p] work assigned to worker p on
level l', w[l'][p] the part of it already done, s[l'] the remaining steps of
level l' within the coarse step, c[p] the new level-l work created by worker
p's parents; G = sum_p c[p], gbar = G / P.

  eta_{l-1}^p = sum_{l' < l} (s_l' g_l'^p - w_l'^p)      predicted remaining work
  d_l^p = gbar_l - (eta_{l-1}^p - mean_p eta_{l-1}) / s_l     desired share

so that, if every worker receives its desired share, the predicted remaining
work including level l is equal on every worker.  The partition delta[p][p']
lays the child work of workers 0..P-1 end to end and cuts it at the
cumulative desired shares of the receiving workers (Sec. 5, partition
figure): sum_p' delta[p][p'] = c[p] and sum_p delta[p][p'] = d[p'].

On one GPU the workers are the serving loop's slots (streams); the same
equations size each slot's next batch so that the slots' predicted remaining
work evens out (serve.Scheduler, policy "balanced").
"""
from __future__ import annotations

import numpy as np


def eta(g, w, s, upto):
    """Predicted remaining work per worker over levels 0..upto-1:
    sum_l' (s[l'] g[l'][p] - w[l'][p])."""
    P = len(g[0]) if g else 0
    out = np.zeros(P)
    for lp in range(upto):
        out += s[lp] * np.asarray(g[lp], dtype=float) - np.asarray(w[lp], dtype=float)
    return out


def desired_distribution(gbar, g, w, s, level):
    """d_level^p = gbar - (eta_{level-1}^p - mean(eta_{level-1})) / s[level]
    (the general form of the distribution equation, Sec. 5)."""
    e = eta(g, w, s, level)
    return gbar - (e - e.mean()) / s[level]


def desired_distribution_levels(gbar, g, w, s, level):
    """The same distribution written level by level before grouping the
    averages: gbar - sum_{l'<level} (s_l' eps_l'^p - omega_l'^p) / s_level, with
    eps = g - mean(g) and omega = w - mean(w) (Sec. 5)."""
    P = len(g[0])
    acc = np.zeros(P)
    for lp in range(level):
        gl = np.asarray(g[lp], dtype=float)
        wl = np.asarray(w[lp], dtype=float)
        acc += s[lp] * (gl - gl.mean()) - (wl - wl.mean())
    return gbar - acc / s[level]


def partition(c, d):
    """delta[p][p']: the new child work c[p] of each worker laid end to end in
    worker order and cut at the cumulative desired shares d[p'] of the
    receiving workers.  Requires sum(c) == sum(d) (up to rounding) and
    non-negative shares."""
    c = np.asarray(c, dtype=float)
    d = np.asarray(d, dtype=float)
    if np.any(c < 0) or np.any(d < 0):
        raise ValueError("child work and desired shares must be non-negative")
    if not np.isclose(c.sum(), d.sum(), rtol=1e-12, atol=1e-9):
        raise ValueError("child work %g and desired shares %g differ" % (c.sum(), d.sum()))
    cs = np.concatenate([[0.0], np.cumsum(c)])
    ds = np.concatenate([[0.0], np.cumsum(d)])
    ds[-1] = cs[-1]
    delta = np.zeros((len(c), len(d)))
    for p in range(len(c)):
        for q in range(len(d)):
            lo, hi = max(cs[p], ds[q]), min(cs[p + 1], ds[q + 1])
            if hi > lo:
                delta[p, q] = hi - lo
    return delta


def assign_items(sizes, shares):
    """Hands discrete items (grids, in their given order) to receivers with the
    allocations `shares` (sum equal to sum(sizes)): each item is laid on the
    same line as the cumulative shares and goes to the receiver that covers
    the largest part of it (the rounding of Sec. 5, grid assignments).
    Returns the receiver index of every item."""
    sizes = np.asarray(sizes, dtype=float)
    edges = np.concatenate([[0.0], np.cumsum(np.asarray(shares, dtype=float))])
    out = []
    a = 0.0
    for sz in sizes:
        b = a + sz
        cover = [max(0.0, min(b, edges[q + 1]) - max(a, edges[q])) for q in range(len(edges) - 1)]
        out.append(int(np.argmax(cover)))
        a = b
    return out
