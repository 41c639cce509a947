"""The global load-balance distribution (Sec. 5, Appendix B) pinned to the
paper's worked example and to the identities it derives -- no GPU."""
import numpy as np
import pytest

from paper_1112_1710_gb300.balance import (assign_items, desired_distribution, desired_distribution_levels, eta,
                                           partition)

# Sec. 5 worked example: three processors, G_0 = 72 level-0 cells distributed
# [32, 20, 20], new level-1 child work c_1 = [32, 8, 8] (G_1 = 48)
G0 = [32, 20, 20]
C1 = [32, 8, 8]
GBAR1 = sum(C1) / 3


def test_worked_example_independent_and_full_compensation():
    assert GBAR1 == 16
    # independently balanced level: d = gbar = [16, 16, 16]
    assert np.allclose(np.full(3, GBAR1), [16, 16, 16])
    # complete compensation of the level-0 imbalance eps_0 = [+8, -4, -4]: [8, 20, 20]
    eps0 = np.array(G0) - np.mean(G0)
    assert np.allclose(eps0, [8, -4, -4])
    assert np.allclose(GBAR1 - eps0, [8, 20, 20])


def test_worked_example_step_weighted_first_distribution():
    # s_0 = 1 remaining level-0 step, s_1 = 2 remaining level-1 steps, nothing done yet
    d = desired_distribution(GBAR1, [G0], [[0, 0, 0]], [1, 2], 1)
    assert np.allclose(d, [12, 18, 18])
    assert np.allclose(desired_distribution_levels(GBAR1, [G0], [[0, 0, 0]], [1, 2], 1), d)


def test_worked_example_second_distribution_with_completed_work():
    # processor 1 completed 6 level-0 updates while waiting: omega_0 = [4, -2, -2]
    w0 = [6, 0, 0]
    assert np.allclose(np.array(w0) - np.mean(w0), [4, -2, -2])
    d = desired_distribution(GBAR1, [G0], [w0], [1, 1], 1)
    assert np.allclose(d, [12, 18, 18])
    assert np.allclose(desired_distribution_levels(GBAR1, [G0], [w0], [1, 1], 1), d)


def test_partition_of_worked_example():
    d = desired_distribution(GBAR1, [G0], [[0, 0, 0]], [1, 2], 1)
    delta = partition(C1, d)
    assert np.allclose(delta, [[12, 18, 2], [0, 0, 8], [0, 0, 8]])
    assert np.allclose(delta.sum(axis=1), C1) and np.allclose(delta.sum(axis=0), d)


@pytest.mark.parametrize("seed", range(5))
def test_shares_equalise_predicted_remaining_work(seed):
    """If every worker gets its desired share (g_l = d_l), the predicted
    remaining work including level l is the same on every worker (the
    equality chain after the distribution equation, Sec. 5); the grouped and
    the level-by-level forms agree."""
    rng = np.random.default_rng(seed)
    P, L = 5, 4
    g = [rng.uniform(50, 150, P) for _ in range(L)]
    s = [2 ** l for l in range(L + 1)]
    w = [rng.uniform(0, 20, P) * (l == 0) for l in range(L)]
    for level in range(1, L + 1):
        gbar = float(rng.uniform(80, 120))
        d = desired_distribution(gbar, g[:level], w[:level], s, level)
        assert np.allclose(d, desired_distribution_levels(gbar, g[:level], w[:level], s, level))
        e = eta(g[:level] + [d], w[:level] + [np.zeros(P)], s, level + 1)
        assert np.allclose(e, e.mean())
        assert np.isclose(d.sum(), P * gbar)


def test_static_mesh_keeps_its_distribution():
    """Appendix B: with a static mesh, after a level-L advance the workers
    spend the wait max_p g_L - g_L^p on coarser work and one level-L step is
    gone; the new desired distribution equals the old one."""
    rng = np.random.default_rng(7)
    P, L = 4, 3
    g = [rng.uniform(50, 150, P) for _ in range(L)]
    s = [1, 2, 4, 8]
    w = [np.zeros(P) for _ in range(L)]
    gbar = 100.0
    d = desired_distribution(gbar, g, w, s, L)
    gL = d
    w2 = [x.copy() for x in w]
    w2[0] = w2[0] + (gL.max() - gL)
    s2 = list(s)
    s2[L] -= 1
    d2 = desired_distribution(gbar, g, w2, s2, L)
    assert np.allclose(d2, d)


def test_assign_items_rounds_to_largest_cover():
    assert assign_items([10, 10, 12], [12, 20]) == [0, 1, 1]
    assert assign_items([5, 5, 5, 5], [10, 10]) == [0, 0, 1, 1]
    with pytest.raises(ValueError):
        partition([1, 2], [4, 4])
