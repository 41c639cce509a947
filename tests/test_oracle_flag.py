"""Pins of the oracle's error flagging for regridding (Sec. 2.1 leaves the
criterion to the application; reading: the normalised central difference
|q(+d) - q(-d)| / (|q(+d)| + 2|q| + |q(-d)|) of q = rho or p along some axis
exceeds theta) -- no GPU.  Closed forms: a uniform state flags nothing; a
density step of ratio 2 gives eta = 1/5 on the cell below it and 1/7 on the
cell above it and 0 elsewhere; a linear density ramp rho_j = 1 + 0.1 j gives
eta_j = 0.2 / (4 + 0.4 j); a pressure step flags like a density step; the
criterion is the same along every axis."""
import numpy as np
import pytest

import synth

G = 2
GAMMA = 5.0 / 3.0


def state(n, rho, p, v=(0.0, 0.0, 0.0), B=(0.3, -0.2, 0.1)):
    """Cells of the whole array (ghosts included) from rho(i, j, k) and p
    given as arrays over (NZ, NY, NX) cell indices."""
    st = synth.empty_patch(n, G)
    N = [a + 2 * G for a in n]
    for a in range(3):
        st[5 + a] = B[a]
    sl = (slice(0, N[2]), slice(0, N[1]), slice(0, N[0]))
    st[(0,) + sl] = rho
    for a in range(3):
        st[(1 + a,) + sl] = rho * v[a]
    ke = 0.5 * rho * sum(x * x for x in v)
    st[(4,) + sl] = p / (GAMMA - 1.0) + ke + 0.5 * sum(b * b for b in B)
    return st


def idx(n):
    N = [a + 2 * G for a in n]
    k, j, i = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    return i - G, j - G, k - G   # interior-relative cell indices


def flags(orc, st, n, theta):
    P = orc.patch(st, n, G, (1.0, 1.0, 1.0))
    return orc.flag(P, orc.params(), theta)


def test_uniform_state_flags_nothing(orc):
    n = (6, 5, 4)
    st = state(n, 1.3, 0.7, v=(0.2, -0.1, 0.3))
    assert flags(orc, st, n, 1e-12).sum() == 0


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("which", ["rho", "p"])
def test_step_flags_closed_form(orc, axis, which):
    n = (8, 8, 8)
    ii = idx(n)[axis]
    jump = np.where(ii >= 4, 2.0, 1.0)
    st = state(n, jump if which == "rho" else 1.0, jump if which == "p" else 1.0)
    want_lo = np.zeros(8, dtype=np.uint8)
    for theta, below, above in ((0.1, 1, 1), (0.15, 1, 0), (0.25, 0, 0)):
        f = flags(orc, st, n, theta)
        line = np.moveaxis(f, 2 - axis, 0)        # flags as a function of the index along `axis`
        expect = want_lo.copy()
        expect[3] = below                          # eta = 1 / (2 + 2 + 1)
        expect[4] = above                          # eta = 1 / (2 + 4 + 1)
        assert np.array_equal(line.reshape(8, -1).max(1), expect), (theta, line.reshape(8, -1).max(1))
        assert np.array_equal(line.reshape(8, -1).min(1), expect)


def test_linear_ramp_threshold(orc):
    n = (4, 12, 4)
    j = idx(n)[1]
    st = state(n, 1.0 + 0.1 * j, 1.0)
    for theta in (0.01, 0.02, 0.03, 0.04):
        f = flags(orc, st, n, theta)
        jj = np.arange(12)
        expect = (0.2 > theta * (4.0 + 0.4 * jj)).astype(np.uint8)
        got = f.transpose(1, 0, 2).reshape(12, -1)
        assert np.array_equal(got.max(1), expect) and np.array_equal(got.min(1), expect), theta
