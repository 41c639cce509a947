"""Pins of the oracle's point functions (limiter, fast speed, physical flux,
HLLD) against closed forms and exact invariants -- no GPU."""
import math

import numpy as np
import pytest

import synth

G = 5.0 / 3.0


def rot(d, w):
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    return np.array([w[0], w[1 + d], w[1 + t1], w[1 + t2], w[4], w[5 + d], w[5 + t1], w[5 + t2]])


def test_limiters_closed_forms(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b = rng.normal(size=2)
        vl = 2 * a * b / (a + b) if a * b > 0 else 0.0
        mm = (a if abs(a) < abs(b) else b) if a * b > 0 else 0.0
        mc = math.copysign(min(2 * abs(a), 2 * abs(b), 0.5 * abs(a + b)), a) if a * b > 0 else 0.0
        assert orc.limiter(0, a, b) == pytest.approx(vl, rel=1e-15, abs=0)
        assert orc.limiter(1, a, b) == mm
        assert orc.limiter(2, a, b) == pytest.approx(mc, rel=1e-15, abs=0)
    # tie-break: a*b <= 0 -> 0, and equal one-sided differences give that difference
    assert orc.limiter(0, 0.0, 1.0) == 0.0 and orc.limiter(0, -1.0, 1.0) == 0.0
    assert orc.limiter(0, 0.3, 0.3) == pytest.approx(0.3, rel=1e-15)


def test_fast_speed_closed_forms(orc):
    # no field: sound speed
    assert orc.fast_speed(1.3, 0.7, 0, 0, 0, G) == pytest.approx(math.sqrt(G * 0.7 / 1.3), rel=1e-15)
    # cold plasma, transverse field: Alfven speed of |B|
    assert orc.fast_speed(2.0, 0.0, 0.0, 0.6, 0.8, G) == pytest.approx(1.0 / math.sqrt(2.0), rel=1e-15)
    # field along the normal: max(sound speed, Alfven speed)
    a = math.sqrt(G * 0.5 / 1.0)
    assert orc.fast_speed(1.0, 0.5, 3.0, 0, 0, G) == pytest.approx(3.0, rel=1e-15)
    assert orc.fast_speed(1.0, 0.5, 0.1, 0, 0, G) == pytest.approx(a, rel=1e-15)
    # general case against the quartic: c^4 - (a2+b2) c^2 + a2 bn2 = 0
    rng = np.random.default_rng(2)
    for w in synth.random_states(rng, 100):
        c = orc.fast_speed(w[0], w[4], w[5], w[6], w[7], G)
        a2, b2, bn2 = G * w[4] / w[0], (w[5:8] ** 2).sum() / w[0], w[5] ** 2 / w[0]
        assert abs(c ** 4 - (a2 + b2) * c ** 2 + a2 * bn2) <= 1e-12 * (a2 + b2) ** 2
        assert c * c >= max(a2, b2) * (1 - 1e-14)


def test_physical_flux_closed_form(orc):
    rng = np.random.default_rng(3)
    for w in synth.random_states(rng, 50):
        rho, v, p, B = w[0], w[1:4], w[4], w[5:8]
        E = p / (G - 1) + 0.5 * rho * v @ v + 0.5 * B @ B
        pt = p + 0.5 * B @ B
        for d in range(3):
            f = orc.flux(d, w, G)
            ref = np.zeros(8)
            ref[0] = rho * v[d]
            ref[1:4] = rho * v[d] * v - B[d] * B
            ref[1 + d] += pt
            ref[4] = (E + pt) * v[d] - B[d] * (v @ B)
            ref[5:8] = v[d] * B - B[d] * v
            np.testing.assert_allclose(f, ref, rtol=1e-13, atol=1e-13)
            assert f[5 + d] == 0.0


@pytest.mark.parametrize("bn_zero", [False, True])
def test_hlld_uniform_state_is_physical_flux(orc, bn_zero):
    rng = np.random.default_rng(4 + bn_zero)
    for w in synth.random_states(rng, 300, bn_zero=bn_zero):
        for d in range(3):
            w2 = w.copy()
            if bn_zero:
                w2[5 + d] = 0.0
            f = orc.hlld(d, w2, w2, w2[5 + d], G)
            ref = orc.flux(d, w2, G)
            scale = np.abs(ref).max() + 1.0
            assert np.abs(f - ref).max() <= 1e-15 * 8 * scale


def test_hlld_mirror_symmetry_is_exact(orc):
    """x -> -x maps (vn, Bn) -> (-vn, -Bn) and swaps the sides; the flux of
    every component that is even under the mirror flips sign, the rest keep it."""
    rng = np.random.default_rng(5)
    W = synth.random_states(rng, 400)
    for t in range(0, 400, 2):
        wl, wr = W[t], W[t + 1]
        for d in range(3):
            bn = 0.5 * (wl[5 + d] + wr[5 + d])
            ml, mr = wr.copy(), wl.copy()
            for m in (ml, mr):
                m[1 + d] = -m[1 + d]
                m[5 + d] = -m[5 + d]
            f = orc.hlld(d, wl, wr, bn, G)
            g = orc.hlld(d, ml, mr, -bn, G)
            sign = -np.ones(8)
            sign[1 + d] = 1.0
            sign[5 + d] = 1.0
            assert np.array_equal(g, sign * f), (d, f, g)


def test_hlld_cyclic_axis_invariance_is_exact(orc):
    rng = np.random.default_rng(6)
    W = synth.random_states(rng, 100)
    for t in range(0, 100, 2):
        wl, wr = W[t], W[t + 1]
        f0 = orc.hlld(0, wl, wr, wl[5], G)
        # rotate x->y->z->x: component x of the state becomes component y
        def perm(w):
            o = w.copy()
            o[1 + 1], o[1 + 2], o[1 + 0] = w[1 + 0], w[1 + 1], w[1 + 2]
            o[5 + 1], o[5 + 2], o[5 + 0] = w[5 + 0], w[5 + 1], w[5 + 2]
            return o
        f1 = orc.hlld(1, perm(wl), perm(wr), wl[5], G)
        assert np.array_equal(perm(f0), f1)


def test_hlld_fan_integral_consistency_and_jump_conditions(orc):
    """The four intermediate states obey the integral form of the conservation
    law over the fan (MK05 Sec. 3); the Rankine-Hugoniot condition holds
    across the contact (F_R** - F_L** = S_M (U_R** - U_L**)); the normal momentum flux of every star region is
    rho* S_M^2 + p_T* - Bn^2 with p_T* from MK05 eq. (23) evaluated from either
    side; normal velocity S_M and the Alfven-wave density jumps are as
    constructed; the wave speeds are ordered."""
    rng = np.random.default_rng(7)
    W = synth.random_states(rng, 600)
    checked = 0
    for t in range(0, 600, 2):
        wl, wr = W[t], W[t + 1]
        d = t % 3
        bn = 0.5 * (wl[5 + d] + wr[5 + d])
        if abs(bn) < 0.05:
            continue
        sp, st, fl = orc.hlld_fan(d, wl, wr, bn, G)
        sl, sls, sm, srs, sr = sp
        assert sl <= sls <= sm <= srs <= sr
        ul, usl, ussl, ussr, usr, ur = st
        lhs = (sls - sl) * usl + (sm - sls) * ussl + (srs - sm) * ussr + (sr - srs) * usr
        rhs = sr * ur - sl * ul - (fl[1] - fl[0])
        scale = (sr - sl) * (np.abs(st).max() + np.abs(fl).max())
        assert np.abs(lhs - rhs).max() <= 1e-12 * scale, (lhs - rhs, scale)
        f_ls = fl[0] + sl * (usl - ul)
        f_lss = f_ls + sls * (ussl - usl)
        f_rs = fl[1] + sr * (usr - ur)
        f_rss = f_rs + srs * (ussr - usr)
        fs = np.abs(fl).max() + (sr - sl) * np.abs(st).max()
        assert np.abs((f_rss - f_lss) - sm * (ussr - ussl)).max() <= 1e-12 * fs
        L, R = rot(d, wl), rot(d, wr)
        pt_l = L[4] + 0.5 * (bn * bn + L[6] ** 2 + L[7] ** 2)
        pt_r = R[4] + 0.5 * (bn * bn + R[6] ** 2 + R[7] ** 2)
        pts_l = pt_l + L[0] * (sl - L[1]) * (sm - L[1])
        pts_r = pt_r + R[0] * (sr - R[1]) * (sm - R[1])
        assert pts_l == pytest.approx(pts_r, rel=1e-11, abs=1e-11 * fs)
        for u, f in ((usl, f_ls), (ussl, f_lss), (ussr, f_rss), (usr, f_rs)):
            assert u[1] == pytest.approx(u[0] * sm, rel=1e-14, abs=1e-14)
            assert f[1] == pytest.approx(u[0] * sm * sm + pts_l - bn * bn, rel=1e-10, abs=1e-11 * fs)
        assert usl[0] == ussl[0] and usr[0] == ussr[0]
        checked += 1
    assert checked > 100


def test_hlld_stationary_contact_and_tangential_discontinuity(orc):
    # contact: rho jumps, p, v = 0, B continuous with Bn != 0
    wl = np.array([1.0, 0, 0, 0, 0.6, 0.7, 0.3, -0.2])
    wr = np.array([0.2, 0, 0, 0, 0.6, 0.7, 0.3, -0.2])
    f = orc.hlld(0, wl, wr, 0.7, G)
    pt = 0.6 + 0.5 * (0.49 + 0.09 + 0.04)
    assert abs(f[0]) <= 1e-15 and abs(f[4]) <= 1e-15
    assert f[1] == pytest.approx(pt - 0.49, rel=1e-14)
    assert f[2] == pytest.approx(-0.7 * 0.3, rel=1e-14) and f[3] == pytest.approx(0.7 * 0.2, rel=1e-14)
    assert abs(f[6]) <= 1e-15 and abs(f[7]) <= 1e-15
    # tangential discontinuity: Bn = 0, rho / p / Bt jump with total-pressure balance
    wl = np.array([1.0, 0, 0, 0, 1.0, 0.0, 1.0, 0.0])
    wr = np.array([0.3, 0, 0, 0, 0.7, 0.0, 0.0, math.sqrt(1.6)])
    f = orc.hlld(0, wl, wr, 0.0, G)
    assert abs(f[0]) <= 1e-15 and abs(f[4]) <= 1e-15
    assert f[1] == pytest.approx(1.5, rel=1e-14)
    # hydrodynamic stationary contact (B = 0) is kept exactly as well
    wl = np.array([1.0, 0, 0.2, 0, 1.0, 0, 0, 0])
    wr = np.array([0.125, 0, -0.4, 0, 1.0, 0, 0, 0])
    f = orc.hlld(0, wl, wr, 0.0, G)
    assert abs(f[0]) <= 1e-15 and f[1] == pytest.approx(1.0, rel=1e-15)


def test_hlld_supersonic_and_upwind_side(orc):
    wl = np.array([1.0, 5.0, 0.1, 0.0, 0.1, 0.3, 0.2, 0.1])
    wr = np.array([0.5, 4.0, -0.1, 0.2, 0.2, 0.3, -0.2, 0.0])
    f, up = orc.hlld(0, wl, wr, 0.3, G, with_upwind=True)
    assert np.array_equal(f, orc.flux(0, np.r_[wl[:5], 0.3, wl[6:]], G)) and up == 1.0
    m = wl.copy(); m[1] = -5.0
    f, up = orc.hlld(0, wr * np.r_[1, -1, 1, 1, 1, 1, 1, 1], m, 0.3, G, with_upwind=True)
    assert up == -1.0
    # subsonic: side follows the sign of the mass flux, ties within eps give 0
    wl = np.array([1.0, 0.1, 0, 0, 1.0, 0.5, 0.2, 0.0])
    wr = np.array([1.0, 0.1, 0, 0, 1.0, 0.5, 0.2, 0.0])
    f, up = orc.hlld(0, wl, wr, 0.5, G, with_upwind=True)
    assert up == 1.0 and f[0] > 0
    wl[1] = wr[1] = 0.0
    f, up = orc.hlld(0, wl, wr, 0.5, G, with_upwind=True)
    assert up == 0.0 and f[0] == 0.0
