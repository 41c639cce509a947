"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the solver: it only lays out arrays and
evaluates the initial conditions of the test problems (Orszag-Tang vortex,
blast wave, linear Alfven wave, uniform states) and the seeded noise.  Both
the FP64 oracle and the GPU path start from the arrays produced here.

Layout of one patch (``patch_shape``): a float array of shape
``(8, NZ+1, NY+1, PX)`` with ``N* = n* + 2g`` and a row pitch ``PX >= NX+1``
rounded up to ``align`` elements.  Planes 0..4 hold rho, Mx, My, Mz, E at cell
centres; planes 5..7 hold Bx, By, Bz on the lower x-, y-, z-faces of each
cell (one extra entry along each normal).  Cell (i, j, k) is ``[q, k, j, i]``.
Only the interior (and the interior faces) are written; ghosts are left at 0
and must be filled by the caller.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 5.0 / 3.0

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 input."""
    z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
    return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, index: np.ndarray) -> np.ndarray:
    """Counter-based U(-1, 1): u = (splitmix64(seed ^ index) >> 11) * 2^-53."""
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed) ^ index.astype(np.uint64))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def patch_shape(n, g: int, align: int = 8):
    nx, ny, nz = (int(v) for v in n)
    NX, NY, NZ = nx + 2 * g, ny + 2 * g, nz + 2 * g
    px = -(-(NX + 1) // align) * align
    return (8, NZ + 1, NY + 1, px)


def empty_patch(n, g: int, dtype=np.float64, align: int = 8) -> np.ndarray:
    return np.zeros(patch_shape(n, g, align), dtype=dtype)


def _centres(n, g, lo_idx, xlo, dx):
    """Cell-centre coordinates of the interior along each axis."""
    out = []
    for d in range(3):
        i = np.arange(n[d], dtype=np.float64) + lo_idx[d]
        out.append(xlo[d] + (i + 0.5) * dx[d])
    return out


def _face_b_from_potential(state, n, g, xlo, dx, lo_idx, A):
    """Face B = discrete curl of an edge-sampled vector potential A(x,y,z) ->
    (Ax, Ay, Az) (callables on broadcast arrays).  Writes the interior faces,
    including the upper boundary faces."""
    nx, ny, nz = n
    i0, j0, k0 = lo_idx

    def edge_coords(axis, ii, jj, kk):
        # edge along `axis` at the lower corner of cell (ii, jj, kk): centred on
        # the cell along `axis`, at the lower face along the other two.
        xs = [xlo[0] + (ii + i0) * dx[0], xlo[1] + (jj + j0) * dx[1], xlo[2] + (kk + k0) * dx[2]]
        pos = [ii, jj, kk]
        xs[axis] = xlo[axis] + (pos[axis] + lo_idx[axis] + 0.5) * dx[axis]
        return xs

    def comp(axis, ii, jj, kk):
        x, y, z = edge_coords(axis, ii, jj, kk)
        return A[axis](x, y, z)

    # Bx on x-faces: i in [0, nx], j in [0, ny), k in [0, nz)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1.0), np.arange(ny + 0.0), np.arange(nz + 0.0), indexing="ij")
    bx = (comp(2, ii, jj + 1, kk) - comp(2, ii, jj, kk)) / dx[1] - (comp(1, ii, jj, kk + 1) - comp(1, ii, jj, kk)) / dx[2]
    ii, jj, kk = np.meshgrid(np.arange(nx + 0.0), np.arange(ny + 1.0), np.arange(nz + 0.0), indexing="ij")
    by = (comp(0, ii, jj, kk + 1) - comp(0, ii, jj, kk)) / dx[2] - (comp(2, ii + 1, jj, kk) - comp(2, ii, jj, kk)) / dx[0]
    ii, jj, kk = np.meshgrid(np.arange(nx + 0.0), np.arange(ny + 0.0), np.arange(nz + 1.0), indexing="ij")
    bz = (comp(1, ii + 1, jj, kk) - comp(1, ii, jj, kk)) / dx[0] - (comp(0, ii, jj + 1, kk) - comp(0, ii, jj, kk)) / dx[1]
    state[5, g:g + nz, g:g + ny, g:g + nx + 1] = np.transpose(bx, (2, 1, 0))
    state[6, g:g + nz, g:g + ny + 1, g:g + nx] = np.transpose(by, (2, 1, 0))
    state[7, g:g + nz + 1, g:g + ny, g:g + nx] = np.transpose(bz, (2, 1, 0))


def _set_cells(state, n, g, rho, vx, vy, vz, p, gamma):
    """Fill rho, M, E of the interior; E uses the face-averaged cell B."""
    nx, ny, nz = n
    sl = (slice(g, g + nz), slice(g, g + ny), slice(g, g + nx))
    bx = 0.5 * (state[5, g:g + nz, g:g + ny, g:g + nx] + state[5, g:g + nz, g:g + ny, g + 1:g + nx + 1])
    by = 0.5 * (state[6, g:g + nz, g:g + ny, g:g + nx] + state[6, g:g + nz, g + 1:g + ny + 1, g:g + nx])
    bz = 0.5 * (state[7, g:g + nz, g:g + ny, g:g + nx] + state[7, g + 1:g + nz + 1, g:g + ny, g:g + nx])
    rho = np.broadcast_to(rho, (nz, ny, nx))
    vx, vy, vz, p = (np.broadcast_to(a, (nz, ny, nx)) for a in (vx, vy, vz, p))
    state[(0,) + sl] = rho
    state[(1,) + sl] = rho * vx
    state[(2,) + sl] = rho * vy
    state[(3,) + sl] = rho * vz
    state[(4,) + sl] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)


class Problem:
    """A generated periodic single-patch problem."""

    def __init__(self, name, state, n, g, dx, xlo, gamma=GAMMA):
        self.name, self.state, self.n, self.g, self.dx, self.xlo, self.gamma = name, state, tuple(n), g, tuple(dx), tuple(xlo), gamma

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def orszag_tang(n: int = 128, g: int = 2, align: int = 8) -> Problem:
    """2D Orszag-Tang vortex on [0,1]^2 (one cell along z): rho = 25/(36 pi),
    p = 5/(12 pi), v = (-sin 2pi y, sin 2pi x), B = B0 (-sin 2pi y, sin 4pi x),
    B0 = 1/sqrt(4 pi); face B from A_z = B0 (cos 4pi x / 4pi + cos 2pi y / 2pi)."""
    nn = (n, n, 1)
    dx = (1.0 / n, 1.0 / n, 1.0 / n)
    xlo = (0.0, 0.0, 0.0)
    st = empty_patch(nn, g, align=align)
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    zero = lambda x, y, z: 0.0 * x
    az = lambda x, y, z: b0 * (np.cos(4.0 * np.pi * x) / (4.0 * np.pi) + np.cos(2.0 * np.pi * y) / (2.0 * np.pi))
    _face_b_from_potential(st, nn, g, xlo, dx, (0, 0, 0), (zero, zero, az))
    x, y, _ = _centres(nn, g, (0, 0, 0), xlo, dx)
    X = x[None, None, :]
    Y = y[None, :, None]
    rho = 25.0 / (36.0 * math.pi)
    p = 5.0 / (12.0 * math.pi)
    _set_cells(st, nn, g, rho, -np.sin(2 * np.pi * Y), np.sin(2 * np.pi * X), 0.0, p, GAMMA)
    return Problem("orszag_tang", st, nn, g, dx, xlo)


def blast(n: int = 128, g: int = 2, seed: int = 1710, noise: float = 0.01, align: int = 8,
          p_in: float = 10.0, p_out: float = 0.1, r0: float = 0.1) -> Problem:
    """3D blast wave on the periodic cube [-1/2, 1/2]^3: rho = 1 + noise*U(-1,1)
    (counter-based, index = i + n (j + n k)), v = 0, p = p_in for r < r0 else
    p_out, B = (1, 1, 0)/sqrt(2)."""
    nn = (n, n, n)
    dx = (1.0 / n,) * 3
    xlo = (-0.5, -0.5, -0.5)
    st = empty_patch(nn, g, align=align)
    b = 1.0 / math.sqrt(2.0)
    st[5, g:g + n, g:g + n, g:g + n + 1] = b
    st[6, g:g + n, g:g + n + 1, g:g + n] = b
    st[7, g:g + n + 1, g:g + n, g:g + n] = 0.0
    x, y, z = _centres(nn, g, (0, 0, 0), xlo, dx)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]
    r2 = X * X + Y * Y + Z * Z
    p = np.where(r2 < r0 * r0, p_in, p_out)
    idx = (np.arange(n, dtype=np.uint64)[None, None, :]
           + np.uint64(n) * (np.arange(n, dtype=np.uint64)[None, :, None]
                             + np.uint64(n) * np.arange(n, dtype=np.uint64)[:, None, None]))
    rho = 1.0 + noise * uniform_pm1(seed, idx) if noise else np.ones((n, n, n))
    _set_cells(st, nn, g, rho, 0.0, 0.0, 0.0, p, GAMMA)
    return Problem("blast", st, nn, g, dx, xlo)


def alfven_wave(n: int, ndim: int = 2, amp: float = 1e-6, g: int = 2, align: int = 8):
    """Linear Alfven wave on the unit periodic box: rho = 1, p = 1/gamma, B0 = k_hat
    (v_A = 1); k = 2 pi (1, 2) in 2D (polarisation along z) or 2 pi (1, 1, 1) in
    3D (polarisation (1, -1, 0)/sqrt 2); dB = amp cos(k.x) e, dv = -dB/sqrt(rho).
    Returns (problem, exact(t) -> dict of cell-centre fields, period)."""
    if ndim == 2:
        nn = (n, n, 1)
        kvec = np.array([2 * np.pi, 4 * np.pi, 0.0])
    else:
        nn = (n, n, n)
        kvec = np.array([2 * np.pi, 2 * np.pi, 2 * np.pi])
    dx = (1.0 / n,) * 3
    xlo = (0.0, 0.0, 0.0)
    kmag = float(np.linalg.norm(kvec))
    khat = kvec / kmag
    e = np.array([0.0, 0.0, 1.0]) if ndim == 2 else np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    axb = np.cross(e, khat)  # dA direction: curl(f(k.x) (e x k_hat)) = f' k x (e x k_hat) = f' |k| e
    st = empty_patch(nn, g, align=align)
    # uniform B0 = k_hat through A0 = (0, 0, B0x y - B0y x) + (B0y z ... ) : use A0 = 1/2 B0 x r
    def A(c):
        def f(x, y, z):
            r = (x, y, z)
            a0 = 0.5 * (khat[(c + 1) % 3] * r[(c + 2) % 3] - khat[(c + 2) % 3] * r[(c + 1) % 3])
            ph = kvec[0] * x + kvec[1] * y + kvec[2] * z
            return a0 + (amp / kmag) * np.sin(ph) * axb[c]
        return f
    _face_b_from_potential(st, nn, g, xlo, dx, (0, 0, 0), (A(0), A(1), A(2)))
    x, y, z = _centres(nn, g, (0, 0, 0), xlo, dx)
    X, Y, Z = x[None, None, :], y[None, :, None], z[:, None, None]

    def fields(t):
        ph = kvec[0] * X + kvec[1] * Y + kvec[2] * Z - kmag * 1.0 * t
        db = amp * np.cos(ph)
        return {"v": [-db * e[c] for c in range(3)], "B": [khat[c] + db * e[c] for c in range(3)]}

    f0 = fields(0.0)
    _set_cells(st, nn, g, 1.0, f0["v"][0], f0["v"][1], f0["v"][2], 1.0 / GAMMA, GAMMA)
    period = 2 * np.pi / kmag
    return Problem("alfven%dd" % ndim, st, nn, g, dx, xlo), fields, period


def uniform(n, g: int = 2, rho=1.3, v=(0.3, -0.2, 0.1), p=0.7, B=(0.4, -0.5, 0.6), align: int = 8) -> Problem:
    nn = tuple(int(a) for a in n)
    dx = tuple(1.0 / a for a in nn)
    st = empty_patch(nn, g, align=align)
    nx, ny, nz = nn
    st[5, g:g + nz, g:g + ny, g:g + nx + 1] = B[0]
    st[6, g:g + nz, g:g + ny + 1, g:g + nx] = B[1]
    st[7, g:g + nz + 1, g:g + ny, g:g + nx] = B[2]
    _set_cells(st, nn, g, rho, v[0], v[1], v[2], p, GAMMA)
    return Problem("uniform", st, nn, g, dx, (0.0, 0.0, 0.0))


def random_states(rng: np.random.Generator, count: int, bn_zero: bool = False) -> np.ndarray:
    """Random positive primitive states (rho, vx, vy, vz, p, Bx, By, Bz)."""
    w = np.empty((count, 8))
    w[:, 0] = rng.uniform(0.1, 3.0, count)
    w[:, 1:4] = rng.uniform(-2.0, 2.0, (count, 3))
    w[:, 4] = rng.uniform(0.05, 3.0, count)
    w[:, 5:8] = rng.uniform(-2.0, 2.0, (count, 3))
    if bn_zero:
        w[:, 5] = 0.0
    return w


def field_loop(n: int, normal: int = 2, v=(1.0, 0.5, 0.0), amp: float = 1e-3, radius: float = 0.3,
               g: int = 2, align: int = 8) -> Problem:
    """Weak magnetic field loop in a uniform flow (the advection test Gardiner
    & Stone 2005 use for their edge EMF): a periodic n x n patch one cell
    thick along axis `normal`, on [-1/2, 1/2] per axis, rho = 1, p = 1,
    velocity v, and face B from the vector potential A_normal = amp (radius -
    r) inside r < radius (r measured in the plane), else 0.  The field is
    passive to rounding (magnetic pressure amp^2 against p = 1)."""
    nn = [n, n, n]
    nn[normal] = 1
    nn = tuple(nn)
    dx = tuple(1.0 / a for a in nn)
    xlo = (-0.5, -0.5, -0.5)
    st = empty_patch(nn, g, align=align)
    t1, t2 = (normal + 1) % 3, (normal + 2) % 3

    def a_n(x, y, z):
        r3 = (x, y, z)
        r = np.sqrt(r3[t1] ** 2 + r3[t2] ** 2)
        return np.where(r < radius, amp * (radius - r), 0.0)

    zero = lambda x, y, z: 0.0 * x
    A = [zero, zero, zero]
    A[normal] = a_n
    _face_b_from_potential(st, nn, g, xlo, dx, (0, 0, 0), tuple(A))
    _set_cells(st, nn, g, 1.0, v[0], v[1], v[2], 1.0, GAMMA)
    return Problem("field_loop", st, nn, g, dx, xlo)


def swirl_2d(n: int, seed: int = 5, g: int = 2, align: int = 8) -> Problem:
    """Smooth 2D state on the unit periodic square whose velocity changes
    sign across the grid along both axes (v_x = 0.8 sin(2 pi y + 0.3) + 0.2
    cos 2 pi x, v_y = 0.7 sin(2 pi x + 1.1) - 0.3 cos 2 pi y, v_z = 0.1), rho = 1 +
    0.2 sin 2 pi (x + y), p = 1, and a field from three seeded Fourier modes of
    A_z (amplitude 0.05 each)."""
    rng = np.random.default_rng(seed)
    nn = (n, n, 1)
    dx = (1.0 / n,) * 3
    xlo = (0.0, 0.0, 0.0)
    st = empty_patch(nn, g, align=align)
    modes = [(int(rng.integers(1, 3)), int(rng.integers(1, 3)), rng.uniform(0, 2 * np.pi), rng.uniform(-1, 1))
             for _ in range(3)]

    def az(x, y, z):
        return sum(0.05 * a * np.cos(2 * np.pi * (kx * x + ky * y) + ph) for kx, ky, ph, a in modes)

    zero = lambda x, y, z: 0.0 * x
    _face_b_from_potential(st, nn, g, xlo, dx, (0, 0, 0), (zero, zero, az))
    x = (np.arange(n) + 0.5) / n
    X, Y = x[None, None, :], x[None, :, None]
    vx = 0.8 * np.sin(2 * np.pi * Y + 0.3) + 0.2 * np.cos(2 * np.pi * X)
    vy = 0.7 * np.sin(2 * np.pi * X + 1.1) - 0.3 * np.cos(2 * np.pi * Y)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * (X + Y))
    _set_cells(st, nn, g, rho, vx, vy, 0.1, 1.0, GAMMA)
    return Problem("swirl_2d", st, nn, g, dx, xlo)


def split_x(pr: Problem, at: int, g: int = None):
    """Two patches cut from a single-patch problem whose ghosts are already
    filled (periodic images): A holds interior cells x < at, B the rest, both
    with g ghost layers taken from the filled array (so each one's ghosts hold
    the other's cells and the periodic images).  Returns (A, B) states and
    their interior sizes."""
    g = pr.g if g is None else g
    assert g == pr.g
    nx, ny, nz = pr.n
    na, nb = (at, ny, nz), (nx - at, ny, nz)
    A = empty_patch(na, g)
    B = empty_patch(nb, g)
    A[:, :, :, :at + 2 * g + 1] = pr.state[:, :, :, :at + 2 * g + 1]
    B[:, :, :, :nx - at + 2 * g + 1] = pr.state[:, :, :, at:nx + 2 * g + 1]
    return A, na, B, nb
