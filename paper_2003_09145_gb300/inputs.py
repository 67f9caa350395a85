"""Seeded synthetic inputs shaped like the paper's test problems.

This module is shared by the CUDA path's tests and benchmark and by the oracle's
tests.  It holds no arithmetic of the numerical method: only initial conditions
given as primitive states (rho, u, [v, [w]], p) and their conversion to the
conservative variables of the Euler equations with the ideal-gas law
E = p/(gamma-1) + rho |u|^2 / 2 (eq. 4.7).

Layout of every returned state: float64 ``[nvar][n_z][n_y][n_x]`` (x fastest),
squeezed to ``[nvar][n]`` in 1D and ``[nvar][n_y][n_x]`` in 2D.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
PERIODIC = 0
TRANSMISSIVE = 1
REFLECTIVE = 2


def prim_to_cons(rho, vel, p, gamma: float = GAMMA) -> np.ndarray:
    """(rho, [u, v, w], p) -> (rho, rho u, ..., E) with E = p/(gamma-1) + rho|u|^2/2."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = [np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape) for v in vel]
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    q2 = sum(v * v for v in vel)
    E = p / (gamma - 1.0) + 0.5 * rho * q2
    return np.ascontiguousarray(np.stack([rho] + [rho * v for v in vel] + [E]))


@dataclass
class Problem:
    """A grid, its boundary types, an initial state and the run parameters."""
    name: str
    U0: np.ndarray
    n: tuple
    dx: tuple
    bc: tuple
    t_end: float
    cfl: float = 0.5
    gamma: float = GAMMA
    x0: tuple = ()          # lower corner of the domain
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))

    def centers(self, d: int) -> np.ndarray:
        """Cell-centre coordinates x_i = a + (i + 1/2) dx along direction d."""
        return self.x0[d] + (np.arange(self.n[d]) + 0.5) * self.dx[d]


def shock_tube(n: int = 200, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
               a: float = 0.0, b: float = 1.0, x_jump: float = 0.5,
               t_end: float = 0.2, name: str = "sod") -> Problem:
    """1D Riemann problem on [a, b], left state where x <= x_jump (eq. 4.8).

    Defaults: Sod's tube on [0,1], N = 200, jump at 0.5, transmissive ends."""
    dx = (b - a) / n
    x = a + (np.arange(n) + 0.5) * dx
    isl = x <= x_jump
    rho = np.where(isl, left[0], right[0])
    u = np.where(isl, left[1], right[1])
    p = np.where(isl, left[2], right[2])
    return Problem(name, prim_to_cons(rho, [u], p), (n,), (dx,), (TRANSMISSIVE,), t_end,
                   x0=(a,), extra={"left": tuple(left), "right": tuple(right), "x_jump": x_jump})


def sod_paper(n: int = 400, t_end: float = 0.14) -> Problem:
    """Sod's tube as in Sec. 4.2 (eq. 4.8): [-0.5, 0.5], left state where x <= 0,
    zero-gradient ends; the paper's figures use N = 400 at t = 0.14."""
    return shock_tube(n, a=-0.5, b=0.5, x_jump=0.0, t_end=t_end, name="sod_paper")


def lax_tube(n: int = 400, t_end: float = 0.13) -> Problem:
    """Lax's tube (eq. 4.9): (0.445, 0.698, 3.528) where x <= 0, else
    (0.5, 0, 0.571), on [-5, 5] with zero-gradient ends; the paper's figures
    use N = 400 at t = 0.13."""
    return shock_tube(n, left=(0.445, 0.698, 3.528), right=(0.5, 0.0, 0.571), a=-5.0, b=5.0,
                      x_jump=0.0, t_end=t_end, name="lax")


def blast_waves(n: int = 400, t_end: float = 0.038) -> Problem:
    """Two interacting blast waves (eq. 4.11) on [0, 1] with reflecting walls:
    at rest, rho = 1, p = 1000 for x < 0.1, 0.01 for 0.1 <= x < 0.9 (the
    printed middle range reads 0 <= x < 0.9), 100 for x >= 0.9; the paper's
    figure uses N = 400 at t = 0.038."""
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    return Problem("blast_waves", prim_to_cons(np.ones(n), [np.zeros(n)], p), (n,), (dx,), (REFLECTIVE,), t_end,
                   x0=(0.0,))


def shu_osher(n: int = 4096, t_end: float = 1.8) -> Problem:
    """Shock / entropy-wave interaction on [-5, 5] (eq. 4.10), with the post-shock
    state given to six digits: (3.857143, 2.629369, 10.3333) for x < -4, else
    rho = 1 + 0.2 sin(5x), u = 0, p = 1; transmissive ends."""
    a, b = -5.0, 5.0
    dx = (b - a) / n
    x = a + (np.arange(n) + 0.5) * dx
    post = x < -4.0
    rho = np.where(post, 3.857143, 1.0 + 0.2 * np.sin(5.0 * x))
    u = np.where(post, 2.629369, 0.0)
    p = np.where(post, 10.3333, 1.0)
    return Problem("shu_osher", prim_to_cons(rho, [u], p), (n,), (dx,), (TRANSMISSIVE,), t_end,
                   x0=(a,))


def entropy_wave(n: int, t_end: float = 2.0, amp: float = 0.2) -> Problem:
    """Smooth periodic density wave on [-1, 1]: rho = 1 + amp sin(pi x), u = 1, p = 1.
    The exact solution is the initial profile advected with speed 1."""
    a, b = -1.0, 1.0
    dx = (b - a) / n
    x = a + (np.arange(n) + 0.5) * dx
    rho = 1.0 + amp * np.sin(np.pi * x)
    return Problem(f"entropy_wave_{n}", prim_to_cons(rho, [np.ones(n)], np.ones(n)), (n,), (dx,),
                   (PERIODIC,), t_end, x0=(a,))


# Scalar linear advection u_t + u_x = 0 on [-1, 1], periodic (Sec. 4.1), on
# the points x_i = -1 + i dx, dx = 2/n.
def scalar_points(n: int) -> np.ndarray:
    return -1.0 + np.arange(n) * (2.0 / n)


def scalar_smooth(n: int) -> np.ndarray:
    """u0 = sin(pi x - sin(pi x) / pi) (eq. 4.5), with two critical points where
    the first derivative vanishes and the third does not: Tab. 1's test."""
    x = scalar_points(n)
    return np.sin(np.pi * x - np.sin(np.pi * x) / np.pi)


def scalar_composite(n: int) -> np.ndarray:
    """The composite profile of eq. 4.6: Gaussians on [-0.8, -0.6), a square
    wave on [-0.4, -0.2), a triangle on [0, 0.2), a half ellipse on
    [0.4, 0.6), 0 elsewhere (a = 0.5, z = -0.7, delta = 0.005, alpha = 10,
    beta = log 2 / (36 delta^2))."""
    x = scalar_points(n)
    a, z, delta, alpha = 0.5, -0.7, 0.005, 10.0
    beta = np.log(2.0) / (36.0 * delta * delta)

    def G(c):
        return np.exp(-beta * (x - c) ** 2)

    def F(c):
        return np.sqrt(np.maximum(1.0 - alpha * alpha * (x - c) ** 2, 0.0))

    u = np.zeros(n)
    m = (x >= -0.8) & (x < -0.6)
    u[m] = ((G(z - delta) + G(z + delta) + 4.0 * G(z)) / 6.0)[m]
    u[(x >= -0.4) & (x < -0.2)] = 1.0
    m = (x >= 0.0) & (x < 0.2)
    u[m] = (1.0 - np.abs(10.0 * (x - 0.1)))[m]
    m = (x >= 0.4) & (x < 0.6)
    u[m] = ((F(a - delta) + F(a + delta) + 4.0 * F(a)) / 6.0)[m]
    return u


# 2D four-quadrant Riemann problem: quadrant states as (rho, u, v, p)
QUADRANTS_LAX_LIU_3 = {
    "NE": (1.5, 0.0, 0.0, 1.5),
    "NW": (0.5323, 1.206, 0.0, 0.3),
    "SW": (0.138, 1.206, 1.206, 0.029),
    "SE": (0.5323, 0.0, 1.206, 0.3),
}


# configuration 12 of the same family (eq. 4.13)
QUADRANTS_CONFIG_12 = {
    "NE": (0.5313, 0.0, 0.0, 0.4),
    "NW": (1.0, 0.7276, 0.0, 1.0),
    "SW": (0.8, 0.0, 0.0, 1.0),
    "SE": (1.0, 0.0, 0.7276, 1.0),
}


def riemann_2d(n: int = 2048, split=(0.8, 0.8), states=QUADRANTS_LAX_LIU_3,
               t_end: float = 0.8, ny: int | None = None) -> Problem:
    """Four-quadrant 2D Riemann problem on [0,1]^2 (eq. 4.14 layout), quadrants split
    at ``split``; a cell is 'east' if x > split[0] and 'north' if y > split[1];
    transmissive boundaries."""
    nx = n
    ny = ny or n
    dx, dy = 1.0 / nx, 1.0 / ny
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y, indexing="xy")       # [ny][nx]
    east = X > split[0]
    north = Y > split[1]
    prim = np.zeros((4, ny, nx))
    for key, mask in (("NE", east & north), ("NW", ~east & north),
                      ("SW", ~east & ~north), ("SE", east & ~north)):
        for c in range(4):
            prim[c][mask] = states[key][c]
    U = prim_to_cons(prim[0], [prim[1], prim[2]], prim[3])
    return Problem("riemann2d", U, (nx, ny), (dx, dy), (TRANSMISSIVE, TRANSMISSIVE), t_end,
                   x0=(0.0, 0.0))


def rayleigh_taylor(nx: int = 128, ny: int = 512, t_end: float = 1.95, perturb: bool = True) -> Problem:
    """Sec. 4.3.2's Rayleigh-Taylor instability (eq. 4.12): [0, 0.25] x [0, 1],
    gamma = 5/3, heavy fluid (rho 2, p = 2y + 1) below y = 1/2 and light fluid
    (rho 1, p = y + 3/2) above, v = -0.025 c cos(8 pi x) with c = sqrt(gamma
    p / rho) (perturb = False: at rest, a hydrostatic state); reflecting left
    and right walls, fixed states (rho, u, v, p) = (2, 0, 0, 1) at the bottom
    and (1, 0, 0, 2.5) at the top; the body force adds rho to the y momentum
    and rho v to the energy (grav = (0, 1)).  extra: grav, bc_state (the
    conservative ghost states, [axis][side])."""
    gamma = 5.0 / 3.0
    dx = (0.25 / nx, 1.0 / ny)
    x = (np.arange(nx) + 0.5) * dx[0]
    y = (np.arange(ny) + 0.5) * dx[1]
    X, Y = np.meshgrid(x, y, indexing="xy")            # [ny][nx]
    low = Y < 0.5
    rho = np.where(low, 2.0, 1.0)
    p = np.where(low, 2.0 * Y + 1.0, Y + 1.5)
    c = np.sqrt(gamma * p / rho)
    v = -0.025 * c * np.cos(8.0 * np.pi * X) if perturb else np.zeros_like(X)
    U0 = prim_to_cons(rho, [np.zeros_like(X), v], p, gamma)
    bottom = prim_to_cons(np.array(2.0), [np.array(0.0), np.array(0.0)], np.array(1.0), gamma)
    top = prim_to_cons(np.array(1.0), [np.array(0.0), np.array(0.0)], np.array(2.5), gamma)
    bc_state = [None, [bottom.reshape(-1).tolist(), top.reshape(-1).tolist()]]
    return Problem("rayleigh_taylor", U0, (nx, ny), dx, (2, 3), t_end, 0.5, gamma, (0.0, 0.0),
                   {"grav": (0.0, 1.0), "bc_state": bc_state})


def riemann_2d_config3(n: int = 1024, t_end: float = 0.3) -> Problem:
    """Sec. 4.3.1's first case (eq. 4.14): the states of QUADRANTS_LAX_LIU_3 split
    at (0.5, 0.5), integrated to t = 0.3 on 1024^2 in the paper."""
    P = riemann_2d(n, split=(0.5, 0.5), states=QUADRANTS_LAX_LIU_3, t_end=t_end)
    P.name = "riemann2d_config3"
    return P


def riemann_2d_config12(n: int = 1024, t_end: float = 0.25) -> Problem:
    """Sec. 4.3.1's second case (eq. 4.13): split at (0.5, 0.5), integrated to
    t = 0.25 on 1024^2 and 2048^2 in the paper."""
    P = riemann_2d(n, split=(0.5, 0.5), states=QUADRANTS_CONFIG_12, t_end=t_end)
    P.name = "riemann2d_config12"
    return P


@dataclass
class TubeBatch:
    """A batch of independent 1D shock tubes on [0, 1] packed as SoA
    ``U[3][sum N]``; problem i owns cells ``offsets[i]:offsets[i+1]``."""
    n: np.ndarray          # int64 [nprob]
    offsets: np.ndarray    # int64 [nprob + 1]
    dx: np.ndarray         # float64 [nprob]
    x_jump: np.ndarray     # float64 [nprob]
    left: np.ndarray       # float64 [nprob][3] (rho, u, p)
    right: np.ndarray      # float64 [nprob][3]
    U0: np.ndarray         # float64 [3][sum N]
    gamma: float = GAMMA

    @property
    def nprob(self) -> int:
        return int(self.n.size)

    @property
    def ncell(self) -> int:
        return int(self.offsets[-1])


def tube_batch(nprob: int = 4096, n_min: int = 64, n_max: int = 4096,
               seed: int = 20200320) -> TubeBatch:
    """Seeded batch of shock tubes: N log-uniform in [n_min, n_max], left/right
    rho ~ U[0.1, 2], u ~ U[-1, 1], p ~ U[0.1, 10], jump x ~ U[0.3, 0.7]."""
    rng = np.random.default_rng(seed)
    logn = rng.uniform(np.log(n_min), np.log(n_max), size=nprob)
    n = np.clip(np.rint(np.exp(logn)).astype(np.int64), n_min, n_max)
    rho = rng.uniform(0.1, 2.0, size=(nprob, 2))
    u = rng.uniform(-1.0, 1.0, size=(nprob, 2))
    p = rng.uniform(0.1, 10.0, size=(nprob, 2))
    xj = rng.uniform(0.3, 0.7, size=nprob)
    offsets = np.zeros(nprob + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(n)
    dx = 1.0 / n.astype(np.float64)
    rho_c = np.empty(offsets[-1])
    u_c = np.empty(offsets[-1])
    p_c = np.empty(offsets[-1])
    for i in range(nprob):
        x = (np.arange(n[i]) + 0.5) * dx[i]
        isl = x <= xj[i]
        s = slice(offsets[i], offsets[i + 1])
        rho_c[s] = np.where(isl, rho[i, 0], rho[i, 1])
        u_c[s] = np.where(isl, u[i, 0], u[i, 1])
        p_c[s] = np.where(isl, p[i, 0], p[i, 1])
    left = np.stack([rho[:, 0], u[:, 0], p[:, 0]], axis=1)
    right = np.stack([rho[:, 1], u[:, 1], p[:, 1]], axis=1)
    return TubeBatch(n, offsets, dx, xj, left, right, prim_to_cons(rho_c, [u_c], p_c))


def solenoidal_turbulence(n: int = 256, mach: float = 0.6, k0: float = 4.0, seed: int = 1,
                          gamma: float = GAMMA, t_end: float = float("inf")) -> Problem:
    """3D periodic box [0, 2 pi]^3 with a random-phase solenoidal velocity field of
    spectrum E(k) ~ k^4 exp(-2 (k/k0)^2), rho = 1, p = 1/gamma (so c = 1), scaled to
    turbulent Mach number sqrt(<|u|^2>)/c = ``mach``."""
    rng = np.random.default_rng(seed)
    L = 2.0 * np.pi
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")  # [x][y][z]
    K2 = KX * KX + KY * KY + KZ * KZ
    K = np.sqrt(K2)
    # random complex amplitudes, made divergence-free by projection
    a = rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))
    K2s = np.where(K2 == 0, 1.0, K2)
    kdota = (KX * a[0] + KY * a[1] + KZ * a[2]) / K2s
    a[0] -= KX * kdota
    a[1] -= KY * kdota
    a[2] -= KZ * kdota
    # shell amplitude so that the energy per shell follows E(k): |a|^2 ~ E(k) / k^2
    Ek = K ** 4 * np.exp(-2.0 * (K / k0) ** 2)
    amp = np.where(K2 == 0, 0.0, np.sqrt(Ek / np.maximum(K2, 1.0)))
    vel = np.real(np.fft.ifftn(a * amp, axes=(1, 2, 3)))
    vel -= vel.mean(axis=(1, 2, 3), keepdims=True)
    urms = np.sqrt(np.mean(np.sum(vel * vel, axis=0)))
    c = np.sqrt(gamma * (1.0 / gamma) / 1.0)
    vel *= mach * c / urms
    # reorder [comp][x][y][z] -> [comp][z][y][x]
    vel = np.ascontiguousarray(np.transpose(vel, (0, 3, 2, 1)))
    rho = np.ones((n, n, n))
    p = np.full((n, n, n), 1.0 / gamma)
    U = prim_to_cons(rho, [vel[0], vel[1], vel[2]], p, gamma)
    h = L / n
    return Problem(f"turbulence3d_{n}", U, (n, n, n), (h, h, h), (PERIODIC,) * 3, t_end,
                   gamma=gamma, x0=(0.0, 0.0, 0.0), extra={"mach": mach, "seed": seed})


def perturbed_target(rho: np.ndarray, scale: float = 1e-2, seed: int = 2) -> np.ndarray:
    """Seeded target density rho + scale * xi, xi ~ N(0, 1), for the adjoint loss."""
    rng = np.random.default_rng(seed)
    return rho + scale * rng.standard_normal(rho.shape)


def random_smooth_state(ndim: int, n, seed: int = 0, amp: float = 0.1) -> np.ndarray:
    """A smooth periodic positive state (sums of low sine modes) for parity tests."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    grids = np.meshgrid(*[2 * np.pi * (np.arange(m) + 0.5) / m for m in reversed(n)], indexing="ij")

    def field_():
        f = np.zeros(shape)
        for _ in range(3):
            ks = rng.integers(1, 4, size=ndim)
            ph = rng.uniform(0, 2 * np.pi)
            f += np.sin(sum(k * g for k, g in zip(ks, grids)) + ph)
        return f / 3.0

    rho = 1.0 + amp * 5 * field_() * 0.5
    rho = np.abs(rho) + 0.2
    vel = [amp * 5 * field_() for _ in range(ndim)]
    p = 1.0 + amp * 3 * field_()
    p = np.abs(p) + 0.2
    return prim_to_cons(rho, vel, p)


def random_discontinuous_state(ndim: int, n, seed: int = 0) -> np.ndarray:
    """Piecewise-constant random blocks plus noise: exercises every selector path."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    blocks = [max(1, m // 5) for m in reversed(n)]
    def blocky(lo, hi):
        coarse = rng.uniform(lo, hi, size=tuple(-(-m // b) for m, b in zip(shape, blocks)))
        f = coarse
        for ax, b in enumerate(blocks):
            f = np.repeat(f, b, axis=ax)
        f = f[tuple(slice(0, m) for m in shape)]
        return f * (1.0 + 0.02 * rng.standard_normal(shape))
    rho = blocky(0.2, 2.0)
    vel = [blocky(-1.0, 1.0) for _ in range(ndim)]
    p = blocky(0.2, 5.0)
    return prim_to_cons(rho, vel, p)
