"""Seeded synthetic workloads: parameter sets, grids and initial fields.

This module is shared by the tests, the benchmark and both implementations
(the CUDA library and the CPU oracle) as the single source of inputs.  It holds
none of the time-stepping arithmetic: only random numbers, initial-condition
recipes and the model parameters of the benchmark problem.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).
A 53-bit uniform in [0, 1) is (x >> 11) * 2**-53, mapped to U(-1, 1) as 2u - 1.
Fields are filled in the order c, eta_1 .. eta_p, each in row-major order with
x fastest, idx = (z * ny + y) * nx + x.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """U(-1, 1) doubles from the SplitMix64 stream."""
    x = splitmix64(seed, count, offset)
    return 2.0 * ((x >> np.uint64(11)).astype(np.float64) * 2.0**-53) - 1.0


@dataclasses.dataclass
class Problem:
    """Model parameters (Section 2.1 of the paper) and grid.

    Defaults are the benchmark's values: kappa_c = kappa_eta = 3, rho^2 = 2,
    c_alpha = 0.3, c_beta = 0.7, w = 1, alpha = 5, M = L = 5.
    """

    n: tuple = (64, 64)
    dx: tuple = None
    p: int = 1
    M: float = 5.0
    L: float = 5.0
    kappa_c: float = 3.0
    kappa_eta: float = 3.0
    rho2: float = 2.0
    c_alpha: float = 0.3
    c_beta: float = 0.7
    w: float = 1.0
    alpha: float = 5.0
    dt: float = 1e-3
    lap: int = 0  # 0 spectral, 1 FS-FD O(dl^2), 2 FS-FD O(dl^4)

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if self.dx is None:
            self.dx = tuple(1.0 for _ in self.n)
        self.dx = tuple(float(v) for v in self.dx)

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def npoints(self) -> int:
        return int(np.prod(self.n))

    @property
    def nf(self) -> int:
        return 1 + self.p

    @property
    def shape(self) -> tuple:
        """numpy shape of one field, slowest axis first: (nz, ny, nx)."""
        return tuple(reversed(self.n))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def fd_stable_dt(prob: Problem) -> float:
    """Largest stable dt of the explicit 5-/7-point FD scheme, linearised.

    The paper finds this bound by trial and error (Section 3).  Here it is the
    von Neumann bound of forward Euler for c_t = M lap(f_cc c - kappa_c lap c)
    with f_cc = 2 rho^2 (exact: f_chem is quadratic in c for any eta) and the
    largest eigenvalue lambda = sum_d 4/dx_d^2 of the discrete -Laplacian:
    dt = 2 / (M lambda (2 rho^2 + kappa_c lambda)).
    """
    lam = sum(4.0 / (d * d) for d in prob.dx)
    return 2.0 / (prob.M * lam * (2.0 * prob.rho2 + prob.kappa_c * lam))


def noise_fields(prob: Problem, seed: int = 0, c0: float = 0.5, eta0: float = 0.5,
                 amp: float = 0.01) -> np.ndarray:
    """c = c0 + amp U(-1,1), eta_i = eta0 + amp U(-1,1); shape (nf, *prob.shape)."""
    N = prob.npoints
    u = uniform_pm1(seed, prob.nf * N)
    base = np.array([c0] + [eta0] * prob.p, dtype=np.float64)
    f = base[:, None] + amp * u.reshape(prob.nf, N)
    return f.reshape((prob.nf,) + prob.shape)


def grid_coords(prob: Problem):
    """Coordinates x_j = j dx (periodic, excluding l), as broadcastable arrays."""
    axes = [np.arange(n) * d for n, d in zip(prob.n, prob.dx)]
    return np.meshgrid(*reversed(axes), indexing="ij")[::-1]


def cosine_mode_fields(prob: Problem, kidx, cbar: float, eps: float,
                       eta_val: float = 0.0, which: int = 0) -> np.ndarray:
    """Uniform fields plus one cosine Fourier mode of integer wavenumber kidx
    on field `which` (0 = c).  Used by the linear-stability checks."""
    coords = grid_coords(prob)
    phase = np.zeros(prob.shape)
    for k, x, n, d in zip(kidx, coords, prob.n, prob.dx):
        phase = phase + 2.0 * math.pi * k * x / (n * d)
    f = np.empty((prob.nf,) + prob.shape)
    f[0] = cbar
    for i in range(prob.p):
        f[1 + i] = eta_val
    f[which] = f[which] + eps * np.cos(phase)
    return f


def tanh_slab_fields(prob: Problem, a: float, b: float, width: float,
                     c_val: float = 0.5) -> np.ndarray:
    """p = 1 slab eta = (tanh((x-a)/width) - tanh((x-b)/width)) / 2 along x."""
    coords = grid_coords(prob)
    x = coords[0]
    f = np.empty((prob.nf,) + prob.shape)
    f[0] = c_val
    f[1] = 0.5 * (np.tanh((x - a) / width) - np.tanh((x - b) / width))
    return f


def benchmark_ic_fields(prob: Problem, c0: float = 0.5, eps: float = 0.05, eta_nu: float = 0.1,
                        psi: float = 1.5) -> np.ndarray:
    """The 2D benchmark initial condition of Section 3 (Eqs. ic_c and ic_eta),
    sampled at x = j dx, y = k dx, for eta_i with i = 1..p:

      c     = c0 + eps [cos(.105x)cos(.11y) + (cos(.13x)cos(.087y))^2
                        + cos(.025x - .15y)cos(.07x - .02y)]
      eta_i = eta_nu {cos(.01i x - 4)cos((.007 + .01i)y)
                      + cos((.11 + .01i)x)cos((.11 + .01i)y)
                      + psi [cos((.046 + .001i)x + (.0405 + .001i)y)
                             cos((.031 + .001i)x - (.004 + .001i)y)]^2}^2

    The fields are not periodic on the grid; Section 3 smooths them with the
    explicit FD scheme up to t = 1 before use (done by the caller)."""
    if prob.ndim != 2:
        raise ValueError("the benchmark initial condition is two-dimensional")
    x, y = grid_coords(prob)
    f = np.empty((prob.nf,) + prob.shape)
    f[0] = c0 + eps * (np.cos(0.105 * x) * np.cos(0.11 * y)
                       + (np.cos(0.13 * x) * np.cos(0.087 * y)) ** 2
                       + np.cos(0.025 * x - 0.15 * y) * np.cos(0.07 * x - 0.02 * y))
    for i in range(1, prob.p + 1):
        a = np.cos(0.01 * i * x - 4.0) * np.cos((0.007 + 0.01 * i) * y)
        b = np.cos((0.11 + 0.01 * i) * x) * np.cos((0.11 + 0.01 * i) * y)
        q = (np.cos((0.046 + 0.001 * i) * x + (0.0405 + 0.001 * i) * y)
             * np.cos((0.031 + 0.001 * i) * x - (0.004 + 0.001 * i) * y))
        f[i] = eta_nu * (a + b + psi * q * q) ** 2
    return f


def extrude_3d(fields2d: np.ndarray, nz: int, dz: float = 1.0, c0: float = 0.5,
               zscale: float = 5.0, power: int = 4, clip: float = 1e-9) -> np.ndarray:
    """3D fields from a 2D state (Eq. ic_eta_3d): c = c0 everywhere and

      eta_i(x, y, z) = (1 + tanh(artanh(2 eta_i^2D(x, y) - 1) - ((z - lz/2)/zscale)^power)) / 2,

    lz = nz dz.  The 2D field is taken index by index (the paper's (2x, 2y)
    maps its 200-wide 2D domain onto the 100-wide cube; here both grids have
    the same number of points per axis).  2 eta - 1 is clipped to
    [-1 + clip, 1 - clip] so artanh stays finite.  Shape (nf, nz, ny, nx)."""
    nf, ny, nx = fields2d.shape
    z = (np.arange(nz) * dz - 0.5 * nz * dz)[:, None, None]
    out = np.empty((nf, nz, ny, nx))
    out[0] = c0
    for i in range(1, nf):
        a = np.arctanh(np.clip(2.0 * fields2d[i] - 1.0, -1.0 + clip, 1.0 - clip))
        out[i] = 0.5 * (1.0 + np.tanh(a[None, :, :] - (z / zscale) ** power))
    return out


def batch_problems(count: int, seed: int = 0, sizes=(128, 256, 512, 1024), p: int = 2,
                   spread: float = 0.5, dt_factor: float = 5.0):
    """Ensemble of 2D problems: size uniform from `sizes` (square grids) and
    M, L, kappa_c, kappa_eta each the benchmark value times
    exp(U(ln(1-spread), ln(1+spread))); dt = dt_factor x the FD-stable dt of
    each member."""
    draws = uniform_pm1(seed ^ 0x5EED, 5 * count).reshape(count, 5)
    lo, hi = math.log(1.0 - spread), math.log(1.0 + spread)
    out = []
    for i in range(count):
        u = (draws[i] + 1.0) / 2.0  # [0, 1)
        n = sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)]
        sc = [math.exp(lo + (hi - lo) * v) for v in u[1:]]
        pr = Problem(n=(n, n), p=p, M=5.0 * sc[0], L=5.0 * sc[1], kappa_c=3.0 * sc[2],
                     kappa_eta=3.0 * sc[3])
        pr.dt = dt_factor * fd_stable_dt(pr)
        out.append(pr)
    return out
