"""Seeded synthetic inputs for the staggered P_N step: media fields and initial moments.

This module holds none of the method's arithmetic (no coupling, no differences, no substep
factors).  It only produces the per-cell arrays that both the CUDA path and the CPU oracle take as
inputs, so that the two sides are fed bit-identical data.  Every array is FP64, laid out
``[z, y, x]`` (media, one moment) or ``[c, z, y, x]`` (a full state, c = l*l + l + m).

Workloads (the paper has no public data set; its only geometry, the reactor showcase of Section
5.2, is given only in a figure, so these synthetic media stand in for its lattice-type problems):

  * ``gaussian_pulse``  periodic unit cube, homogeneous scatterer, Gaussian u_0 of unit sum;
  * ``checkerboard``    the 7^3-block lattice on [0,7]^3 (absorbers sigma_a = 10 in a
                        checkerboard over the interior 5^3, scatterers sigma_s = 1 elsewhere,
                        a source q = 1 in u_0 on the central block), vacuum boundaries;
  * ``random_blocks``   sigma_s log-uniform in [0.1, 10], constant per 8^3 block, sigma_a = 0.01;
  * ``reactor_like``    a stand-in for the reactor showcase of Section 5.2: fuel rods 5 cells
                        (1 length unit) thick with source q = 2 in water (sigma_a = 10) inside a
                        concrete shell (sigma_a = 5), sigma_s = 1 everywhere, vacuum boundaries;
  * ``random_state`` / ``random_media``  dense random fields for parity tests.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Instance:
    """One problem: order N, cubic grid n^3 (or nz, ny, nx), media, initial u_0, boundary."""

    N: int
    shape: tuple          # (nz, ny, nx)
    h: float
    dt: float
    bc: str               # "periodic" | "vacuum"
    sigma_a: np.ndarray
    sigma_s: np.ndarray
    q: np.ndarray
    u0: np.ndarray        # initial zeroth moment [z, y, x]; every other moment starts at 0
    name: str = ""

    @property
    def n_c(self) -> int:
        return (self.N + 1) ** 2

    def full_state(self) -> np.ndarray:
        u = np.zeros((self.n_c,) + tuple(self.shape))
        u[0] = self.u0
        return u


def cell_centres(n: int, L: float) -> np.ndarray:
    """Centres (i + 1/2) h of n cells on [0, L]."""
    return (np.arange(n) + 0.5) * (L / n)


def gaussian(n: int, width: float, L: float = 1.0, centre: float = 0.5) -> np.ndarray:
    """exp(-|x - centre|^2 / (2 width^2)) at the cell centres (Euclidean distance), unit sum."""
    x = cell_centres(n, L)
    g1 = np.exp(-((x - centre * L) ** 2) / (2.0 * width**2))
    g = g1[:, None, None] * g1[None, :, None] * g1[None, None, :]
    return g / g.sum()


def lattice_blocks(n: int, L: float = 7.0):
    """Block index floor(centre) in 0..6 of every cell along one axis of the [0,7]^3 lattice."""
    return np.minimum(np.floor(cell_centres(n, L)).astype(np.int64), int(L) - 1)


def checkerboard_media(n: int):
    """sigma_a, sigma_s, q of the 7^3 lattice at n^3 cells.

    Absorber (sigma_a = 10, sigma_s = 0) iff the block is inside the interior 5^3 (indices 1..5 on
    every axis), bx + by + bz is odd (the parity of the interior corners) and it is not the central
    block (3,3,3).  The central block is a scatterer with q = 1; every other block is a scatterer
    (sigma_s = 1, sigma_a = 0).
    """
    b = lattice_blocks(n)
    BZ, BY, BX = np.meshgrid(b, b, b, indexing="ij")
    interior = (BX >= 1) & (BX <= 5) & (BY >= 1) & (BY <= 5) & (BZ >= 1) & (BZ <= 5)
    centre = (BX == 3) & (BY == 3) & (BZ == 3)
    absorber = interior & ((BX + BY + BZ) % 2 == 1) & ~centre
    sigma_a = np.where(absorber, 10.0, 0.0)
    sigma_s = np.where(absorber, 0.0, 1.0)
    q = np.where(centre, 1.0, 0.0)
    return sigma_a, sigma_s, q


def gaussian_pulse(N: int, n: int, width: float = 0.08, sigma_s: float = 1.0,
                   sigma_a: float = 0.0, name: str = "gaussian") -> Instance:
    """Periodic [0,1]^3, h = 1/n, dt = 0.3 h, homogeneous media, Gaussian u_0 of unit sum."""
    h = 1.0 / n
    shape = (n, n, n)
    return Instance(N, shape, h, 0.3 * h, "periodic",
                    np.full(shape, sigma_a), np.full(shape, sigma_s), np.zeros(shape),
                    gaussian(n, width), name)


def checkerboard(N: int, n: int, name: str = "checkerboard") -> Instance:
    """The [0,7]^3 lattice at n^3 cells, h = 7/n, dt = 0.3 h, vacuum, zero initial state."""
    h = 7.0 / n
    sa, ss, q = checkerboard_media(n)
    return Instance(N, (n, n, n), h, 0.3 * h, "vacuum", sa, ss, q, np.zeros((n, n, n)), name)


def random_blocks(N: int, n: int, seed: int = 2, block: int = 8, name: str = "random_blocks") -> Instance:
    """Periodic [0,1]^3: sigma_s = exp(U(ln 0.1, ln 10)) per block^3 (draws in block order
    bz, by, bx), sigma_a = 0.01, q = 0, Gaussian u_0 of width 0.1 and unit sum."""
    rng = np.random.default_rng(seed)
    nb = -(-n // block)
    vals = np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=(nb, nb, nb)))
    idx = np.arange(n) // block
    ss = vals[idx[:, None, None], idx[None, :, None], idx[None, None, :]]
    h = 1.0 / n
    shape = (n, n, n)
    return Instance(N, shape, h, 0.3 * h, "periodic", np.full(shape, 0.01), ss,
                    np.zeros(shape), gaussian(n, 0.1), name)


def reactor_media(n: int, shell: int | None = None, rod: int = 5, pitch: int = 10):
    """sigma_a, sigma_s, q of the reactor-like cube at n^3 cells.

    The paper's figure of the geometry is not available, so this is a reading of its text: a
    concrete shell of `shell` cells (default n // 16, at least 1) on every face (sigma_a = 5); inside
    it water (sigma_a = 10); a core in the middle half of the inner box in x and y and its middle
    three quarters in z holds fuel rods along z, `rod` x `rod` cells each on a `pitch`-cell lattice
    (source q = 2, no absorption).  sigma_s = 1 everywhere.
    """
    shell = max(1, n // 16) if shell is None else shell
    i = np.arange(n)
    inner = (i >= shell) & (i < n - shell)
    w = n - 2 * shell
    core_xy = (i >= shell + w // 4) & (i < n - shell - w // 4)
    core_z = (i >= shell + w // 8) & (i < n - shell - w // 8)
    rod_xy = core_xy & (((i - shell - w // 4) % pitch) < rod)
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    inside = inner[Z] & inner[Y] & inner[X]
    fuel = rod_xy[X] & rod_xy[Y] & core_z[Z] & inside
    sigma_a = np.where(inside, 10.0, 5.0)
    sigma_a = np.where(fuel, 0.0, sigma_a)
    sigma_s = np.ones((n, n, n))
    q = np.where(fuel, 2.0, 0.0)
    return sigma_a, sigma_s, q


def reactor_like(N: int, n: int, h: float = 0.2, name: str = "reactor_like") -> Instance:
    """The reactor-like cube (``reactor_media``) at n^3 cells of size h (1 length unit = 5 cells),
    dt = 0.3 h, vacuum boundaries, zero initial state."""
    sa, ss, q = reactor_media(n)
    return Instance(N, (n, n, n), h, 0.3 * h, "vacuum", sa, ss, q, np.zeros((n, n, n)), name)


def batch_instances(count: int = 64, seed: int = 3, orders=(1, 3, 5, 9, 15),
                    side_range=(24, 96)) -> list[Instance]:
    """Independent instances: N uniform over `orders`, side uniform on `side_range` (inclusive),
    media kind by a fair coin (Gaussian pulse rules or checkerboard rules)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice(orders))
        n = int(rng.integers(side_range[0], side_range[1] + 1))
        if rng.integers(0, 2) == 0:
            out.append(gaussian_pulse(N, n, name=f"b{i}-gauss"))
        else:
            out.append(checkerboard(N, n, name=f"b{i}-checker"))
    return out


def detector_box(n: int = 96) -> np.ndarray:
    """Detector weights: 1 on cells x in [70, 82), y, z in [42, 54) (inside block (5,3,3) at 96^3)."""
    w = np.zeros((n, n, n))
    s = n / 96.0
    x0, x1 = int(round(70 * s)), int(round(82 * s))
    y0, y1 = int(round(42 * s)), int(round(54 * s))
    w[y0:y1, y0:y1, x0:x1] = 1.0
    return w


def random_media(shape, seed: int, lo: float = 0.0, hi: float = 2.0):
    rng = np.random.default_rng(seed)
    sa = rng.uniform(lo, hi, size=shape)
    ss = rng.uniform(lo, hi, size=shape)
    q = rng.uniform(0.0, 1.0, size=shape)
    return sa, ss, q


def random_state(N: int, shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(((N + 1) ** 2,) + tuple(shape))


def random_instance(N: int, shape, seed: int, bc: str = "periodic", h: float = 0.1,
                    dt_ratio: float = 0.3) -> tuple[Instance, np.ndarray]:
    """Random media and a dense random state on an arbitrary (nz, ny, nx) grid."""
    sa, ss, q = random_media(shape, seed)
    u = random_state(N, shape, seed + 1000)
    inst = Instance(N, tuple(shape), h, dt_ratio * h, bc, sa, ss, q, u[0], f"random-{seed}")
    return inst, u
