"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds geometry and random numbers only: it evaluates no part of
the scattering method (no polarizability, Green function, FFT, circulant or
solver arithmetic).  Both the CPU oracle and the CUDA path receive the arrays
made here as inputs.

Conventions
-----------
* A box of ``l x m x n`` voxels (edges along x, y, z) is stored as a C-order
  array of shape ``(n, m, l)``: x is the fastest index, matching the loop order
  of the paper's Algorithm 1 (Section 2.2).
* Voxel centres are ``r = dx * (i - (l-1)/2, j - (m-1)/2, k - (n-1)/2)``
  (box centred on the origin).
* Material index per voxel: 0 = air, 1..K = material ``K`` (ice = 1).
* The scatterer of the paper's experiments is a hexagonal prism (Section 4):
  hexagon of circumradius ``a_h`` in the xy-plane with corners on the +-x
  axis, prism axis along z, height ``L``.  A voxel belongs to the prism when
  its centre does (ties inside, with a 1e-9*dx slack).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "voxel_centres", "hex_prism_mask", "sphere_mask", "prism_box",
    "random_direction", "polarisations", "random_field", "PrismCase",
    "small_prism_case", "prism_case", "config2_cases", "pad_box", "next_pow2",
    "uneven_batch_cases",
]


def voxel_centres(l: int, m: int, n: int, dx: float) -> np.ndarray:
    """Centres of an l x m x n box centred on the origin, shape (n, m, l, 3)."""
    x = (np.arange(l) - (l - 1) / 2.0) * dx
    y = (np.arange(m) - (m - 1) / 2.0) * dx
    z = (np.arange(n) - (n - 1) / 2.0) * dx
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([xx, yy, zz], axis=-1)


def hex_prism_mask(l: int, m: int, n: int, dx: float, a_h: float, height: float,
                   material: int = 1) -> np.ndarray:
    """uint8 (n, m, l) material index of a centred hexagonal prism."""
    r = voxel_centres(l, m, n, dx)
    ax, ay, az = np.abs(r[..., 0]), np.abs(r[..., 1]), np.abs(r[..., 2])
    s3 = math.sqrt(3.0)
    eps = 1e-9 * dx
    inside = ((ay <= 0.5 * s3 * a_h + eps)
              & (s3 * ax + ay <= s3 * a_h + eps)
              & (az <= 0.5 * height + eps))
    return np.where(inside, np.uint8(material), np.uint8(0)).astype(np.uint8)


def sphere_mask(l: int, m: int, n: int, dx: float, radius: float,
                material: int = 1) -> np.ndarray:
    """uint8 (n, m, l) material index of a centred sphere."""
    r = voxel_centres(l, m, n, dx)
    inside = (r ** 2).sum(-1) <= radius * radius + 1e-9 * dx
    return np.where(inside, np.uint8(material), np.uint8(0)).astype(np.uint8)


def prism_box(N: int, aspect: float) -> tuple[int, int, int]:
    """Box edges (l, m, n) for a prism N voxels across its corners.

    The hexagon spans 2*a_h = N*dx along x; the box is N x N in the plane and
    ``round(aspect*N)`` voxels high, aspect = L / (2 a_h).
    """
    return N, N, max(1, int(round(aspect * N)))


def random_direction(rng: np.random.Generator) -> np.ndarray:
    """Unit vector from a normalised standard-normal draw."""
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def polarisations(d: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Two unit polarisations orthogonal to the unit direction d.

    e1 = normalise(d x z) (x if d is parallel to z), e2 = d x e1.
    """
    d = np.asarray(d, dtype=np.float64)
    e1 = np.cross(d, np.array([0.0, 0.0, 1.0]))
    nrm = np.linalg.norm(e1)
    if nrm < 1e-12:
        e1 = np.array([1.0, 0.0, 0.0])
    else:
        e1 = e1 / nrm
    e2 = np.cross(d, e1)
    return e1, e2 / np.linalg.norm(e2)


def random_field(shape, rng: np.random.Generator, dtype=np.complex128) -> np.ndarray:
    """Complex standard-normal array (real and imaginary parts independent)."""
    out = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return out.astype(dtype)


def pad_box(mat: np.ndarray, l: int, m: int, n: int) -> np.ndarray:
    """Embed an (n0, m0, l0) material array centred in a larger air box.

    The shift keeps voxel centres on the same lattice; the offsets are even
    so that ``voxel_centres`` of the padded box coincides with the original
    centres when each added margin is even.
    """
    n0, m0, l0 = mat.shape
    out = np.zeros((n, m, l), dtype=mat.dtype)
    oz, oy, ox = (n - n0) // 2, (m - m0) // 2, (l - l0) // 2
    out[oz:oz + n0, oy:oy + m0, ox:ox + l0] = mat
    return out


@dataclass
class PrismCase:
    """One synthetic scattering problem on a hexagonal prism."""
    N: int                      # voxels across the hexagon's corners
    size_param: float           # x = k a_h
    eps: list                   # complex permittivity per material (eps = m^2)
    aspect: float = 1.0         # L / (2 a_h)
    a_h: float = 1.0            # hexagon circumradius (length unit)
    dirs: list = field(default_factory=lambda: [np.array([0.0, 0.0, 1.0])])
    pols: list = field(default_factory=lambda: [np.array([1.0, 0.0, 0.0])])

    box: tuple | None = None    # (l, m, n) air-padded box; None: the prism's own box

    @property
    def dims(self) -> tuple[int, int, int]:
        return tuple(self.box) if self.box is not None else prism_box(self.N, self.aspect)

    @property
    def dx(self) -> float:
        return 2.0 * self.a_h / self.N

    @property
    def k(self) -> float:
        return self.size_param / self.a_h

    def mask(self) -> np.ndarray:
        l, m, n = self.dims
        return hex_prism_mask(l, m, n, self.dx, self.a_h, 2.0 * self.aspect * self.a_h)

    @property
    def nrhs(self) -> int:
        return len(self.dirs)


def prism_case(N: int, size_param: float, m_index: complex, aspect: float = 1.0,
               dirs=None, pols=None) -> PrismCase:
    """Prism with one material of refractive index m (eps = m^2)."""
    c = PrismCase(N=N, size_param=size_param, eps=[complex(m_index) ** 2], aspect=aspect)
    if dirs is not None:
        c.dirs = [np.asarray(d, dtype=np.float64) for d in dirs]
        c.pols = [np.asarray(p, dtype=np.float64) for p in pols]
    return c


def small_prism_case() -> PrismCase:
    """16^3 prism, x = 5, m = 1.31, +z incidence, x-polarised."""
    return prism_case(16, 5.0, 1.31, 1.0)


def config2_cases(N: int = 64, size_param: float = 20.0, seed: int = 0):
    """The 3 refractive indices x 3 aspects sweep, one seeded direction, 2 polarisations.

    Returns a list of PrismCase, each with two right-hand sides (e1, e2).
    """
    rng = np.random.default_rng(seed)
    d = random_direction(rng)
    e1, e2 = polarisations(d)
    cases = []
    for m_index in (1.31, 1.31 + 0.05j, 1.78):
        for aspect in (0.5, 1.0, 2.0):
            cases.append(prism_case(N, size_param, m_index, aspect,
                                    dirs=[d, d], pols=[e1, e2]))
    return cases


def next_pow2(v: int) -> int:
    """Smallest power of two >= v."""
    p = 1
    while p < v:
        p *= 2
    return p


def next_even_smooth(v: int) -> int:
    """Smallest even 7-smooth number (2^a 3^b 5^c 7^d, a >= 1) >= v."""
    e = max(2, v + (v % 2))
    while True:
        r = e
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        if r == 1:
            return e
        e += 2


def uneven_batch_cases(count: int = 32, seed: int = 2, kd: float = 0.6, pad_pow2: bool = True,
                       pad_smooth: bool = False):
    """An uneven batch of prisms: edges N_i drawn uniformly from 24..96, size
    parameter x_i = kd N_i / 2 (voxel size k dx = kd), refractive index
    U[1.3, 1.8] + i U[0, 0.1], aspect 1, +z incidence, x-polarised.  With
    pad_pow2 each prism sits centred in the power-of-two box that holds it,
    with pad_smooth in the smallest box of even 7-smooth edges (air padding)."""
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(count):
        N = int(rng.integers(24, 97))
        m_index = complex(rng.uniform(1.3, 1.8), rng.uniform(0.0, 0.1))
        c = prism_case(N, kd * N / 2.0, m_index, 1.0)
        if pad_smooth:
            L = next_even_smooth(N)
            c.box = (L, L, L)
        elif pad_pow2:
            L = next_pow2(N)
            c.box = (L, L, L)
        cases.append(c)
    return cases
